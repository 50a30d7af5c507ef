"""Pins of the learned-closure oracle (no GPU): BF16 rounding and the activations against
torch's own routines, the hand-derived backward against finite differences, Adam
against torch.optim.Adam, and the features / label on flows with known answers."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as ML
from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for


def test_bf16_rounding_matches_torch_including_ties():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-30, 30, 100000))).astype(np.float32)
    # exact ties: midpoints between consecutive bfloat16 values
    b = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    up = (b.view(np.uint32) + 0x10000).view(np.float32)
    ties = ((b.astype(np.float64) + up.astype(np.float64)) / 2).astype(np.float32)
    for arr in (x, ties):
        ref = torch.from_numpy(arr).to(torch.bfloat16).float().numpy().astype(np.float64)
        got = ML.bf16(arr)
        assert np.array_equal(got, ref)


def test_activations_match_torch():
    z = np.linspace(-8, 8, 2001)
    t = torch.from_numpy(z)
    np.testing.assert_allclose(ML.gelu(z), torch.nn.functional.gelu(t).numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ML.softplus(z), torch.nn.functional.softplus(t).numpy(), rtol=1e-12,
                               atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(ML.gelu_grad(z), (ML.gelu(z + h) - ML.gelu(z - h)) / (2 * h), rtol=1e-6,
                               atol=1e-9)
    np.testing.assert_allclose(ML.softplus_grad(z), (ML.softplus(z + h) - ML.softplus(z - h)) / (2 * h),
                               rtol=1e-6, atol=1e-9)


def test_backward_matches_finite_differences():
    p = ML.init_params(1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, ML.NIN))
    t = np.abs(rng.standard_normal(40))
    L, g = ML.loss_and_grads(p, X, t, quantize=False)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k].reshape(-1)[idx] += h
            pm[k].reshape(-1)[idx] -= h
            fd = (ML.loss_and_grads(pp, X, t, False)[0] - ML.loss_and_grads(pm, X, t, False)[0]) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-8), (k, idx, fd, an)


def test_forward_matches_torch_network():
    """The FP64 network equals the same network written with torch.nn layers."""
    p = ML.init_params(3)
    X = np.random.default_rng(4).standard_normal((17, ML.NIN))
    net = torch.nn.Sequential(torch.nn.Linear(14, 64), torch.nn.GELU(), torch.nn.Linear(64, 64),
                              torch.nn.GELU(), torch.nn.Linear(64, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"].T))
        net[0].bias.copy_(torch.from_numpy(p["b1"]))
        net[2].weight.copy_(torch.from_numpy(p["W2"].T))
        net[2].bias.copy_(torch.from_numpy(p["b2"]))
        net[4].weight.copy_(torch.from_numpy(p["w3"][None, :]))
        net[4].bias.copy_(torch.from_numpy(np.atleast_1d(p["b3"])))
        ref = net(torch.from_numpy(X)).numpy()[:, 0]
    y, _, _ = ML.forward(p, X, quantize=False)
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-14)


def test_adam_matches_torch_optimizer():
    p = ML.init_params(5)
    g = {k: np.random.default_rng(6).standard_normal(v.shape) for k, v in p.items()}
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-3)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(vv) for k, vv in p.items()}
    for step in (1, 2, 3):
        for k in tp:
            tp[k].grad = torch.tensor(g[k] * step)
        opt.step()
        p, m, v = ML.adam_step(p, {k: g[k] * step for k in g}, m, v, step)
    for k in p:
        np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-15)


def test_features_uniform_flow_and_linear_shear():
    g = 1.4
    rho = np.ones((4, 6, 8))
    u = np.stack([0.5 * rho, 0 * rho, 0 * rho])
    w = synth._conservative(rho, u, rho / g, g)
    P = params_for(w)
    assert np.all(ML.features(w, P) == 0.0)
    # periodic shear u1 = A sin(2 pi y / Ly): du1/dy at the cells, v1 = u1 - mean
    ny = 16
    y = (np.arange(ny) + 0.5) / 8.0
    A = 0.1
    rho = np.ones((2, ny, 8))
    u1 = A * np.sin(2 * np.pi * y / 2.0)[None, :, None] * np.ones_like(rho)
    w = synth._conservative(rho, np.stack([u1, 0 * rho, 0 * rho]), rho / g, g)
    P = params_for(w)
    f = ML.features(w, P).reshape(2, ny, 8, 14)
    cb = 1.0
    np.testing.assert_allclose(f[..., 1], u1 / cb, atol=1e-15)
    dy = P.dx[1]
    exact_central = A * (np.sin(2 * np.pi * (y + dy) / 2.0) - np.sin(2 * np.pi * (y - dy) / 2.0)) / (2 * dy)
    np.testing.assert_allclose(f[0, :, 0, 5 + 0 * 3 + 1], exact_central, rtol=1e-12, atol=1e-14)
    assert np.all(np.abs(f[..., [0, 4]]) < 1e-14)


def test_label_zero_for_uniform_flow_and_nonnegative():
    w = synth.perturbed_uniform(6, 5, 4, seed=7, amp=0.1)
    P = params_for(w)
    lam = synth.random_field(w.shape, 8)
    r = ML.label_rate(w, lam, P)
    assert np.all(r >= 0.0) and np.all(np.isfinite(r))
    g = 1.4
    rho = np.ones((3, 4, 5))
    wu = synth._conservative(rho, np.stack([0.5 * rho, 0 * rho, 0 * rho]), rho / g, g)
    assert np.all(ML.label_rate(wu, lam[:, :3, :4, :5], params_for(wu)) == 0.0)


@pytest.mark.parametrize("nz", [1, 3])
def test_label_closed_form_on_a_sinusoidal_shear(nz):
    """Uniform rho and p with u1 = A sin(k_y y): a and b are uniform and div u = 0, so
    M1 = 0 and M = -M2 has one entry, -du1/dy, in row u1, column u2 (the printed M2's
    velocity block).  Its central difference is exactly A cos(k_y y) sin(k_y h_y) / h_y.  With
    v_hat = (0, B sin(k_x x), C, D sin(k_x x), 0) the label is
    max(0, v_hat^T M v_hat) / |grad v_hat|^2 = max(0, -G B C sin(k_x x)) / (B'^2 (cos(k_x x)
    sin(k_x h_x) / h_x)^2), with B'^2 = B^2 in 2D (the u3 component is outside the
    (rho, u1, u2, p) block) and B^2 + D^2 in 3D."""
    g = 1.4
    nx, ny = 12, 8
    hx, hy, hz = 1.0 / nx, 1.5 / nx, 2.0 / nx   # unequal, so a mixed-up axis shows
    A, B, C, D = 0.3, 0.7, -1.3, 0.9
    ky = 2 * math.pi / (ny * hy)
    kx = 2 * math.pi / (nx * hx)
    y = (np.arange(ny) + 0.5) * hy
    x = (np.arange(nx) + 0.5) * hx
    Y = np.broadcast_to(y[None, :, None], (nz, ny, nx))
    X = np.broadcast_to(x[None, None, :], (nz, ny, nx))
    rho = np.full((nz, ny, nx), 1.2)
    u = np.stack([A * np.sin(ky * Y), np.zeros_like(rho), np.zeros_like(rho)])
    w = synth._conservative(rho, u, np.full_like(rho, 0.8 / g), g)
    P = params_for(w)
    P.dx = (hx, hy, hz)
    vh = np.stack([np.zeros_like(rho), B * np.sin(kx * X), np.full_like(rho, C), D * np.sin(kx * X),
                   np.zeros_like(rho)])
    # lam = T^T v_hat, so that the label's own T^{-T} lam gives v_hat back
    T = O.transform_T(w, P)
    lam = np.moveaxis(np.einsum("...ji,...j->...i", T, np.moveaxis(vh, 0, -1)), -1, 0)
    G = A * np.cos(ky * Y) * math.sin(ky * hy) / hy
    B2 = B * B if nz == 1 else B * B + D * D
    grad2 = B2 * (np.cos(kx * X) * math.sin(kx * hx) / hx) ** 2
    expect = np.maximum(-G * B * C * np.sin(kx * X), 0.0) / grad2
    got = ML.label_rate(w, lam, P)
    np.testing.assert_allclose(got, expect, rtol=1e-10, atol=1e-12 * expect.max())
    assert np.count_nonzero(expect) > expect.size // 4   # both signs of the growth occur


def test_bf16_backward_moves_each_gradient_within_its_rounding_bound():
    """Rounding dZ2 and dZ1 to BF16 before the products they enter leaves the loss and
    the gradients that do not pass through them (w3, b3, b2) unchanged, and moves every
    weight-gradient entry by at most its products' magnitudes times the BF16 unit
    roundoff 2^-8 (8 significant bits, round to nearest: one rounding per product for
    W2; for W1, the rounding of dZ1 plus the propagated rounding of dZ2 through dH1)."""
    rng = np.random.default_rng(21)
    X = rng.standard_normal((96, ML.NIN))
    t = np.abs(rng.standard_normal(96))
    p = ML.init_params(22)
    L0, g0 = ML.loss_and_grads(p, X, t, True, bf16_backward=False)
    L1, g1 = ML.loss_and_grads(p, X, t, True, bf16_backward=True)
    assert L0 == L1
    for k in ("w3", "b3", "b2"):
        assert np.array_equal(g0[k], g1[k]), k
    u = 2.0 ** -8
    _, _, c = ML.forward(p, X, True)
    y = c["y"]
    dy = 2.0 * (ML.softplus(y) - t) / X.shape[0] * ML.softplus_grad(y)
    dZ2 = np.outer(dy, ML.bf16(p["w3"])) * ML.gelu_grad(c["Z2"])
    bound_W2 = np.abs(c["H1q"]).T @ np.abs(dZ2) * u
    assert np.all(np.abs(g1["W2"] - g0["W2"]) <= bound_W2 * (1 + 1e-9) + 1e-300)
    assert not np.array_equal(g1["W2"], g0["W2"])          # the rounding is really there
    dH1_abs = np.abs(dZ2) @ np.abs(ML.bf16(p["W2"])).T
    dZ1_abs = dH1_abs * np.abs(ML.gelu_grad(c["Z1"]))
    bound_W1 = np.abs(c["X0"]).T @ (dZ1_abs * (2 * u + u * u))
    assert np.all(np.abs(g1["W1"] - g0["W1"]) <= bound_W1 * (1 + 1e-9) + 1e-300)
    bound_b1 = np.sum(dZ1_abs * u, axis=0)
    assert np.all(np.abs(g1["b1"] - g0["b1"]) <= bound_b1 * (1 + 1e-9) + 1e-300)
