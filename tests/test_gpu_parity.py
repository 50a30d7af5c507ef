"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle, element by
element, on seeded inputs that span several tiles (32 x 4 columns per CTA) with ragged
edges, 2D and 3D boxes, batches, and the degenerate sizes (one plane, boxes smaller
than a tile).

Tolerances: FP64 mode must match the oracle to 1e-10 relative L2 (single operators are
held to 1e-12); mixed mode (FP32 fluxes, FP64 accumulation) to 1e-4 over a short
horizon.  Float outputs (sigma_1, nu) are compared at float precision."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

SHAPES = [(7, 5, 3), (37, 9, 5), (40, 12, 1), (3, 2, 1), (33, 5, 6)]


def _api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_06959_gb300 import api, build
    import os
    if not os.path.exists(build.OUT):
        build.build()
    return api


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_solver(api, w, P, precision=0, batch=1):
    nz, ny, nx = w.shape[-3:]
    return api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt,
                      precision=precision, plane_i=P.plane_i, pt_in=P.pt_in, batch=batch)


def state(shape, seed, amp=0.05):
    return synth.perturbed_uniform(*shape, seed=seed, amp=amp)


@pytest.mark.parametrize("shape", SHAPES)
def test_rhs_fp64(shape):
    api = _api()
    w = state(shape, 1)
    P = params_for(w, mu=0.02)
    s = synth.random_field(w.shape, 2, 0.1)
    S = make_solver(api, w, P)
    R = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs(dev(w), R, dev(s))
    ref = O.residual(w, P, s)
    assert rel_l2(host(R), ref) < 1e-12


@pytest.mark.parametrize("shape", SHAPES)
def test_rhs_transpose_fp64(shape):
    api = _api()
    w = state(shape, 3)
    P = params_for(w, mu=0.02)
    a = synth.random_field(w.shape, 4)
    S = make_solver(api, w, P)
    out = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs_transpose(dev(w), dev(a), out)
    ref = O.residual_transpose(w, a, P)
    assert rel_l2(host(out), ref) < 1e-12


@pytest.mark.parametrize("shape", [(7, 5, 3), (37, 9, 5), (40, 12, 1)])
def test_rhs_tangent_fp64(shape):
    api = _api()
    w = state(shape, 5)
    P = params_for(w, mu=0.02)
    v = synth.random_field(w.shape, 6)
    S = make_solver(api, w, P)
    out = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs_tangent(dev(w), dev(v), out)
    assert rel_l2(host(out), O.residual_tangent(w, v, P)) < 1e-12


def test_uniform_flow_rhs_is_exactly_zero_on_gpu():
    api = _api()
    g = 1.4
    rho = np.full((3, 9, 37), 1.2)
    u = np.stack([0.8 * rho, -0.1 * rho, 0.3 * rho]) / rho
    w = synth._conservative(rho, u, np.full_like(rho, 0.7), g)
    P = params_for(w, mu=0.05)
    for prec in (0, 1):
        S = make_solver(api, w, P, prec)
        R = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        S.rhs(dev(w), R)
        assert torch.count_nonzero(R).item() == 0


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1)])
def test_primal_step_fp64_multistep(shape):
    api = _api()
    w0 = state(shape, 7, 0.05)
    P = params_for(w0, mu=0.02, dt=2e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.random_field(w0.shape[1:], 8)
    S = make_solver(api, w0, P)
    a = dev(w0)
    b = torch.empty_like(a)
    sd = dev(s)
    w = w0
    for _ in range(10):
        S.primal_step(a, b, sd)
        a, b = b, a
        w, _ = O.rk4_step(w, P, s)
    assert rel_l2(host(a), w) < 1e-12


def test_batched_boxes_are_independent():
    api = _api()
    shape = (33, 6, 4)
    ws = np.stack([state(shape, 10 + i) for i in range(3)])
    P = params_for(ws[0], mu=0.02, dt=2e-3)
    S = make_solver(api, ws[0], P, batch=3)
    a = dev(ws)
    b = torch.empty_like(a)
    S.primal_step(a, b)
    got = host(b)
    for i in range(3):
        ref, _ = O.rk4_step(ws[i], P)
        assert rel_l2(got[i], ref) < 1e-12


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1), (7, 5, 3)])
def test_adjoint_step_fp64_with_viscosity_and_source_seed(shape):
    api = _api()
    w = state(shape, 11)
    P = params_for(w, mu=0.02, dt=2e-3)
    lam = synth.random_field(w.shape, 12)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 13))).astype(np.float32)
    S = make_solver(api, w, P)
    lo = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    sb = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    S.adjoint_step(dev(w), dev(lam), lo, nu=dev(nu), sbar=sb)
    ref, sref = O.rk4_adjoint_step(w, lam, P, None, nu.astype(np.float64))
    assert rel_l2(host(lo), ref) < 1e-12
    assert rel_l2(host(sb), sref) < 1e-12
    lo2 = torch.empty_like(lo)
    S.adjoint_step(dev(w), dev(lam), lo2)
    ref2, _ = O.rk4_adjoint_step(w, lam, P)
    assert rel_l2(host(lo2), ref2) < 1e-12


def test_tangent_step_matches_oracle():
    api = _api()
    w = state((33, 6, 4), 14)
    P = params_for(w, mu=0.02, dt=2e-3)
    wd = synth.random_field(w.shape, 15)
    sd = synth.random_field(w.shape, 16)
    S = make_solver(api, w, P)
    out = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.tangent_step(dev(w), dev(wd), out, None, dev(sd))
    ref = O.rk4_tangent_step(w, wd, P, None, sd)
    assert rel_l2(host(out), ref) < 1e-12


@pytest.mark.parametrize("shape", [(40, 12, 1), (37, 9, 5), (8, 4, 2)])
def test_objective_value_and_gradient(shape):
    api = _api()
    w = state(shape, 17, 0.08)
    P = params_for(w)
    S = make_solver(api, w, P)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    S.objective(dev(w), J, 0.5, lam)
    assert abs(J.item() - 0.5 * O.objective(w, P)) <= 1e-13 * abs(O.objective(w, P)) + 1e-16
    ref = 0.5 * O.objective_grad(w, P)
    assert rel_l2(host(lam), ref) < 1e-12
    assert S.last_error() == 0


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_sigma1_field(shape, prec):
    api = _api()
    w = state(shape, 19, 0.1)
    P = params_for(w)
    S = make_solver(api, w, P, prec)
    sig = torch.empty(w.shape[1:], dtype=torch.float32, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    S.growth_sigma1(dev(w), sig, stats)
    ref = O.sigma1_field(w, P)
    tol = 1e-6 if prec == 0 else 2e-4
    np.testing.assert_allclose(host(sig), ref, rtol=tol, atol=tol * ref.max())
    st = host(stats)
    assert abs(st[0] - host(sig).max()) == 0.0
    assert abs(st[1] - host(sig).astype(np.float64).mean()) < 1e-12 * st[1]


def test_nu_rule_and_viscosity_operator():
    api = _api()
    shape = (37, 9, 5)
    w = state(shape, 21)
    P = params_for(w, dt=1e-3)
    S = make_solver(api, w, P)
    s1 = np.abs(synth.random_field(w.shape[1:], 22)).astype(np.float32)
    nu = torch.empty(w.shape[1:], dtype=torch.float32, device="cuda")
    S.add_adjoint_viscosity(dev(s1), 1e-4, nu, tau=0.5)
    ref = np.where(s1 > 0.5, np.float32(1e-4) * s1, 0).astype(np.float32)
    np.testing.assert_array_equal(host(nu), ref)
    assert S.last_error() == 0
    a = synth.random_field(w.shape, 23)
    out = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    S.apply_adjoint_viscosity(nu, dev(a), out)
    assert rel_l2(host(out), O.viscosity_apply(a, host(nu).astype(np.float64), P)) < 1e-12
    # an excessive coefficient is flagged, not silently used
    S.add_adjoint_viscosity(dev(s1), 1e3, nu)
    assert S.last_error() == api.NS_ERR_UNSTABLE


@pytest.mark.parametrize("prec", [0, 1])
def test_viscosity_cap_holds_nu_at_the_stability_limit(prec):
    """With ns_set_viscosity_cap the rule's coefficient is min(lambda sigma_1, limit),
    limit = 2.78 / (dt * 4 sum_d 1/dx_d^2) for RK4, with no error flag; without the cap
    the same coefficient is left as it is and flagged.  Both the float rule and the FP64
    rule, and the rule inside a sweep."""
    api = _api()
    shape = (37, 9, 5)
    w = state(shape, 21)
    P = params_for(w, dt=1e-3)
    S = make_solver(api, w, P, prec)
    limit = 2.78 / (P.dt * 4.0 * sum(1.0 / d ** 2 for d in P.dx))
    s1 = np.abs(synth.random_field(w.shape[1:], 22))
    lam = 1.5 * limit / s1.max()            # the largest cells exceed the limit
    for dt_ in (np.float32, np.float64):
        sig = torch.from_numpy(s1.astype(dt_)).cuda()
        nu = torch.empty_like(sig)
        S.add_adjoint_viscosity(sig, lam, nu)
        raw = (dt_(lam) * s1.astype(dt_)).astype(dt_)
        np.testing.assert_array_equal(host(nu), raw)
        assert S.last_error() == api.NS_ERR_UNSTABLE
        S.set_viscosity_cap(True)
        S.add_adjoint_viscosity(sig, lam, nu)
        assert S.last_error() == 0
        np.testing.assert_array_equal(host(nu), np.minimum(raw, dt_(limit)))
        assert (host(nu) == dt_(limit)).any() and (host(nu) < dt_(limit)).any()
        S.set_viscosity_cap(False)
    # a sweep whose rule exceeds the limit: flagged without the cap, clean with it
    opts = S.run_opts(6, api.NS_CKPT_ALL, 0, 40.0 * P.dx[0] ** 2)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.adjoint_run(dev(w), opts, arena, J, lam0)
    assert S.last_error() == api.NS_ERR_UNSTABLE
    S.set_viscosity_cap(True)
    S.adjoint_run(dev(w), opts, arena, J, lam0)
    assert S.last_error() == 0 and torch.isfinite(lam0).all()


def test_adjoint_energy_and_nonfinite_flag():
    api = _api()
    shape = (37, 9, 5)
    w = state(shape, 24, 0.1)
    P = params_for(w)
    lam = synth.random_field(w.shape, 25)
    S = make_solver(api, w, P)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    S.adjoint_energy(dev(w), dev(lam), E)
    ref = O.adjoint_energy(w, lam, P)
    assert abs(E.item() - ref) < 1e-12 * ref
    bad = lam.copy()
    bad[2, 1, 1, 1] = np.nan
    S.adjoint_energy(dev(w), dev(bad), E)
    assert S.last_error() == api.NS_ERR_NONFINITE
    assert S.last_error() == 0


def test_dot_combine_and_wave_speed():
    api = _api()
    shape = (37, 9, 5)
    w = state(shape, 26)
    P = params_for(w)
    S = make_solver(api, w, P)
    n = w[1].size
    phi = synth.random_field((7, n), 27)
    a = synth.random_field(n, 28)
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    S.dot(dev(a), dev(phi), out)
    np.testing.assert_allclose(host(out), phi @ a, rtol=1e-12)
    th = synth.random_field(7, 29)
    s = torch.empty(n, dtype=torch.float64, device="cuda")
    S.combine(dev(th), dev(phi), s)
    np.testing.assert_allclose(host(s), th @ phi, rtol=1e-12, atol=1e-12)
    m = torch.empty(1, dtype=torch.float64, device="cuda")
    S.max_wave_speed(dev(w), m)
    assert abs(m.item() - O.max_wave_speed(w, P)) < 1e-14


def test_gpu_dot_product_test_whole_trajectory():
    """<lam^0, dw0> + <sbar, ds> from the GPU adjoint sweep equals the GPU tangent dJbar
    (both FP64, both on the device): the discrete adjoint is exact on the GPU too."""
    api = _api()
    shape = (33, 10, 3)
    w0 = synth.isentropic_vortex(*shape, noise=1e-3, seed=3)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    steps = 6
    S = make_solver(api, w0, P)
    ws = [dev(w0)]
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(steps):
        nxt = torch.empty_like(ws[-1])
        S.primal_step(ws[-1], nxt)
        ws.append(nxt)
    dw = dev(synth.random_field(w0.shape, 30, 1e-2))
    ds = dev(synth.random_field(w0.shape, 31, 1e-2))
    # tangent: dJbar = sum_n <dJ/dw(w^n), wd^n> / N
    wd = dw.clone()
    Jd = 0.0
    for n in range(steps):
        nw = torch.empty_like(wd)
        S.tangent_step(ws[n], wd, nw, None, ds)
        wd = nw
        g = torch.zeros_like(wd)
        J.zero_()
        S.objective(ws[n + 1], J, 1.0 / steps, g)
        Jd += torch.sum(g * wd).item()
    lam = torch.zeros_like(dw)
    sbar = torch.zeros_like(dw)
    for n in range(steps, 0, -1):
        S.objective(ws[n], J, 1.0 / steps, lam)
        nl = torch.empty_like(lam)
        S.adjoint_step(ws[n - 1], lam, nl, sbar=sbar)
        lam = nl
    lhs = torch.sum(lam * dw).item() + torch.sum(sbar * ds).item()
    assert abs(lhs - Jd) < 1e-11 * abs(Jd)


def test_full_trajectory_matches_oracle_fp64():
    """Vortex box 64 x 64, 40 steps, store-all: Jbar and dJbar/dw^0 against the oracle."""
    api = _api()
    w0 = synth.isentropic_vortex(64, 64, 1, noise=1e-3, seed=1)
    P = params_for(w0, mu=0.5 / 1000)
    P.dt = 0.5 * P.dx[0] / O.max_wave_speed(w0, P)
    steps = 40
    ws_ref, Jref = O.primal_run(w0, P, steps)
    lam_ref, _ = O.adjoint_run(ws_ref, P)
    S = make_solver(api, w0, P)
    ws = [dev(w0)]
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(steps):
        nxt = torch.empty_like(ws[-1])
        S.primal_step(ws[-1], nxt)
        S.objective(nxt, J, 1.0 / steps)
        ws.append(nxt)
    lam = torch.zeros_like(ws[0])
    for n in range(steps, 0, -1):
        S.objective(ws[n], torch.zeros(1, dtype=torch.float64, device="cuda"), 1.0 / steps, lam)
        nl = torch.empty_like(lam)
        S.adjoint_step(ws[n - 1], lam, nl)
        lam = nl
    assert abs(J.item() - Jref) < 1e-12 * abs(Jref)
    assert rel_l2(host(ws[-1]), ws_ref[-1]) < 1e-12
    assert rel_l2(host(lam), lam_ref) < 1e-10


def test_mixed_precision_short_horizon():
    """Mixed mode (FP32 fluxes and transposes, FP64 state and accumulation) against the
    FP64 oracle over 20 steps of the 64 x 64 vortex: relative L2 below 1e-4 for the final
    state and for dJbar/dw^0."""
    api = _api()
    w0 = synth.isentropic_vortex(64, 64, 1, noise=1e-3, seed=1)
    P = params_for(w0, mu=0.5 / 1000)
    P.dt = 0.5 * P.dx[0] / O.max_wave_speed(w0, P)
    steps = 20
    ws_ref, Jref = O.primal_run(w0, P, steps)
    lam_ref, _ = O.adjoint_run(ws_ref, P)
    S = make_solver(api, w0, P, precision=1)
    ws = [dev(w0)]
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(steps):
        nxt = torch.empty_like(ws[-1])
        S.primal_step(ws[-1], nxt)
        S.objective(nxt, J, 1.0 / steps)
        ws.append(nxt)
    lam = torch.zeros_like(ws[0])
    for n in range(steps, 0, -1):
        S.objective(ws[n], torch.zeros(1, dtype=torch.float64, device="cuda"), 1.0 / steps, lam)
        nl = torch.empty_like(lam)
        S.adjoint_step(ws[n - 1], lam, nl)
        lam = nl
    assert rel_l2(host(ws[-1]), ws_ref[-1]) < 1e-4
    assert abs(J.item() - Jref) < 1e-4 * abs(Jref)
    assert rel_l2(host(lam), lam_ref) < 1e-4


def test_float_mirror_conversion_matches_cuda_rounding():
    """The integer-ALU double -> float conversion of the mixed path equals CUDA's own
    round-to-nearest-even conversion bit for bit over the normal float range (random
    values, exact ties, both signs, extreme exponents) and flushes values below the
    smallest normal float to signed zero."""
    api = _api()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200001) * np.exp(rng.uniform(-80, 80, 200001))
    f = rng.standard_normal(50000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + nxt.astype(np.float64)) / 2.0
    big = np.array([3.4028234e38, -3.4028234e38, 1.1754944e-38, -1.1754944e-38, 1.0, -0.0, 0.0])
    vals = np.concatenate([x, ties, big])
    vals = vals[(np.abs(vals) >= np.finfo(np.float32).tiny) | (vals == 0)]
    vals = vals[np.abs(vals) <= np.finfo(np.float32).max]
    S = api.Solver(4, 4, 1, 0.1)
    out = torch.empty(vals.size, dtype=torch.float32, device="cuda")
    S.to_float(dev(vals), out)
    ref = dev(vals).float()
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    tiny = np.array([1e-39, -1e-40, 1e-300, -1e-320, 0.0])
    out2 = torch.empty(tiny.size, dtype=torch.float32, device="cuda")
    S.to_float(dev(tiny), out2)
    o2 = host(out2)
    assert np.all(o2 == 0.0) and np.array_equal(np.signbit(o2), np.signbit(tiny))
    sp = np.array([np.inf, -np.inf, np.nan, 1e39, -1e300])
    out3 = torch.empty(sp.size, dtype=torch.float32, device="cuda")
    S.to_float(dev(sp), out3)
    o3 = host(out3)
    assert o3[0] == np.inf and o3[1] == -np.inf and np.isnan(o3[2]) and o3[3] == np.inf and o3[4] == -np.inf


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1), (7, 5, 3)])
def test_mixed_single_operators(shape):
    """Mixed mode per operator: residual, transposed residual, one RK4 step and one
    adjoint step (with viscosity and source seeds) within FP32 rounding of the oracle."""
    api = _api()
    w = state(shape, 41)
    P = params_for(w, mu=0.02, dt=2e-3)
    S = make_solver(api, w, P, 1)
    R = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs(dev(w), R)
    assert rel_l2(host(R), O.residual(w, P)) < 2e-5
    a = synth.random_field(w.shape, 42)
    S.rhs_transpose(dev(w), dev(a), R)
    assert rel_l2(host(R), O.residual_transpose(w, a, P)) < 2e-5
    w1 = torch.empty_like(R)
    S.primal_step(dev(w), w1)
    ref, _ = O.rk4_step(w, P)
    assert rel_l2(host(w1) - w, ref - w) < 2e-5
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 43))).astype(np.float32)
    lo = torch.empty_like(R)
    sb = torch.zeros_like(R)
    S.adjoint_step(dev(w), dev(a), lo, nu=dev(nu), sbar=sb)
    lref, sref = O.rk4_adjoint_step(w, a, P, None, nu.astype(np.float64))
    assert rel_l2(host(lo) - a, lref - a) < 2e-5
    assert rel_l2(host(sb), sref) < 2e-5


@pytest.mark.parametrize("shape", [(40, 12, 1), (37, 9, 5), (64, 48, 48)])
def test_objective_mixed_precision(shape):
    """The objective of a mixed-precision context is FP64 too (two launches)."""
    api = _api()
    w = state(shape, 18, 0.08)
    P = params_for(w)
    S = make_solver(api, w, P, 1)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    for _ in range(2):
        S.objective(dev(w), J, 0.5, lam)
    Jref = O.objective(w, P)
    assert abs(J.item() - Jref) <= 1e-12 * abs(Jref)
    assert rel_l2(host(lam), O.objective_grad(w, P)) < 1e-12
    assert S.last_error() == 0
