"""torch.autograd.Function over the GPU discrete adjoint: a batch of 3D boxes (vortex
columns with noise), the pressure loss with a 64-parameter x-momentum source, gradients
with respect to the initial states and to the source parameters, checked against the
oracle's store-all adjoint, against central finite differences (eps = 1e-6, FP64) of the
GPU primal, under the added adjoint viscosity, and in mixed precision."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, make_solver, rel_l2
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

NX, NY, NZ, B, N = 24, 12, 12, 2, 8


def _setup(precision=0, lam_tilde=0.0, schedule=0, param=0):
    api = _api()
    from paper_1511_06959_gb300 import autograd
    ws = np.stack([synth.isentropic_vortex(NX, NY, NZ, noise=1e-3, seed=3 + b) for b in range(B)])
    P = params_for(ws[0], mu=0.5 / 1000, mach=0.5)
    P.dt = 0.5 * P.dx[0] / max(O.max_wave_speed(w, P) for w in ws)
    phi = synth.forcing_bumps(NX, NY, NZ, n=64)
    S = make_solver(api, ws[0], P, precision, batch=B)
    prob = autograd.SourceProblem(S, dev(phi), N, schedule, param, lam_tilde * P.dx[0] ** 2)
    return api, prob, ws, P, phi


def _loss_and_grads(prob, ws, theta, c):
    w0 = dev(ws).requires_grad_(True)
    th = dev(theta).requires_grad_(True)
    J = prob(w0, th)
    L = torch.sum(J * dev(c))
    L.backward()
    return J.detach(), w0.grad.detach(), th.grad.detach()


def test_gradients_match_oracle_store_all_adjoint():
    api, prob, ws, P, phi = _setup()
    rng = np.random.default_rng(0)
    theta = 0.05 * rng.standard_normal(64)
    c = np.array([0.7, -1.3])
    J, gw, gth = _loss_and_grads(prob, ws, theta, c)
    gth_ref = np.zeros(64)
    for b in range(B):
        s = np.zeros_like(ws[b])
        s[1] = np.tensordot(theta, phi, axes=1)
        traj, Jref = O.primal_run(ws[b], P, N, s)
        lam, sbar = O.adjoint_run(traj, P, s)
        assert abs(J[b].item() - Jref) <= 1e-12 * abs(Jref)
        assert rel_l2(host(gw[b]), c[b] * lam) < 1e-10
        gth_ref += c[b] * np.tensordot(phi, sbar[1], axes=([1, 2, 3], [0, 1, 2]))
    assert rel_l2(host(gth), gth_ref) < 1e-10


def test_gradients_match_central_differences():
    api, prob, ws, P, phi = _setup(schedule=2, param=2)
    rng = np.random.default_rng(1)
    theta = 0.05 * rng.standard_normal(64)
    c = np.array([1.0, 0.5])
    _, gw, gth = _loss_and_grads(prob, ws, theta, c)
    eps = 1e-6

    def L(w, th):
        with torch.no_grad():
            return float(torch.sum(prob(dev(w), dev(th)) * dev(c)))

    for seed in (2, 3):
        dw = synth.random_field(ws.shape, seed)
        fd = (L(ws + eps * dw, theta) - L(ws - eps * dw, theta)) / (2 * eps)
        ad = float(torch.sum(gw * dev(dw)))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    for m in (0, 27, 63):
        e = np.zeros(64)
        e[m] = 1.0
        fd = (L(ws, theta + eps * e) - L(ws, theta - eps * e)) / (2 * eps)
        assert abs(fd - gth[m].item()) <= 1e-6 * max(abs(fd), 1e-12), (m, fd, gth[m].item())


@pytest.mark.parametrize("lam_tilde", [0.1, 0.5, 1.0])
def test_stabilised_gradients_match_oracle(lam_tilde):
    api, prob, ws, P, phi = _setup(lam_tilde=lam_tilde)
    theta = np.zeros(64)
    c = np.array([1.0, 1.0])
    _, gw, _ = _loss_and_grads(prob, ws, theta, c)
    coef = lam_tilde * P.dx[0] ** 2
    for b in range(B):
        traj, _ = O.primal_run(ws[b], P, N)
        lam, _ = O.adjoint_run(traj, P, None, lambda w: coef * O.sigma1_field(w, P))
        assert rel_l2(host(gw[b]), lam) < 1e-6


def test_mixed_precision_gradients_close_to_fp64():
    _, prob64, ws, P, phi = _setup(precision=0)
    _, prob32, _, _, _ = _setup(precision=1)
    theta = 0.05 * np.random.default_rng(4).standard_normal(64)
    c = np.array([1.0, -1.0])
    J64, gw64, gth64 = _loss_and_grads(prob64, ws, theta, c)
    J32, gw32, gth32 = _loss_and_grads(prob32, ws, theta, c)
    assert rel_l2(host(J32), host(J64)) < 1e-6
    assert rel_l2(host(gw32), host(gw64)) < 1e-4
    assert rel_l2(host(gth32), host(gth64)) < 1e-4


def test_backward_of_a_replaced_forward_raises():
    """Two losses on one solver: the second forward replaces the first's checkpoints, so
    the first loss's backward must raise instead of reversing the second trajectory; the
    second loss's backward still matches the oracle, and a second backward of it raises."""
    api, prob, ws, P, phi = _setup()
    theta_a = np.zeros(64)
    theta_b = 0.05 * np.random.default_rng(4).standard_normal(64)
    w_a = dev(ws).requires_grad_(True)
    w_b = dev(ws).requires_grad_(True)
    J_a = prob(w_a, dev(theta_a))
    J_b = prob(w_b, dev(theta_b).requires_grad_(True))
    with pytest.raises(RuntimeError, match="no longer hold"):
        torch.sum(J_a).backward()
    L_b = torch.sum(J_b)
    L_b.backward(retain_graph=True)
    s = np.zeros_like(ws[0])
    s[1] = np.tensordot(theta_b, phi, axes=1)
    traj, _ = O.primal_run(ws[0], P, N, s)
    lam, _ = O.adjoint_run(traj, P, s)
    assert rel_l2(host(w_b.grad[0]), lam) < 1e-10
    with pytest.raises(RuntimeError, match="no longer hold"):
        L_b.backward()
