"""The autograd wrapper at the full size of its workload: a batch of 8 vortex columns of
96x48x48 cells (1.77 M cells), 100 steps, the pressure loss with a 64-parameter
x-momentum source.  Gradients with respect to the initial states and to the source
parameters are checked against central finite differences (eps = 1e-6, FP64) of the GPU
primal; the mixed-precision gradients against the FP64 ones for every lambda of the
sweep {0, 0.1, 0.5, 1}; and the per-cell sigma_1 field of the batch is produced and
consistent with its statistics.  (The oracle adjoint at this size would take tens of
minutes on the host; the small-box tests compare with it.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1511_06959_gb300 import synth
from paper_1511_06959_gb300 import config as C
from tests.test_gpu_parity import _api, dev, host, rel_l2

pytestmark = pytest.mark.gpu

WL = C.WORKLOADS["column96"]


def _problem(api, ws, dt, precision, lam_tilde):
    from paper_1511_06959_gb300 import autograd
    S = api.Solver(WL.nx, WL.ny, WL.nz, WL.dx, gamma=WL.gamma, mu=WL.mu, Pr=WL.Pr, dt=dt,
                   precision=precision, plane_i=WL.plane_i, pt_in=WL.pt_in, batch=WL.batch)
    phi = dev(synth.forcing_bumps(WL.nx, WL.ny, WL.nz, n=64))
    prob = autograd.SourceProblem(S, phi, WL.nsteps, api.NS_CKPT_REVOLVE, 8, lam_tilde * WL.dx[0] ** 2)
    return S, prob


@pytest.fixture(scope="module")
def batch():
    api = _api()
    ws = np.stack([synth.isentropic_vortex(WL.nx, WL.ny, WL.nz, mach=WL.mach, noise=1e-3, seed=WL.seed + b)
                   for b in range(WL.batch)])
    S = api.Solver(WL.nx, WL.ny, WL.nz, WL.dx, gamma=WL.gamma, mu=WL.mu, Pr=WL.Pr, batch=WL.batch)
    m = torch.empty(1, dtype=torch.float64, device="cuda")
    S.max_wave_speed(dev(ws), m)
    return api, ws, C.cfl_dt(WL, m.item())


def _grads(prob, ws, theta, c):
    w0 = dev(ws).requires_grad_(True)
    th = dev(theta).requires_grad_(True)
    J = prob(w0, th)
    torch.sum(J * dev(c)).backward()
    return J.detach(), w0.grad.detach(), th.grad.detach()


def test_fp64_gradients_match_central_differences(batch):
    api, ws, dt = batch
    _, prob = _problem(api, ws, dt, api.NS_FP64, 0.0)
    rng = np.random.default_rng(5)
    theta = 0.05 * rng.standard_normal(64)
    c = rng.uniform(0.5, 1.5, WL.batch)
    _, gw, gth = _grads(prob, ws, theta, c)
    eps = 1e-6

    def L(w, th):
        with torch.no_grad():
            return float(torch.sum(prob(dev(w), dev(th)) * dev(c)))

    dw = synth.random_field(ws.shape, 6)
    fd = (L(ws + eps * dw, theta) - L(ws - eps * dw, theta)) / (2 * eps)
    ad = float(torch.sum(gw * dev(dw)))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    # the two largest source sensitivities (at 100 steps most bumps barely reach the
    # plane, and FD rounding noise would swamp their tiny gradients)
    for m in np.argsort(-np.abs(host(gth)))[:2]:
        e = np.zeros(64)
        e[m] = 1.0
        fd = (L(ws, theta + eps * e) - L(ws, theta - eps * e)) / (2 * eps)
        assert abs(fd - gth[m].item()) <= 1e-6 * max(abs(fd), 1e-12), (m, fd, gth[m].item())


@pytest.mark.parametrize("lam_tilde", [0.0, 0.1, 0.5, 1.0])
def test_mixed_precision_gradients_close_to_fp64(batch, lam_tilde):
    api, ws, dt = batch
    theta = 0.05 * np.random.default_rng(7).standard_normal(64)
    c = np.ones(WL.batch)
    S64, p64 = _problem(api, ws, dt, api.NS_FP64, lam_tilde)
    J64, gw64, gth64 = _grads(p64, ws, theta, c)
    assert S64.last_error() == 0
    S32, p32 = _problem(api, ws, dt, api.NS_MIXED, lam_tilde)
    J32, gw32, gth32 = _grads(p32, ws, theta, c)
    assert S32.last_error() == 0
    assert rel_l2(host(J32), host(J64)) < 1e-6
    assert rel_l2(host(gw32), host(gw64)) < 1e-4
    assert rel_l2(host(gth32), host(gth64)) < 1e-4


def test_sigma1_field_of_the_batch(batch):
    api, ws, dt = batch
    S, _ = _problem(api, ws, dt, api.NS_MIXED, 0.0)
    sig = torch.empty((WL.batch, WL.nz, WL.ny, WL.nx), dtype=torch.float32, device="cuda")
    stats = torch.empty((WL.batch, 2), dtype=torch.float64, device="cuda")
    S.growth_sigma1(dev(ws), sig, stats)
    s = host(sig).astype(np.float64)
    st = host(stats)
    assert np.all(np.isfinite(s)) and np.all(s >= 0.0)
    for b in range(WL.batch):
        assert st[b, 0] == s[b].max()
        assert abs(st[b, 1] - s[b].mean()) <= 1e-12 * st[b, 1]
