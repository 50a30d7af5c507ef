"""Parity at the workloads' own sizes and horizons.

- The 64x64 isentropic vortex (Mach 0.5, Re 1000, CFL 0.5), 200 RK4 steps with every
  state stored: the time-averaged pressure loss and its gradient with respect to the
  initial state against the oracle's store-all adjoint, to 1e-10 in FP64 and 1e-4 in
  mixed precision.  This is the full horizon of that workload (a non-chaotic one: the
  adjoint stays bounded), not a shortened one.
- One 96x48x48 vortex column with the 64-bump x-momentum forcing through the autograd
  wrapper (the batched workload's box size) over 20 steps: the gradients with respect to
  the initial state and to the 64 forcing parameters against the oracle's adjoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import config as C
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, make_solver, rel_l2

pytestmark = pytest.mark.gpu


def _params(wl, w):
    P = O.Params(gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dx=wl.dx, plane_i=wl.plane_i, pt_in=wl.pt_in)
    P.dt = C.cfl_dt(wl, O.max_wave_speed(w, P))
    return P


@pytest.fixture(scope="module")
def vortex64():
    wl = C.WORKLOADS["vortex64"]
    w0 = wl.initial_state()
    P = _params(wl, w0)
    traj, Jref = O.primal_run(w0, P, wl.nsteps)
    lam_ref, _ = O.adjoint_run(traj, P)
    return wl, w0, P, Jref, lam_ref


@pytest.mark.parametrize("prec", [0, 1])
def test_vortex64_full_horizon_store_all(vortex64, prec):
    wl, w0, P, Jref, lam_ref = vortex64
    assert wl.nsteps == 200 and wl.schedule == "all"
    api = _api()
    S = make_solver(api, w0, P, prec)
    opts = S.run_opts(wl.nsteps, api.NS_CKPT_ALL, 0)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    S.adjoint_run(dev(w0), opts, arena, J, lam0)
    torch.cuda.synchronize()
    assert S.last_error() == 0
    tol = 1e-10 if prec == 0 else 1e-4
    assert abs(J.item() - Jref) <= tol * abs(Jref)
    assert rel_l2(host(lam0), lam_ref) < tol


def test_column96_autograd_against_oracle():
    api = _api()
    from paper_1511_06959_gb300 import autograd
    wl = C.WORKLOADS["column96"]
    N = 20
    w0 = synth.isentropic_vortex(wl.nx, wl.ny, wl.nz, mach=wl.mach, noise=1e-3, seed=wl.seed)
    P = _params(wl, w0)
    phi = synth.forcing_bumps(wl.nx, wl.ny, wl.nz, n=64)
    theta = 0.02 * np.random.default_rng(7).standard_normal(64)
    S = make_solver(api, w0[None], P, 0, batch=1)
    prob = autograd.SourceProblem(S, dev(phi), N, api.NS_CKPT_REVOLVE, 4)
    wt = dev(w0[None]).requires_grad_(True)
    th = dev(theta).requires_grad_(True)
    J = prob(wt, th)
    J.sum().backward()
    s = np.zeros_like(w0)
    s[1] = np.tensordot(theta, phi, axes=1)
    traj, Jref = O.primal_run(w0, P, N, s)
    lam_ref, sbar_ref = O.adjoint_run(traj, P, s)
    assert abs(J.item() - Jref) <= 1e-10 * abs(Jref)
    assert rel_l2(host(wt.grad[0]), lam_ref) < 1e-10
    gth_ref = np.tensordot(phi, sbar_ref[1], axes=([1, 2, 3], [0, 1, 2]))
    assert rel_l2(host(th.grad), gth_ref) < 1e-10
