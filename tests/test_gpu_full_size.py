"""Parity at the benchmark's own size and launch configuration: the 128x64x64 transonic
turbulent box of bench.py (its initial state, viscosity, time step and context), one
primal step, one stabilised adjoint step with the objective source and sigma_1, and the
objective, compared element by element with the oracle in both precision modes.  One
step of the oracle on this machine takes seconds, so the whole fields are compared, not
samples; the 1000-step sweep itself is covered by the mixed-versus-FP64 comparison that
bench.py reports."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import config as C
from tests.test_gpu_parity import _api, dev, host, rel_l2

pytestmark = pytest.mark.gpu

WL = C.WORKLOADS["box128"]


@pytest.fixture(scope="module")
def box():
    api = _api()
    w = WL.initial_state()
    P = O.Params(gamma=WL.gamma, mu=WL.mu, Pr=WL.Pr, dx=WL.dx, plane_i=WL.plane_i, pt_in=WL.pt_in)
    P.dt = C.cfl_dt(WL, O.max_wave_speed(w, P))
    w1, _ = O.rk4_step(w, P)
    lam = O.objective_grad(w1, P) / WL.nsteps
    nu = WL.lam_coef * O.sigma1_field(w, P)
    lam0, _ = O.rk4_adjoint_step(w, lam, P, None, nu)
    lam0 = lam0 + O.objective_grad(w, P) / WL.nsteps
    return api, w, P, w1, lam, lam0, O.objective(w1, P)


def _solver(api, P, prec):
    return api.Solver(WL.nx, WL.ny, WL.nz, WL.dx, gamma=WL.gamma, mu=WL.mu, Pr=WL.Pr, dt=P.dt,
                      precision=prec, plane_i=WL.plane_i, pt_in=WL.pt_in)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_objective_and_stabilised_adjoint_step(box, prec):
    api, w, P, w1_ref, lam, lam0_ref, J_ref = box
    S = _solver(api, P, prec)
    wd = dev(w)
    w1 = torch.empty_like(wd)
    S.primal_step(wd, w1)
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(w1) - w, w1_ref - w) < tol
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.objective(dev(w1_ref), J, 1.0)          # FP64 in both modes: the same input
    assert abs(J.item() - J_ref) <= 1e-12 * abs(J_ref)
    # sigma_1 and nu in FP64 in the FP64 context (the _f64 entry points), FP32 in mixed
    sig = torch.empty(w.shape[1:], dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    S.growth_sigma1(wd, sig)
    nu = torch.empty_like(sig)
    S.add_adjoint_viscosity(sig, WL.lam_coef, nu)
    lo = torch.empty_like(wd)
    S.adjoint_step(wd, dev(lam), lo, nu=nu)
    S.objective(wd, torch.zeros(1, dtype=torch.float64, device="cuda"), 1.0 / WL.nsteps, lo)
    assert S.last_error() == 0
    tol = 1e-10 if prec == 0 else 1e-4
    assert rel_l2(host(lo), lam0_ref) < tol
    if prec == 0:
        np.testing.assert_allclose(host(sig), O.sigma1_field(w, P), rtol=1e-12, atol=1e-12 * abs(host(sig)).max())


def test_f64_entry_points_refuse_a_mixed_context(box):
    api, w, P, *_ = box
    S = _solver(api, P, 1)
    wd = dev(w)
    sig = torch.empty(w.shape[1:], dtype=torch.float64, device="cuda")
    with pytest.raises(api.NsError):
        S.growth_sigma1(wd, sig)
    with pytest.raises(api.NsError):
        S.adjoint_step(wd, wd.clone(), torch.empty_like(wd), nu=sig)
