"""GPU parity of the SSP-RK3 path (ns_params.scheme = NS_SSPRK3, section "Numerical
methods") against the oracle's Shu-Osher stages and their hand-reversed adjoint:
one step, its tangent and its adjoint (with and without added viscosity and source
seeds) in both precision modes, the checkpointed sweep across schedules, and the
scheme's own stability limit for the added viscosity.

Tolerances as for RK4: FP64 single operators 1e-12 and sweeps 1e-10 relative L2; mixed
mode 1e-4 over the short horizons used here."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, rel_l2, state
from tests.test_gpu_sweep import _run
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu


def _p3(w, **kw):
    P = params_for(w, **kw)
    P.scheme = "ssprk3"
    return P


def _solver(api, w, P, precision=0, batch=1):
    nz, ny, nx = w.shape[-3:]
    return api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt,
                      precision=precision, plane_i=P.plane_i, pt_in=P.pt_in, batch=batch,
                      scheme=api.NS_SSPRK3)


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1), (7, 5, 3), (3, 2, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_primal_steps_match_oracle(shape, prec):
    api = _api()
    w0 = state(shape, 71)
    P = _p3(w0, mu=0.02, dt=2e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.random_field(w0.shape[1:], 72)
    S = _solver(api, w0, P, prec)
    a, b = dev(w0), torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    w = w0
    for _ in range(6):
        S.primal_step(a, b, dev(s))
        a, b = b, a
        w, _ = O.ssprk3_step(w, P, s)
    tol = 1e-12 if prec == 0 else 1e-6
    assert rel_l2(host(a), w) < tol


def test_tangent_step_matches_oracle():
    api = _api()
    w = state((33, 6, 4), 73)
    P = _p3(w, mu=0.02, dt=2e-3)
    wd = synth.random_field(w.shape, 74)
    sd = synth.random_field(w.shape, 75)
    S = _solver(api, w, P)
    out = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.tangent_step(dev(w), dev(wd), out, None, dev(sd))
    assert rel_l2(host(out), O.ssprk3_tangent_step(w, wd, P, None, sd)) < 1e-12


@pytest.mark.parametrize("shape", [(37, 9, 5), (40, 12, 1), (7, 5, 3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_step_with_viscosity_and_source_seed(shape, prec):
    api = _api()
    w = state(shape, 76)
    P = _p3(w, mu=0.02, dt=2e-3)
    lam = synth.random_field(w.shape, 77)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 78))).astype(np.float32)
    S = _solver(api, w, P, prec)
    lo = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    sb = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    S.adjoint_step(dev(w), dev(lam), lo, nu=dev(nu), sbar=sb)
    ref, sref = O.ssprk3_adjoint_step(w, lam, P, None, nu.astype(np.float64))
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(lo), ref) < tol
    assert rel_l2(host(sb), sref) < tol
    lo2 = torch.empty_like(lo)
    S.adjoint_step(dev(w), dev(lam), lo2)
    ref2, _ = O.ssprk3_adjoint_step(w, lam, P)
    assert rel_l2(host(lo2), ref2) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_schedules_agree_bitwise_and_match_oracle(prec):
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = _p3(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N = 13
    S = _solver(api, w0, P, prec)
    res = [_run(api, S, w0, N, sch, prm, s) for sch, prm in [(0, 0), (1, 4), (2, 3), (2, 1)]]
    for J, lam, sb, _, _ in res[1:]:
        assert torch.equal(J, res[0][0])
        assert torch.equal(lam, res[0][1])
        assert torch.equal(sb, res[0][2])
    ws, Jref = O.primal_run(w0, P, N, s)
    lam_ref, sbar_ref = O.adjoint_run(ws, P, s)
    tol = 1e-10 if prec == 0 else 1e-4
    J, lam, sb, _, _ = res[0]
    assert abs(J.item() - Jref) <= tol * abs(Jref)
    assert rel_l2(host(lam), lam_ref) < tol
    assert rel_l2(host(sb), sbar_ref) < tol


def test_stabilised_sweep_matches_oracle():
    api = _api()
    w0 = synth.isentropic_vortex(40, 12, 1, noise=1e-3, seed=6)
    P = _p3(w0, mu=1e-3, dt=4e-3)
    N = 9
    lam_coef = 0.5 * P.dx[0] ** 2
    S = _solver(api, w0, P)
    J, lam, sb, E, st = _run(api, S, w0, N, 1, 3, lam_coef=lam_coef, energy=True, sigma=True)
    assert S.last_error() == 0
    ws, _ = O.primal_run(w0, P, N)
    lam_ref, _ = O.adjoint_run(ws, P, None, lambda w: lam_coef * O.sigma1_field(w, P))
    assert rel_l2(host(lam), lam_ref) < 1e-6


def test_viscosity_limit_is_the_schemes():
    """dt nu sum_d 4/dx_d^2 = 2.6 lies inside RK4's real-axis interval (2.78) and outside
    SSP-RK3's (2.51): only the SSP-RK3 context flags it."""
    api = _api()
    w = state((16, 8, 1), 79)
    P = params_for(w, mu=0.0, dt=1e-3)
    k = 4.0 * (1.0 / P.dx[0] ** 2 + 1.0 / P.dx[1] ** 2)
    nu_val = 2.6 / (P.dt * k)
    sig = torch.ones(w[0].size, dtype=torch.float32, device="cuda")
    nu = torch.empty_like(sig)
    for scheme, flagged in [(api.NS_RK4, False), (api.NS_SSPRK3, True)]:
        nz, ny, nx = w.shape[1:]
        S = api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, dt=P.dt, plane_i=P.plane_i,
                       pt_in=P.pt_in, scheme=scheme)
        S.add_adjoint_viscosity(sig, nu_val, nu)
        torch.cuda.synchronize()
        assert (S.last_error() == api.NS_ERR_UNSTABLE) == flagged
