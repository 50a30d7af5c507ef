"""GPU parity of the per-variable added adjoint viscosity (ns_set_viscosity_split: the
separate viscosities for rho, rho u and rho E that the paper's conclusion names as a
next step) against the oracle with Params.nu_split: the operator alone, one adjoint
step in both precisions and for both integrators, the stabilised sweep, the stability
check with the largest factor, and argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, make_solver, rel_l2, state
from tests.test_gpu_sweep import _run
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

SPLIT = (0.5, 2.0, 3.0)


def test_operator_matches_oracle():
    api = _api()
    w = state((37, 9, 5), 91)
    P = params_for(w, mu=0.02, dt=2e-3)
    P.nu_split = SPLIT
    a = synth.random_field(w.shape, 92)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 93))).astype(np.float32)
    S = make_solver(api, w, P)
    S.set_viscosity_split(*SPLIT)
    out = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    S.apply_adjoint_viscosity(dev(nu), dev(a), out)
    assert rel_l2(host(out), O.viscosity_apply(a, nu.astype(np.float64), P)) < 1e-13


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scheme", ["rk4", "ssprk3"])
def test_adjoint_step_matches_oracle(prec, scheme):
    api = _api()
    w = state((37, 9, 5), 94)
    P = params_for(w, mu=0.02, dt=2e-3)
    P.nu_split, P.scheme = SPLIT, scheme
    lam = synth.random_field(w.shape, 95)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 96))).astype(np.float32)
    nz, ny, nx = w.shape[1:]
    S = api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec,
                   plane_i=P.plane_i, pt_in=P.pt_in,
                   scheme=api.NS_SSPRK3 if scheme == "ssprk3" else api.NS_RK4)
    S.set_viscosity_split(*SPLIT)
    lo = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    sb = torch.zeros_like(lo)
    S.adjoint_step(dev(w), dev(lam), lo, nu=dev(nu), sbar=sb)
    ref, sref = O.adjoint_step(w, lam, P, None, nu.astype(np.float64))
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(lo), ref) < tol
    assert rel_l2(host(sb), sref) < tol
    # the split matters: the single-coefficient adjoint differs
    P1 = params_for(w, mu=0.02, dt=2e-3)
    P1.scheme = scheme
    ref1, _ = O.adjoint_step(w, lam, P1, None, nu.astype(np.float64))
    assert rel_l2(ref1, ref) > 100 * tol


def test_stabilised_sweep_matches_oracle():
    api = _api()
    w0 = synth.isentropic_vortex(40, 12, 1, noise=1e-3, seed=6)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    P.nu_split = SPLIT
    N = 9
    lam_coef = 0.3 * P.dx[0] ** 2
    S = make_solver(api, w0, P)
    S.set_viscosity_split(*SPLIT)
    J, lam, sb, E, st = _run(api, S, w0, N, 1, 3, lam_coef=lam_coef)
    assert S.last_error() == 0
    ws, _ = O.primal_run(w0, P, N)
    lam_ref, _ = O.adjoint_run(ws, P, None, lambda w: lam_coef * O.sigma1_field(w, P))
    assert rel_l2(host(lam), lam_ref) < 1e-6


def test_stability_check_uses_the_largest_factor():
    """dt nu sum_d 4/dx_d^2 = 2.0 is stable for RK4 with factors 1 and unstable once the
    largest factor is 2 (4.0 > 2.78)."""
    api = _api()
    w = state((16, 8, 1), 97)
    P = params_for(w, mu=0.0, dt=1e-3)
    k = 4.0 * (1.0 / P.dx[0] ** 2 + 1.0 / P.dx[1] ** 2)
    nu_val = 2.0 / (P.dt * k)
    sig = torch.ones(w[0].size, dtype=torch.float32, device="cuda")
    nu = torch.empty_like(sig)
    S = make_solver(api, w, P)
    S.add_adjoint_viscosity(sig, nu_val, nu)
    assert S.last_error() == 0
    S.set_viscosity_split(1.0, 2.0, 1.0)
    S.add_adjoint_viscosity(sig, nu_val, nu)
    assert S.last_error() == api.NS_ERR_UNSTABLE


def test_bad_factors_are_rejected():
    api = _api()
    w = state((8, 4, 1), 98)
    S = make_solver(api, w, params_for(w))
    for bad in [(-1.0, 1.0, 1.0), (1.0, float("nan"), 1.0), (1.0, 1.0, float("inf"))]:
        with pytest.raises(api.NsError) as e:
            S.set_viscosity_split(*bad)
        assert e.value.code == api.NS_ERR_ARG
