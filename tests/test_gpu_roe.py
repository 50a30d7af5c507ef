"""GPU parity of the Roe-dissipation flux (ns_params.flux = NS_FLUX_ROE, section
"Numerical methods") against the oracle, whose tangent and transpose of the dissipation
come from complex-step Jacobians (independent of the kernels' hand-reversed adjoint):
the residual, its tangent and transpose, the GPU dot-product identity, steps with both
integrators, the adjoint step with viscosity and source seeds, and the checkpointed
sweep across schedules, in both precisions where the mode exists.

Tolerances as for the central flux: FP64 operators 1e-12, FP64 sweeps 1e-10; mixed mode
2e-5 per operator and 1e-4 over a short horizon."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, rel_l2, state
from tests.test_gpu_sweep import _run
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

SHAPES = [(37, 9, 5), (40, 12, 1), (7, 5, 3), (3, 2, 1)]


def _pr(w, scheme="rk4", **kw):
    P = params_for(w, **kw)
    P.flux, P.scheme = "roe", scheme
    return P


def _solver(api, w, P, precision=0):
    nz, ny, nx = w.shape[-3:]
    return api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt,
                      precision=precision, plane_i=P.plane_i, pt_in=P.pt_in,
                      scheme=api.NS_SSPRK3 if P.scheme == "ssprk3" else api.NS_RK4,
                      flux=api.NS_FLUX_ROE, roe_delta=P.roe_delta)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_residual_and_transpose(shape, prec):
    api = _api()
    w = state(shape, 121, 0.1)
    P = _pr(w, mu=0.02)
    S = _solver(api, w, P, prec)
    R = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs(dev(w), R)
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(R), O.residual(w, P)) < tol
    a = synth.random_field(w.shape, 122)
    S.rhs_transpose(dev(w), dev(a), R)
    assert rel_l2(host(R), O.residual_transpose(w, a, P)) < tol


@pytest.mark.parametrize("shape", SHAPES)
def test_tangent_and_gpu_dot_product(shape):
    api = _api()
    w = state(shape, 123, 0.1)
    P = _pr(w, mu=0.02)
    S = _solver(api, w, P)
    v = synth.random_field(w.shape, 124)
    a = synth.random_field(w.shape, 125)
    Jv = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    JTa = torch.empty_like(Jv)
    S.rhs_tangent(dev(w), dev(v), Jv)
    S.rhs_transpose(dev(w), dev(a), JTa)
    assert rel_l2(host(Jv), O.residual_tangent(w, v, P)) < 1e-12
    lhs, rhs = float(np.sum(a * host(Jv))), float(np.sum(host(JTa) * v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("scheme", ["rk4", "ssprk3"])
@pytest.mark.parametrize("prec", [0, 1])
def test_steps_and_adjoint_step(scheme, prec):
    api = _api()
    w = state((37, 9, 5), 126, 0.08)
    P = _pr(w, scheme, mu=0.02, dt=2e-3)
    S = _solver(api, w, P, prec)
    w1 = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.primal_step(dev(w), w1)
    ref, _ = O.step(w, P)
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(w1) - w, ref - w) < tol
    lam = synth.random_field(w.shape, 127)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 128))).astype(np.float32)
    lo = torch.empty_like(w1)
    sb = torch.zeros_like(w1)
    S.adjoint_step(dev(w), dev(lam), lo, nu=dev(nu), sbar=sb)
    lref, sref = O.adjoint_step(w, lam, P, None, nu.astype(np.float64))
    assert rel_l2(host(lo) - lam, lref - lam) < tol
    assert rel_l2(host(sb), sref) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_schedules_agree_bitwise_and_match_oracle(prec):
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = _pr(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N = 9
    S = _solver(api, w0, P, prec)
    res = [_run(api, S, w0, N, sch, prm, s) for sch, prm in [(0, 0), (1, 4), (2, 3)]]
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


def test_bad_entropy_fix_is_rejected():
    api = _api()
    w = state((8, 4, 1), 129)
    P = params_for(w)
    with pytest.raises(api.NsError) as e:
        api.Solver(8, 4, 1, P.dx, flux=api.NS_FLUX_ROE, roe_delta=0.0)
    assert e.value.code == api.NS_ERR_ARG
