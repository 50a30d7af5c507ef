"""Bounded boxes on the GPU against the oracle: characteristic inflow and outflow in x,
isothermal no-slip walls in y, and both (section "Numerical methods": non-reflecting
inlet and outlet; section "Problem setup": the isothermal vane surface).  The residual,
the transposed residual with the added viscosity (closed boundary faces), sigma_1 with
the ghosts, and a bounded, sourced trajectory (steps, the time-averaged objective, the
adjoint with the objective source and the source sensitivity) are compared element by
element with the oracle's padded-box forms, in both precisions, on ragged sizes."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, rel_l2
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

BCS = {"inout": 1, "walls": 2, "inout_walls": 3}
FAR = (1.02, 0.48, 0.03, -0.02, 0.98 / 1.4)
WALL_E = (1.70, 1.90)


def _case(shape, seed, bc, mu=0.01, dt=2e-3):
    nx, ny, nz = shape
    w = synth.perturbed_uniform(nx, ny, nz, seed=seed, amp=0.06)
    P = dataclasses.replace(params_for(w, mu=mu, dt=dt), bc=bc, far=FAR, wall_e=WALL_E)
    return w, P


def _solver(api, w, P, prec):
    nz, ny, nx = w.shape[1:]
    S = api.Solver(nx, ny, nz, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec,
                   plane_i=P.plane_i, pt_in=P.pt_in)
    S.set_boundaries(BCS[P.bc], far=FAR, wall_e=WALL_E)
    return S


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(37, 9, 5), (33, 10, 1)])
def test_bounded_residual_and_transpose(bc, prec, shape):
    api = _api()
    w, P = _case(shape, 41, bc)
    s = 0.05 * synth.random_field(w.shape, 42)
    a = synth.random_field(w.shape, 43)
    nu = (0.01 * np.abs(synth.random_field(w.shape[1:], 44))).astype(np.float32)
    S = _solver(api, w, P, prec)
    R = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    S.rhs(dev(w), R, dev(s))
    tol = 1e-12 if prec == 0 else 2e-5
    assert rel_l2(host(R), O.residual(w, P, s)) < tol
    T = torch.empty_like(R)
    S.rhs_transpose(dev(w), dev(a), T, nu=dev(nu))
    ref = O.residual_transpose(w, a, P) + O.viscosity_apply(a, nu.astype(np.float64), P)
    assert rel_l2(host(T), ref) < tol
    S.rhs_transpose(dev(w), dev(a), T)
    assert rel_l2(host(T), O.residual_transpose(w, a, P)) < tol
    assert S.last_error() == 0


@pytest.mark.parametrize("bc", list(BCS))
def test_bounded_transpose_is_the_adjoint_of_the_residual_on_gpu(bc):
    """<a, J v> = <J^T a, v> with J v from central differences of the GPU's own bounded
    residual (FP64): the transpose kernels and the ghost pull-back fit the residual kernels."""
    api = _api()
    w, P = _case((21, 7, 3), 45, bc, mu=0.02)
    a = synth.random_field(w.shape, 46)
    v = synth.random_field(w.shape, 47)
    S = _solver(api, w, P, 0)
    Rp = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    Rm = torch.empty_like(Rp)
    h = 1e-6
    S.rhs(dev(w + h * v), Rp)
    S.rhs(dev(w - h * v), Rm)
    Jv = (host(Rp) - host(Rm)) / (2 * h)
    T = torch.empty_like(Rp)
    S.rhs_transpose(dev(w), dev(a), T)
    lhs, rhs = float(np.sum(a * Jv)), float(np.sum(host(T) * v))
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs)


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("prec", [0, 1])
def test_bounded_sigma1(bc, prec):
    api = _api()
    w, P = _case((37, 9, 5), 48, bc)
    S = _solver(api, w, P, prec)
    sig = torch.empty(w.shape[1:], dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    S.growth_sigma1(dev(w), sig)
    ref = O.sigma1_field(w, P)
    if prec == 0:
        np.testing.assert_allclose(host(sig), ref, rtol=1e-12, atol=1e-12 * ref.max())
    else:
        assert rel_l2(host(sig).astype(np.float64), ref) < 2e-4


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("prec", [0, 1])
def test_bounded_sourced_trajectory(bc, prec):
    """N steps with a source, Jbar, the adjoint with the objective source, dJbar/dw0 and
    the source sensitivity, against the oracle's store-all adjoint of the bounded box;
    the stabilised variant with the sigma_1 rule's viscosity in FP64 contexts."""
    api = _api()
    w0, P = _case((33, 10, 4), 49, bc, mu=0.01, dt=3e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 4, n=4)[0]
    N = 6
    S = _solver(api, w0, P, prec)
    sd = dev(s)
    ws = [dev(w0)]
    for n in range(N):
        w1 = torch.empty_like(ws[0])
        S.primal_step(ws[-1], w1, s=sd)
        ws.append(w1)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(1, N + 1):
        S.objective(ws[n], J, 1.0 / N)
    lam = torch.zeros_like(ws[0])
    S.objective(ws[N], torch.zeros_like(J), 1.0 / N, lam)
    sbar = torch.zeros_like(lam)
    for n in range(N - 1, -1, -1):
        lo = torch.empty_like(lam)
        S.adjoint_step(ws[n], lam, lo, s=sd, sbar=sbar)
        lam = lo
        if n >= 1:
            S.objective(ws[n], torch.zeros_like(J), 1.0 / N, lam)
    torch.cuda.synchronize()
    assert S.last_error() == 0
    traj, Jref = O.primal_run(w0, P, N, s)
    lam_ref, sbar_ref = O.adjoint_run(traj, P, s)
    tol = 1e-10 if prec == 0 else 1e-4
    for n in (1, N):
        assert rel_l2(host(ws[n]) - w0, traj[n] - w0) < (1e-12 if prec == 0 else 2e-5)
    assert abs(J.item() - Jref) <= tol * abs(Jref)
    assert rel_l2(host(lam), lam_ref) < tol
    assert rel_l2(host(sbar), sbar_ref) < tol


@pytest.mark.parametrize("bc", list(BCS))
def test_bounded_stabilised_adjoint_step_fp64(bc):
    """One adjoint step with nu = lambda sigma_1 computed on the bounded box in FP64 (the
    _f64 entry points) against the oracle's step with its own sigma_1."""
    api = _api()
    w, P = _case((37, 9, 5), 50, bc)
    lam = synth.random_field(w.shape, 51)
    lam_coef = 0.5 * P.dx[0] ** 2
    S = _solver(api, w, P, 0)
    sig = torch.empty(w.shape[1:], dtype=torch.float64, device="cuda")
    S.growth_sigma1(dev(w), sig)
    nu = torch.empty_like(sig)
    S.add_adjoint_viscosity(sig, lam_coef, nu)
    lo = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    sb = torch.zeros_like(lo)
    S.adjoint_step(dev(w), dev(lam), lo, nu=nu, sbar=sb)
    ref, sref = O.rk4_adjoint_step(w, lam, P, None, lam_coef * O.sigma1_field(w, P))
    assert S.last_error() == 0
    assert rel_l2(host(lo), ref) < 1e-10
    assert rel_l2(host(sb), sref) < 1e-12


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("sched", [(1, 3), (2, 3), (4, 3)])
def test_bounded_checkpointed_sweep(bc, prec, sched, tmp_path):
    """ns_adjoint_run on a bounded box (stride, revolve and disk-tier schedules, the sigma_1
    rule's viscosity, a source, the energy series) gives the bits of the same calls made
    step by step with every state kept, and matches the oracle's stabilised adjoint."""
    api = _api()
    w0, P = _case((33, 10, 4), 53, bc, mu=0.01, dt=3e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 4, n=4)[0]
    N = 8
    lam_coef = 0.4 * P.dx[0] ** 2
    S = _solver(api, w0, P, prec)
    sd = dev(s)
    # step by step: the forward states, then the reverse with sigma_1, nu and the source
    ws = [dev(w0)]
    for n in range(N):
        w1 = torch.empty_like(ws[0])
        S.primal_step(ws[-1], w1, s=sd)
        ws.append(w1)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(ws[0])
    sbar = torch.zeros_like(lam)
    E = torch.zeros((N + 1, 1), dtype=torch.float64, device="cuda")
    S.objective(ws[N], J, 1.0 / N, lam)
    S.adjoint_energy(ws[N], lam, E[N])
    sdt = torch.float64 if prec == 0 else torch.float32
    sig = torch.empty(w0.shape[1:], dtype=sdt, device="cuda")
    nu = torch.empty_like(sig)
    for n in range(N - 1, -1, -1):
        S.growth_sigma1(ws[n], sig)
        S.add_adjoint_viscosity(sig, lam_coef, nu)
        lo = torch.empty_like(lam)
        S.adjoint_step(ws[n], lam, lo, s=sd, nu=nu, sbar=sbar)
        lam = lo
        if n >= 1:
            S.objective(ws[n], J, 1.0 / N, lam)
        S.adjoint_energy(ws[n], lam, E[n])
    schedule, param = sched
    path = str(tmp_path / "snap.bin") if schedule == 4 else None
    opts = S.run_opts(N, schedule, param, lam_coef, 0.0, True, disk_path=path)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    Js = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(lam)
    sb0 = torch.empty_like(lam)
    Es = torch.zeros_like(E)
    S.adjoint_run(dev(w0), opts, arena, Js, lam0, s=sd, sbar=sb0, energy=Es)
    torch.cuda.synchronize()
    assert S.last_error() == 0
    assert torch.equal(Js, J) and torch.equal(lam0, lam) and torch.equal(sb0, sbar) and torch.equal(Es, E)
    traj, Jref = O.primal_run(w0, P, N, s)
    nu_of = lambda w: lam_coef * O.sigma1_field(w, P)
    lam_ref, sbar_ref = O.adjoint_run(traj, P, s, nu_of)
    tol = 1e-10 if prec == 0 else 1e-4
    assert abs(Js.item() - Jref) <= tol * abs(Jref)
    assert rel_l2(host(lam0), lam_ref) < tol
    assert rel_l2(host(sb0), sbar_ref) < tol


def test_bounded_context_refuses_the_periodic_only_calls():
    api = _api()
    w, P = _case((12, 6, 2), 52, "inout")
    S = _solver(api, w, P, 0)
    wd = dev(w)
    out = torch.empty_like(wd)
    with pytest.raises(api.NsError):
        S.rhs_tangent(wd, wd.clone(), out)
    # the sweep runs on a bounded box, but without sigma_1 statistics or the learned closure
    opts = S.run_opts(3, api.NS_CKPT_ALL, 0, record_sigma=True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    with pytest.raises(api.NsError):
        S.adjoint_run(wd, opts, arena, torch.empty(1, dtype=torch.float64, device="cuda"), out)
    with pytest.raises(api.NsError):
        S.set_boundaries(api.NS_BC_INOUT, far=None)
    with pytest.raises(api.NsError):
        S.set_boundaries(api.NS_BC_WALLS, wall_e=(1.0, -1.0))
    # back to periodic: the periodic residual again
    S.set_boundaries(api.NS_BC_PERIODIC)
    S.rhs(wd, out)
    assert rel_l2(host(out), O.residual(w, dataclasses.replace(P, bc="periodic"))) < 1e-12
