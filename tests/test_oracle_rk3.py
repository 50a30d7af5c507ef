"""Pins of the oracle's SSP-RK3 integrator (section "Numerical methods": the paper's
strong-stability-preserving third-order Runge-Kutta method) and of its hand-reversed
discrete adjoint.  No GPU.

  * the Shu-Osher stages equal the method's published Butcher tableau
    (c = (0, 1, 1/2), a21 = 1, a31 = a32 = 1/4, b = (1/6, 1/6, 2/3)) to roundoff;
  * third order in time against a fine RK4 reference (error ratio 8 per halving);
  * the SSP property (bounds and total variation kept) on the forward-Euler-monotone
    upwind discretisation of inviscid Burgers at the forward-Euler step;
  * tangent against central differences of the step, adjoint against the tangent
    (dot product, one step and a whole sourced trajectory), and the adjoint gradient
    of Jbar against central finite differences.
"""
import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _p3(w, **kw):
    P = params_for(w, **kw)
    P.scheme = "ssprk3"
    return P


def test_shu_osher_stages_equal_butcher_tableau():
    w = synth.perturbed_uniform(6, 5, 3, seed=61, amp=0.08)
    P = _p3(w, mu=0.02, dt=3e-3)
    s = 0.05 * synth.random_field(w.shape, 62)
    got, (W1, W2, W3) = O.ssprk3_step(w, P, s)
    dt = P.dt
    k1 = O.residual(w, P, s)
    k2 = O.residual(w + dt * k1, P, s)
    k3 = O.residual(w + dt * (0.25 * k1 + 0.25 * k2), P, s)
    ref = w + dt * (k1 / 6.0 + k2 / 6.0 + 2.0 * k3 / 3.0)
    scale = np.max(np.abs(w))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(W3, w + dt * (0.25 * k1 + 0.25 * k2), rtol=0, atol=1e-14 * scale)


def test_third_order_in_time():
    """Same spatial operator, so the difference to a fine RK4 solution is the
    time-stepping error alone: it falls by 2^3 per halving of dt for SSP-RK3 (and by
    2^4 for RK4, a check of the harness)."""
    n = 16
    w0 = synth.isentropic_vortex(n, n, 1, noise=0.0)
    P = params_for(w0, mu=1e-3, dt=0.0)
    T = 0.04
    Pf = params_for(w0, mu=1e-3, dt=T / 256)
    ref = w0
    for _ in range(256):
        ref, _ = O.rk4_step(ref, Pf)
    errs = {}
    for scheme in ("ssprk3", "rk4"):
        e = []
        for m in (8, 16, 32):
            P.dt, P.scheme = T / m, scheme
            w = w0
            for _ in range(m):
                w, _ = O.step(w, P)
            e.append(np.max(np.abs(w - ref)))
        errs[scheme] = e
    r3 = [errs["ssprk3"][i] / errs["ssprk3"][i + 1] for i in range(2)]
    r4 = [errs["rk4"][i] / errs["rk4"][i + 1] for i in range(2)]
    assert all(6.5 < r < 9.5 for r in r3), (errs, r3)
    assert all(12.0 < r < 20.0 for r in r4), (errs, r4)


def test_strong_stability_on_upwind_burgers():
    """SSP: wherever forward Euler keeps a solution within its initial bounds, the SSP-RK3
    step does too, at the same step.  Inviscid Burgers with the upwind flux for u >= 0
    is such a discretisation (forward Euler is monotone for dt max u / dx <= 1); the
    residual is swapped for it for this check only."""
    n = 64
    u = np.full((5, 1, 1, n), 0.2)
    u[0, 0, 0, n // 4: n // 2] = 1.0

    def upwind_burgers(w, P, s=None):
        f = 0.5 * w * w
        return -(f - np.roll(f, 1, axis=3)) / P.dx[0]

    P = O.Params(dx=(1.0, 1.0, 1.0), dt=1.0)   # CFL = dt max u / dx = 1
    saved = O.residual
    try:
        O.residual = upwind_burgers
        w = u.copy()
        tv0 = np.abs(np.diff(w[0, 0, 0], append=w[0, 0, 0, :1])).sum()
        for _ in range(40):
            w, _ = O.ssprk3_step(w, P)
            tv = np.abs(np.diff(w[0, 0, 0], append=w[0, 0, 0, :1])).sum()
            assert w[0].min() >= 0.2 - 1e-14 and w[0].max() <= 1.0 + 1e-14
            assert tv <= tv0 + 1e-13
            tv0 = tv
    finally:
        O.residual = saved


def test_tangent_step_matches_central_differences():
    w = synth.perturbed_uniform(5, 4, 3, seed=63, amp=0.06)
    P = _p3(w, mu=0.02, dt=2e-3)
    dw = synth.random_field(w.shape, 64)
    h = 1e-6
    fd = (O.ssprk3_step(w + h * dw, P)[0] - O.ssprk3_step(w - h * dw, P)[0]) / (2 * h)
    t = O.ssprk3_tangent_step(w, dw, P)
    np.testing.assert_allclose(t, fd, rtol=0, atol=1e-7 * np.max(np.abs(fd)))


@pytest.mark.parametrize("with_nu", [False, True])
def test_adjoint_step_dot_product(with_nu):
    """<lam, T dw> = <T^T lam, dw> for one step; with the added viscosity, nu = 0
    reproduces the plain adjoint bit for bit and nu > 0 changes it."""
    w = synth.perturbed_uniform(6, 5, 3, seed=65, amp=0.05)
    P = _p3(w, mu=0.02, dt=2e-3)
    lam = synth.random_field(w.shape, 66)
    dw = synth.random_field(w.shape, 67)
    if not with_nu:
        l0, _ = O.ssprk3_adjoint_step(w, lam, P)
        t = O.ssprk3_tangent_step(w, dw, P)
        assert _rel(O.dot(lam, t), O.dot(l0, dw)) < 1e-13
    else:
        nu = np.abs(synth.random_field(w.shape[1:], 68)) * 1e-3
        a, _ = O.ssprk3_adjoint_step(w, lam, P)
        b, _ = O.ssprk3_adjoint_step(w, lam, P, nu=nu)
        # nu = 0 reproduces the plain adjoint bit for bit; nu > 0 changes it
        c, _ = O.ssprk3_adjoint_step(w, lam, P, nu=np.zeros(w.shape[1:]))
        assert np.array_equal(a, c)
        assert not np.allclose(a, b, rtol=1e-12, atol=0)


def test_trajectory_dot_product_with_source():
    w0 = synth.isentropic_vortex(12, 10, 1, noise=1e-3, seed=2)
    P = _p3(w0, mu=0.01, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.1 * synth.forcing_bumps(12, 10, 1, n=4)[1]
    ws, _ = O.primal_run(w0, P, 6, s)
    lam0, sbar = O.adjoint_run(ws, P, s)
    dw = synth.random_field(w0.shape, 8, 1e-2)
    ds = synth.random_field(w0.shape, 9, 1e-2)
    Jd = O.tangent_run(ws, dw, P, s, ds)
    assert _rel(Jd, O.dot(lam0, dw) + O.dot(sbar, ds)) < 1e-12


def test_trajectory_gradient_matches_central_fd():
    n = 16
    w0 = synth.isentropic_vortex(n, n, 1, noise=1e-3, seed=1)
    P = _p3(w0, mu=0.5 / 1000, dt=0.5 / n / 2.0)
    phi = synth.forcing_bumps(n, n, 1, n=4)
    steps = 8
    ws, _ = O.primal_run(w0, P, steps)
    lam0, sbar = O.adjoint_run(ws, P)
    eps = 1e-6
    dw = synth.random_field(w0.shape, 12)
    _, Jp = O.primal_run(w0 + eps * dw, P, steps)
    _, Jm = O.primal_run(w0 - eps * dw, P, steps)
    assert _rel((Jp - Jm) / (2 * eps), O.dot(lam0, dw)) < 1e-6
    ds = np.zeros_like(w0)
    ds[1] = phi[1]
    _, Jp = O.primal_run(w0, P, steps, eps * ds)
    _, Jm = O.primal_run(w0, P, steps, -eps * ds)
    assert _rel((Jp - Jm) / (2 * eps), O.dot(sbar, ds)) < 1e-6


def test_conserves_mass_momentum_energy():
    w = synth.perturbed_uniform(7, 5, 3, seed=69, amp=0.08)
    P = _p3(w, mu=0.02, dt=2e-3)
    tot0 = w.sum(axis=(1, 2, 3))
    for _ in range(5):
        w, _ = O.ssprk3_step(w, P)
    np.testing.assert_allclose(w.sum(axis=(1, 2, 3)), tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())
