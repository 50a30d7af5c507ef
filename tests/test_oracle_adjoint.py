"""Pins of the oracle's hand-derived tangent and transpose (the discrete adjoint of
section "Unsteady adjoint" / "Implementation") against brute-force finite-difference
Jacobians, against each other (dot-product identity), and against central finite
differences of the time-averaged objective.  No GPU."""
import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("shape", [(3, 4, 2), (4, 3, 1)])
def test_tangent_and_transpose_equal_fd_jacobian(shape):
    """Build the dense Jacobian dR/dw column by column with central differences of the
    residual; the tangent must reproduce J v and the transpose J^T a (FD-independent
    of either hand derivation)."""
    w = synth.perturbed_uniform(*shape, seed=11, amp=0.1)
    P = params_for(w, mu=0.05)
    n = w.size
    J = np.empty((n, n))
    h = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        e = e.reshape(w.shape)
        J[:, j] = ((O.residual(w + e, P) - O.residual(w - e, P)) / (2 * h)).ravel()
    v = synth.random_field(w.shape, 1)
    a = synth.random_field(w.shape, 2)
    Jv = O.residual_tangent(w, v, P).ravel()
    JTa = O.residual_transpose(w, a, P).ravel()
    scale = np.max(np.abs(J)) * 10
    np.testing.assert_allclose(Jv, J @ v.ravel(), atol=2e-7 * scale, rtol=0)
    np.testing.assert_allclose(JTa, J.T @ a.ravel(), atol=2e-7 * scale, rtol=0)


@pytest.mark.parametrize("shape", [(7, 5, 3), (9, 6, 1), (5, 7, 4), (2, 3, 5)])
def test_transpose_dot_product_identity(shape):
    """<a, J v> = <J^T a, v> to roundoff, with random a, v and a random state w."""
    w = synth.perturbed_uniform(*shape, seed=21, amp=0.08)
    P = params_for(w, mu=0.03)
    v = synth.random_field(w.shape, 3)
    a = synth.random_field(w.shape, 4)
    lhs = O.dot(a, O.residual_tangent(w, v, P))
    rhs = O.dot(O.residual_transpose(w, a, P), v)
    assert _rel(lhs, rhs) < 1e-13


def test_inviscid_transpose_is_euler_jacobian_transpose():
    """With mu = 0 the transpose at cell c is sum_d A_d(w_c)^T (a(c+e_d) - a(c-e_d))/(2dx)
    where A_d = dF_d/dw (section "Unsteady adjoint", the A_kji term): compare with A_d
    built by finite differences of the Euler flux cell by cell."""
    w = synth.perturbed_uniform(5, 4, 3, seed=31, amp=0.1)
    P = params_for(w, mu=0.0)
    a = synth.random_field(w.shape, 5)
    got = O.residual_transpose(w, a, P)
    ref = np.zeros_like(w)
    h = 1e-7
    for d in range(3):
        A = np.empty((5, 5) + w.shape[1:])
        for k in range(5):
            e = np.zeros_like(w)
            e[k] = h
            A[:, k] = (O.euler_flux(w + e, d, P) - O.euler_flux(w - e, d, P)) / (2 * h)
        da = (np.roll(a, -1, axis=3 - d) - np.roll(a, 1, axis=3 - d)) / (2 * P.dx[d])
        ref += np.einsum("ik...,i...->k...", A, da)
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=1e-7 * np.max(np.abs(ref)))


def test_rk4_step_adjoint_dot_product():
    """<lam, T delta w> = <T^T lam, delta w> for one RK4 step, T its tangent map, with
    added adjoint viscosity switched off and on (the viscosity operator is symmetric,
    so it enters both sides alike only in the adjoint: checked separately)."""
    w = synth.perturbed_uniform(6, 5, 3, seed=41, amp=0.05)
    P = params_for(w, mu=0.02, dt=2e-3)
    lam = synth.random_field(w.shape, 6)
    dw = synth.random_field(w.shape, 7)
    t = O.rk4_tangent_step(w, dw, P)
    l0, _ = O.rk4_adjoint_step(w, lam, P)
    assert _rel(O.dot(lam, t), O.dot(l0, dw)) < 1e-13


def test_trajectory_dot_product_with_source():
    """Dot-product test of the whole sweep: <lam^0, dw^0> + <sbar, ds> equals the tangent
    dJbar along (dw^0, ds), for a run with a nonzero source."""
    w0 = synth.isentropic_vortex(12, 10, 1, noise=1e-3, seed=2)
    P = params_for(w0, mu=0.01, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.1 * synth.forcing_bumps(12, 10, 1, n=4)[1]
    ws, _ = O.primal_run(w0, P, 6, s)
    lam0, sbar = O.adjoint_run(ws, P, s)
    dw = synth.random_field(w0.shape, 8, 1e-2)
    ds = synth.random_field(w0.shape, 9, 1e-2)
    Jd = O.tangent_run(ws, dw, P, s, ds)
    assert _rel(Jd, O.dot(lam0, dw) + O.dot(sbar, ds)) < 1e-12


def test_trajectory_gradient_matches_central_fd():
    """Central finite differences of Jbar (eps = 1e-6) along random initial-state
    directions and along two forcing shapes agree with the adjoint gradient
    (short, non-chaotic horizon)."""
    n = 16
    w0 = synth.isentropic_vortex(n, n, 1, noise=1e-3, seed=1)
    P = params_for(w0, mu=0.5 / 1000, dt=0.5 / n / 2.0)
    phi = synth.forcing_bumps(n, n, 1, n=4)
    steps = 8
    _, J0 = O.primal_run(w0, P, steps)
    ws, _ = O.primal_run(w0, P, steps)
    lam0, sbar = O.adjoint_run(ws, P)
    eps = 1e-6
    for seed in (12, 13):
        dw = synth.random_field(w0.shape, seed)
        _, Jp = O.primal_run(w0 + eps * dw, P, steps)
        _, Jm = O.primal_run(w0 - eps * dw, P, steps)
        fd = (Jp - Jm) / (2 * eps)
        assert _rel(fd, O.dot(lam0, dw)) < 1e-6, (fd, O.dot(lam0, dw))
    for m in (1, 2):
        ds = np.zeros_like(w0)
        ds[1] = phi[m]
        _, Jp = O.primal_run(w0, P, steps, eps * ds)
        _, Jm = O.primal_run(w0, P, steps, -eps * ds)
        fd = (Jp - Jm) / (2 * eps)
        assert _rel(fd, O.dot(sbar, ds)) < 1e-6, (fd, O.dot(sbar, ds))


def test_adjoint_viscosity_zero_is_bitwise_plain_adjoint():
    """nu = 0 everywhere reproduces the unstabilised adjoint bit for bit."""
    w = synth.perturbed_uniform(5, 4, 3, seed=51)
    P = params_for(w, mu=0.02, dt=2e-3)
    lam = synth.random_field(w.shape, 10)
    a, _ = O.rk4_adjoint_step(w, lam, P)
    b, _ = O.rk4_adjoint_step(w, lam, P, nu=np.zeros(w.shape[1:]))
    assert np.array_equal(a, b)


def test_viscosity_operator_symmetric_nsd_and_fourier_eigenvalue():
    """L_nu (section "Energy analysis", added lambda sigma_1 term) is symmetric and
    negative semidefinite; for constant nu a Fourier mode is an eigenvector with the
    discrete-Laplacian eigenvalue -nu sum_d (2 - 2 cos(2 pi k_d / n_d)) / dx_d^2."""
    shp = (6, 5, 4)
    w = synth.perturbed_uniform(*shp, seed=61)
    P = params_for(w)
    nu = np.abs(synth.random_field(shp[::-1], 14)) + 0.1
    a = synth.random_field(w.shape, 15)
    b = synth.random_field(w.shape, 16)
    La = O.viscosity_apply(a, nu, P)
    Lb = O.viscosity_apply(b, nu, P)
    assert _rel(O.dot(La, b), O.dot(a, Lb)) < 1e-13
    assert O.dot(a, La) < 0.0
    nx, ny, nz = shp
    k = (2, 1, 1)
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    mode = np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz))
    am = np.broadcast_to(mode, w.shape).copy()
    c = 0.37
    lam_ev = -c * sum((2 - 2 * np.cos(2 * np.pi * k[d] / (nx, ny, nz)[d])) / P.dx[d] ** 2
                      for d in range(3))
    np.testing.assert_allclose(O.viscosity_apply(am, np.full(shp[::-1], c), P), lam_ev * am,
                               rtol=1e-12, atol=1e-12 * abs(lam_ev))


def test_viscosity_split_scales_each_state_variable():
    """Per-variable adjoint viscosity (the conclusion's next step): with factors
    (f_rho, f_mom, f_en) each adjoint component equals the single-coefficient operator
    with nu scaled by its own factor, and the operator stays symmetric negative
    semidefinite for non-negative factors."""
    w = synth.perturbed_uniform(6, 5, 4, seed=81)
    P = params_for(w, mu=0.02, dt=2e-3)
    a = synth.random_field(w.shape, 82)
    b = synth.random_field(w.shape, 83)
    nu = np.abs(synth.random_field(w.shape[1:], 84)) * 1e-3
    f = (0.5, 2.0, 3.0)
    Ps = params_for(w, mu=0.02, dt=2e-3)
    Ps.nu_split = f
    got = O.viscosity_apply(a, nu, Ps)
    for v, fv in zip(range(5), (f[0], f[1], f[1], f[1], f[2])):
        ref = O.viscosity_apply(a, fv * nu, P)[v]
        np.testing.assert_allclose(got[v], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert O.dot(a, O.viscosity_apply(a, nu, Ps)) <= 0.0
    assert _rel(O.dot(a, O.viscosity_apply(b, nu, Ps)), O.dot(O.viscosity_apply(a, nu, Ps), b)) < 1e-13
