"""Pins of the oracle's symmetrisation, growth matrix M = M1 - M2, sigma_1 and the
adjoint energy (sections "Symmetrization" and "Energy analysis").  No GPU."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for


def _one_state(seed=0, g=1.4):
    rng = np.random.default_rng(seed)
    rho = 0.8 + 0.4 * rng.random()
    u = rng.standard_normal(3) * 0.4
    p = 0.5 + 0.5 * rng.random()
    return rho, u, p


def test_symmetrizer_makes_printed_Ahat():
    """T A_j T^-1 equals the printed symmetric A_hat_{:j:} for each direction, where
    A_j = dF_j/dw is taken by finite differences of the Euler flux and T = S V
    (section "Symmetrization").  This fixes S, V (including the sign of its
    -u_k/rho column) and the printed A_hat."""
    g = 1.4
    for seed in range(4):
        rho, u, p = _one_state(seed)
        w = synth._conservative(np.full((1, 1, 1), rho), u.reshape(3, 1, 1, 1) * np.ones((3, 1, 1, 1)),
                                np.full((1, 1, 1), p), g)
        P = O.Params(gamma=g)
        T = O.transform_T(w, P)[0, 0, 0]
        c = math.sqrt(g * p / rho)
        h = 1e-7
        for j in range(3):
            A = np.empty((5, 5))
            for k in range(5):
                e = np.zeros_like(w)
                e[k] = h
                A[:, k] = ((O.euler_flux(w + e, j, P) - O.euler_flux(w - e, j, P)) / (2 * h))[:, 0, 0, 0]
            Ah = T @ A @ np.linalg.inv(T)
            ref = O.symmetric_flux_matrix(u[j], c, j, g)
            np.testing.assert_allclose(Ah, ref, atol=3e-7)
            np.testing.assert_allclose(Ah, Ah.T, atol=3e-7)


def test_V_is_primitive_jacobian():
    """V = dq/dw with q = (rho, u, p): finite differences of the primitives."""
    g = 1.4
    rho, u, p = _one_state(3)
    w = synth._conservative(np.full((1, 1, 1), rho), u.reshape(3, 1, 1, 1) * np.ones((3, 1, 1, 1)),
                            np.full((1, 1, 1), p), g)
    P = O.Params(gamma=g)

    def q_of(ww):
        r, uu, e, pp = O.primitives(ww, P)
        return np.array([r.item(), uu[0].item(), uu[1].item(), uu[2].item(), pp.item()])

    h = 1e-7
    V = np.empty((5, 5))
    for k in range(5):
        e = np.zeros_like(w)
        e[k] = h
        V[:, k] = (q_of(w + e) - q_of(w - e)) / (2 * h)
    np.testing.assert_allclose(O.primitive_jacobian_V(np.array(rho), u, g), V, atol=1e-8)


def test_closed_form_growth_matrix_equals_definition():
    """The printed closed forms of M1 and M2 equal their definitions (dA_hat/dq,
    S and S^-1 of section "Energy analysis") when both are fed one consistent gradient
    (grad a, grad b from grad rho, grad p by the chain rule).  Random states and
    gradients; this pins the printed (partly garbled) matrices."""
    g = 1.4
    rng = np.random.default_rng(7)
    n = 20
    q = np.empty((5, n))
    q[0] = 0.7 + 0.6 * rng.random(n)
    q[1:4] = 0.5 * rng.standard_normal((3, n))
    q[4] = 0.4 + 0.6 * rng.random(n)
    dq = rng.standard_normal((5, 3, n))
    rho, p = q[0], q[4]
    c = np.sqrt(g * p / rho)
    dc = np.stack([c / 2 * (dq[4, j] / p - dq[0, j] / rho) for j in range(3)])
    db = dc / math.sqrt(g)
    da = dc * math.sqrt((g - 1) / g)
    Mg = O.growth_matrix_generic(q, dq, g)
    Mc = O.growth_matrix_closed(q, dq, db, da, g)
    np.testing.assert_allclose(Mc, Mg, rtol=1e-12, atol=1e-12)
    # M2 has a zero first column: dA_hat/dv_0 = 0 because c does not change along v_0
    M1 = O.growth_matrix_closed(q, np.zeros_like(dq), np.zeros_like(db), np.zeros_like(da), g)
    assert np.all(M1 == 0.0)


def test_solid_body_rotation_sigma1():
    """Uniform rho, p and a rigid rotation du1/dx2 = -Om, du2/dx1 = Om: M1 = 0 and M = -M2
    has the rotation block, so sigma_1 = Om."""
    g = 1.4
    Om = 0.83
    q = np.array([1.1, 0.2, -0.1, 0.0, 0.7]).reshape(5, 1)
    dq = np.zeros((5, 3, 1))
    dq[1, 1] = -Om
    dq[2, 0] = Om
    M = O.growth_matrix_closed(q, dq, np.zeros((3, 1)), np.zeros((3, 1)), g)
    s = np.linalg.svd(M[0], compute_uv=False)
    assert abs(s[0] - Om) < 1e-14


def test_sigma1_field_uniform_zero_and_svd_vs_eig():
    """sigma_1 = 0 on a uniform flow; on a random flow sigma_1 from the SVD equals
    sqrt(max eig(M^T M)) (two library routes); 2D uses the (rho, u1, u2, p) block."""
    g = 1.4
    rho = np.ones((3, 4, 5))
    u = np.stack([0.5 * rho, 0 * rho, 0 * rho])
    w = synth._conservative(rho, u, rho / g, g)
    P = params_for(w)
    assert np.all(O.sigma1_field(w, P) == 0.0)
    for shp in [(6, 5, 4), (7, 6, 1)]:
        w = synth.perturbed_uniform(*shp, seed=9, amp=0.1)
        P = params_for(w)
        s1 = O.sigma1_field(w, P)
        M = O.growth_matrix_field(w, P)
        if shp[2] == 1:
            idx = [0, 1, 2, 4]
            M = M[..., idx, :][..., :, idx]
        ev = np.linalg.eigvalsh(np.swapaxes(M, -1, -2) @ M)[..., -1]
        np.testing.assert_allclose(s1, np.sqrt(ev), rtol=1e-10)


def test_sigma1_converges_to_analytic_gradient_form():
    """With smooth periodic fields the central-difference M approaches the closed form
    evaluated with exact gradients at second order in dx."""
    g = 1.4
    errs = []
    for n in (16, 32):
        x = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        k = 2 * np.pi
        rho = 1 + 0.1 * np.sin(k * X) * np.cos(k * Z)
        u = np.stack([0.5 + 0.1 * np.sin(k * Y), 0.1 * np.cos(k * X), 0.1 * np.sin(k * Z)])
        p = (1 + 0.1 * np.cos(k * Y)) / g
        w = synth._conservative(rho, u, p, g)
        P = O.Params(gamma=g, dx=(1 / n, 1 / n, 1 / n))
        M = O.growth_matrix_field(w, P)
        q = np.stack([rho, u[0], u[1], u[2], p])
        dq = np.zeros((5, 3) + rho.shape)
        dq[0, 0] = 0.1 * k * np.cos(k * X) * np.cos(k * Z)
        dq[0, 2] = -0.1 * k * np.sin(k * X) * np.sin(k * Z)
        dq[1, 1] = 0.1 * k * np.cos(k * Y)
        dq[2, 0] = -0.1 * k * np.sin(k * X)
        dq[3, 2] = 0.1 * k * np.cos(k * Z)
        dq[4, 1] = -0.1 * k * np.sin(k * Y) / g
        c = np.sqrt(g * p / rho)
        dc = np.stack([c / 2 * (dq[4, j] / p - dq[0, j] / rho) for j in range(3)])
        Mex = O.growth_matrix_closed(q, dq, dc / math.sqrt(g), dc * math.sqrt((g - 1) / g), g)
        errs.append(np.max(np.abs(M - Mex)))
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_symmetric_adjoint_roundtrip_and_sensitivity_invariance():
    """w_hat = T^T v_hat (section "Symmetrization"): the solve round-trips, and the
    sensitivity is the same in either variable set: <w_hat, dw> = <v_hat, T dw>."""
    w = synth.perturbed_uniform(5, 4, 3, seed=71, amp=0.1)
    P = params_for(w)
    lam = synth.random_field(w.shape, 17)
    vh = O.symmetric_adjoint(w, lam, P)
    T = O.transform_T(w, P)
    back = np.einsum("...ki,k...->i...", T, vh)
    np.testing.assert_allclose(back, lam, rtol=1e-12, atol=1e-12)
    dw = synth.random_field(w.shape, 18)
    dv = np.einsum("...ik,k...->i...", T, dw)
    assert abs(O.dot(lam, dw) - O.dot(vh, dv)) < 1e-11 * abs(O.dot(lam, dw))
    E = O.adjoint_energy(w, lam, P)
    assert abs(E - np.sum(vh * vh) * np.prod(P.dx)) < 1e-12 * E


@pytest.mark.parametrize("shape", [(12, 5, 3), (7, 4, 1)])
def test_adjoint_energy_is_the_integral_of_vhat_squared(shape):
    """E_vhat = int v_hat . v_hat dV (section "Energy analysis", read as a sum of
    squares): on a uniform state with v_hat = (a sin(2 pi x / L_x), 0, b, 0, 0) the
    midpoint sum of sin^2 over a whole period is exactly half the cell count, so
    E = (a^2 / 2 + b^2) L_x L_y L_z at any resolution."""
    nx, ny, nz = shape
    g = 1.4
    rho = np.full((nz, ny, nx), 1.2)
    u = np.stack([np.full_like(rho, 0.4), np.full_like(rho, -0.1), np.zeros_like(rho)])
    w = synth._conservative(rho, u, np.full_like(rho, 0.8 / g), g)
    P = params_for(w)
    dx = P.dx
    x = (np.arange(nx) + 0.5) * dx[0]
    a, b = 0.7, -0.3
    vh = np.zeros_like(w)
    vh[0] = a * np.sin(2 * math.pi * x / (nx * dx[0]))
    vh[2] = b
    T = O.transform_T(w, P)
    lam = np.moveaxis(np.einsum("...ji,...j->...i", T, np.moveaxis(vh, 0, -1)), -1, 0)
    volume = nx * dx[0] * ny * dx[1] * nz * dx[2]
    assert O.adjoint_energy(w, lam, P) == pytest.approx((a * a / 2 + b * b) * volume, rel=1e-12)
