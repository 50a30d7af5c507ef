"""Pins of the oracle's Roe dissipation (section "Numerical methods": the approximate
Roe solver of the paper's flow solver) and of the residual, tangent and transpose with
it.  No GPU.

  * Roe's defining property: with the signed eigenvalues the dissipation operator is the
    Roe matrix, A~ (wR - wL) = F(wR) - F(wL), to roundoff, in every direction;
  * consistency (no dissipation between equal states) and upwinding (supersonic faces
    give F(wL) exactly);
  * the entropy fix is continuous with a continuous derivative at |lam| = delta;
  * the complex-step tangent and transpose against brute-force finite-difference
    Jacobians, the dot-product identity, uniform flow and conservation, and the adjoint
    of a whole trajectory against its tangent and against central differences of Jbar.
"""
import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for, uniform


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _roe(w, **kw):
    P = params_for(w, **kw)
    P.flux = "roe"
    return P


@pytest.mark.parametrize("d", [0, 1, 2])
def test_signed_dissipation_is_the_roe_matrix(d):
    wL = synth.perturbed_uniform(7, 5, 3, seed=101, amp=0.2)
    wR = synth.perturbed_uniform(7, 5, 3, seed=102, amp=0.2)
    P = _roe(wL)
    D = O.roe_dissipation(wL, wR, d, P, signed=True)
    ref = 0.5 * (O.euler_flux(wR, d, P) - O.euler_flux(wL, d, P))
    np.testing.assert_allclose(D, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_consistency_and_supersonic_upwinding():
    w = synth.perturbed_uniform(6, 4, 3, seed=103, amp=0.1)
    P = _roe(w)
    for d in range(3):
        assert np.array_equal(O.roe_dissipation(w, w, d, P), np.zeros_like(w))
    # supersonic along x (u ~ 2.5 c): every wave speed exceeds delta, so
    # (F_L + F_R)/2 - D = F_L
    rho = 1.0 + 0.1 * np.abs(synth.random_field((3, 4, 6), 104))
    g = 1.4
    uL = np.stack([2.5 + 0.05 * synth.random_field((3, 4, 6), 105), 0.1 * rho, -0.2 * rho])
    wL = synth._conservative(rho, uL, rho / g, g)
    wR = synth._conservative(1.1 * rho, uL * 1.05, 1.2 * rho / g, g)
    F = O.euler_flux(wL, 0, P)
    phi = 0.5 * (F + O.euler_flux(wR, 0, P)) - O.roe_dissipation(wL, wR, 0, P)
    np.testing.assert_allclose(phi, F, rtol=0, atol=1e-13 * np.abs(F).max())


def test_entropy_fix_is_c1_at_delta():
    delta = 0.3
    h = 1e-7
    for x0 in (delta, -delta):
        lo = O._abs_fix(np.array(x0 - h), delta, False)
        hi = O._abs_fix(np.array(x0 + h), delta, False)
        assert abs(hi - lo) < 3e-7                      # value continuous
        dl = (O._abs_fix(np.array(x0 - h), delta, False) - O._abs_fix(np.array(x0 - 2 * h), delta, False)) / h
        dr = (O._abs_fix(np.array(x0 + 2 * h), delta, False) - O._abs_fix(np.array(x0 + h), delta, False)) / h
        assert abs(dl - dr) < 1e-5                      # derivative continuous
        assert abs(dr - np.sign(x0)) < 1e-5


@pytest.mark.parametrize("shape", [(3, 4, 2), (4, 3, 1)])
def test_tangent_and_transpose_equal_fd_jacobian(shape):
    w = synth.perturbed_uniform(*shape, seed=106, amp=0.1)
    P = _roe(w, mu=0.05)
    n = w.size
    J = np.empty((n, n))
    h = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        e = e.reshape(w.shape)
        J[:, j] = ((O.residual(w + e, P) - O.residual(w - e, P)) / (2 * h)).ravel()
    v = synth.random_field(w.shape, 107)
    a = synth.random_field(w.shape, 108)
    scale = np.max(np.abs(J)) * 10
    np.testing.assert_allclose(O.residual_tangent(w, v, P).ravel(), J @ v.ravel(), atol=2e-7 * scale, rtol=0)
    np.testing.assert_allclose(O.residual_transpose(w, a, P).ravel(), J.T @ a.ravel(), atol=2e-7 * scale, rtol=0)


@pytest.mark.parametrize("shape", [(7, 5, 3), (9, 6, 1)])
def test_transpose_dot_product_identity(shape):
    w = synth.perturbed_uniform(*shape, seed=109, amp=0.08)
    P = _roe(w, mu=0.03)
    v = synth.random_field(w.shape, 110)
    a = synth.random_field(w.shape, 111)
    assert _rel(O.dot(a, O.residual_tangent(w, v, P)), O.dot(O.residual_transpose(w, a, P), v)) < 1e-13


def test_uniform_flow_and_conservation():
    w = uniform(5, 4, 3)
    P = _roe(w, mu=0.02)
    assert np.array_equal(O.residual(w, P), np.zeros_like(w))
    w = synth.perturbed_uniform(7, 5, 3, seed=112, amp=0.1)
    P = _roe(w, mu=0.02, dt=2e-3)
    tot0 = w.sum(axis=(1, 2, 3))
    for _ in range(4):
        w, _ = O.rk4_step(w, P)
    np.testing.assert_allclose(w.sum(axis=(1, 2, 3)), tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())


@pytest.mark.parametrize("scheme", ["rk4", "ssprk3"])
def test_trajectory_adjoint_dot_product_and_fd(scheme):
    n = 12
    w0 = synth.isentropic_vortex(n, 10, 1, noise=1e-3, seed=2)
    P = _roe(w0, mu=0.01, dt=4e-3)
    P.scheme = scheme
    s = np.zeros_like(w0)
    s[1] = 0.1 * synth.forcing_bumps(n, 10, 1, n=4)[1]
    ws, _ = O.primal_run(w0, P, 5, s)
    lam0, sbar = O.adjoint_run(ws, P, s)
    dw = synth.random_field(w0.shape, 113, 1e-2)
    ds = synth.random_field(w0.shape, 114, 1e-2)
    Jd = O.tangent_run(ws, dw, P, s, ds)
    assert _rel(Jd, O.dot(lam0, dw) + O.dot(sbar, ds)) < 1e-12
    eps = 1e-6
    _, Jp = O.primal_run(w0 + eps * dw, P, 5, s)
    _, Jm = O.primal_run(w0 - eps * dw, P, 5, s)
    assert _rel((Jp - Jm) / (2 * eps), O.dot(lam0, dw)) < 1e-6
