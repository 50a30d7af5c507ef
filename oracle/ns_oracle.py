"""Plain FP64 CPU oracle for the unsteady adjoint of the compressible Navier-Stokes
equations (Talnikar, Wang & Laskowski, "Unsteady adjoint of pressure loss for a
fundamental transonic turbine vane", arXiv 1511.06959).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it.
It shares no code with the CUDA path.  Every array is numpy float64; every stencil is
an ``np.roll`` on a periodic box, written so that it can be read against the paper.

Layout: one box is ``w[5, nz, ny, nx]`` with x fastest; w = (rho, rho u1, rho u2,
rho u3, rho E) as in Eq. (e:vector).  Direction d = 0, 1, 2 is x, y, z; it maps to
numpy axis 3 - d.  A 2D box is nz = 1: every z difference of a periodic size-1 axis
is exactly zero, so the 3D formulas reduce to 2D without a special case.  Boxes are
periodic, or (Params.bc = "inout") bounded in x by characteristic inflow and outflow
columns of ghost cells; see the section on characteristic boundaries.

Discretisation (readings of a paper whose own solver was SSP-RK3 + Roe on an
unstructured mesh, section "Numerical methods"):
  * convective face flux  Phi^c_{i+1/2} = (F(w_i) + F(w_{i+1})) / 2   (central, 2nd order),
    optionally minus the Roe dissipation |A~|(w_{i+1} - w_i)/2 of the paper's solver
  * viscous face flux from the face gradient of (u1, u2, u3, e): the normal part is the
    compact difference (q_{i+1} - q_i)/dx_d, the tangential parts are the mean of the
    two cell-centred central differences; the face velocity is the two-cell mean
  * R(w)_i = -sum_d (Phi_{d,i+1/2} - Phi_{d,i-1/2}) / dx_d + s_i,  Phi = Phi^c - F^v
  * classical RK4 in time with a constant dt, or the paper's SSP-RK3 (Shu-Osher form)
  * heat flux alpha grad e with alpha = gamma mu / Pr  (so alpha grad e = k grad T)

Functions whose result has no independent pin are marked "parity unpinned" in their
docstring; at present every function below is pinned by a test in tests/.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NVAR = 5


# ----------------------------------------------------------------------------------
# parameters and stencil helpers
# ----------------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Physical and discrete parameters of one periodic box.

    gamma, mu, Pr: ideal gas and constant viscosity of Eq. (e:navier).
    dx: cell sizes (dx, dy, dz).  dt: the constant time step.
    scheme: "rk4" (classical fourth-order Runge-Kutta) or "ssprk3" (the three-stage
    third-order strong-stability-preserving Runge-Kutta method of section "Numerical
    methods", in Shu-Osher form).
    nu_split: factors of the added adjoint viscosity for the adjoint of rho, of rho u
    (three components) and of rho E: the separate viscosities per state variable that
    the conclusion names as a next step; (1, 1, 1) is the single coefficient of section
    "Energy analysis".
    flux: "central" (Phi = (F_L + F_R)/2 - F^v) or "roe" (the approximate Roe solver of
    section "Numerical methods": the central flux minus the dissipation |A~|(w_R-w_L)/2).
    roe_delta: Harten's entropy fix, |lam| replaced by (lam^2 + delta^2)/(2 delta)
    where |lam| < delta, delta = roe_delta times the Roe-averaged sound speed.
    plane_i: the objective plane is the x-face between cell columns plane_i-1 and
    plane_i.  pt_in: the reference stagnation pressure p_{t,in} of Eq. (e:pressure_loss).
    bc: "periodic" (every direction); "inout": characteristic inflow at x = 0 and
    outflow at x = L_x (section "Numerical methods": non-reflecting inlet and outlet);
    "walls": isothermal no-slip walls at y = 0 and y = L_y (the vane surface is
    isothermal, section "Problem setup"); "inout_walls": both.  The other
    directions stay periodic.  far: the far-field primitive state (rho, u1, u2, u3, p)
    the characteristic conditions refer to.  wall_e: the internal energy e = c_v T of
    the bottom and the top wall.
    """

    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 0.72
    dx: tuple = (1.0, 1.0, 1.0)
    dt: float = 0.0
    plane_i: int = 0
    pt_in: float = 1.0
    scheme: str = "rk4"
    nu_split: tuple = (1.0, 1.0, 1.0)
    flux: str = "central"
    roe_delta: float = 0.1
    bc: str = "periodic"
    far: tuple = (1.0, 0.5, 0.0, 0.0, 1.0 / 1.4)
    wall_e: tuple = (1.0 / 0.56, 1.0 / 0.56)

    @property
    def alpha(self) -> float:
        """Heat-flux coefficient of Eq. (e:navier): alpha grad e = (mu c_p / Pr) grad T."""
        return self.gamma * self.mu / self.Pr


def _sh3(f, d, s):
    """sh for a field shaped (..., nz, ny, nx): the last three axes are the grid."""
    axis = f.ndim - 1 - d
    return np.roll(f, -s, axis=axis)


# ----------------------------------------------------------------------------------
# primitive variables and the Euler flux, Eq. (e:navier) and Eq. (e:vector)
# ----------------------------------------------------------------------------------
def primitives(w, P: Params):
    """rho, u[3], e, p from w = (rho, rho u, rho E): e = E - u.u/2, p = (gamma-1) rho e
    (Eq. e:navier)."""
    rho = w[0]
    u = w[1:4] / rho
    e = w[4] / rho - 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    p = (P.gamma - 1.0) * rho * e
    return rho, u, e, p


def euler_flux(w, d, P: Params):
    """Column d of F in Eq. (e:vector): (rho u_d, rho u_d u + p e_d, (rho E + p) u_d)."""
    rho, u, e, p = primitives(w, P)
    F = np.empty_like(w)
    F[0] = w[1 + d]
    for k in range(3):
        F[1 + k] = w[1 + d] * u[k]
    F[1 + d] += p
    F[4] = (w[4] + p) * u[d]
    return F


# ----------------------------------------------------------------------------------
# viscous face flux, Eq. (e:navier) stress and heat flux, Eq. (e:vector) F^v
# ----------------------------------------------------------------------------------
def _visc_q(w, P):
    """The four quantities whose gradients enter F^v: (u1, u2, u3, e)."""
    rho, u, e, p = primitives(w, P)
    return np.stack([u[0], u[1], u[2], e])


def face_gradient(q, d, P: Params):
    """Gradient g[k, l] of q_k at the face between c and c + e_d (for every c).

    Normal direction l = d: (q(c+e_d) - q(c)) / dx_d.
    Tangential l != d: mean of the cell-centred central differences at c and c + e_d.
    """
    g = np.empty((q.shape[0], 3) + q.shape[1:])
    for l in range(3):
        if l == d:
            g[:, l] = (_sh3(q, d, 1) - q) / P.dx[d]
        else:
            G = (_sh3(q, l, 1) - _sh3(q, l, -1)) / (2.0 * P.dx[l])
            g[:, l] = 0.5 * (G + _sh3(G, d, 1))
    return g


def stress_row(g, d, P: Params):
    """Row d of sigma = mu (grad u + grad u^T) - 2/3 mu (div u) I  (Eq. e:navier),
    from a velocity gradient g[k, l] = du_k/dx_l."""
    div = g[0, 0] + g[1, 1] + g[2, 2]
    sig = np.empty((3,) + g.shape[2:])
    for j in range(3):
        sig[j] = P.mu * (g[j, d] + g[d, j])
        if j == d:
            sig[j] -= (2.0 / 3.0) * P.mu * div
    return sig


def viscous_face_flux(w, d, P: Params):
    """F^v_d (Eq. e:vector) at the face between c and c + e_d:
    (0, sigma_d1, sigma_d2, sigma_d3, u_f . sigma_d + alpha de/dx_d)."""
    q = _visc_q(w, P)
    g = face_gradient(q, d, P)
    sig = stress_row(g, d, P)
    uf = 0.5 * (q[0:3] + _sh3(q[0:3], d, 1))
    Fv = np.zeros_like(w)
    Fv[1:4] = sig
    Fv[4] = uf[0] * sig[0] + uf[1] * sig[1] + uf[2] * sig[2] + P.alpha * g[3, d]
    return Fv


# ----------------------------------------------------------------------------------
# Roe dissipation (section "Numerical methods": the approximate Roe solver).  Written
# for real or complex arrays: the tangent and the transpose of this term are taken by
# complex-step differentiation, independently of any hand derivation.
# ----------------------------------------------------------------------------------
def _abs_fix(lam, delta, signed):
    """|lam| with Harten's entropy fix (C^1 at |lam| = delta); signed=True returns lam
    itself (the Roe matrix A~ instead of |A~|).  The sign is taken from the real part,
    so the function is complex-step differentiable."""
    if signed:
        return lam
    re = np.real(lam)
    mag = np.where(re >= 0, lam, -lam)
    return np.where(np.abs(re) < np.real(delta), (lam * lam + delta * delta) / (2.0 * delta), mag)


def roe_dissipation(wL, wR, d, P: Params, signed=False):
    """D = |A~(wL, wR)| (wR - wL) / 2 for a face with normal e_d (Roe 1981): Roe averages
    u~, H~ weighted by sqrt(rho), rho~ = sqrt(rho_L rho_R), c~^2 = (gamma-1)(H~ - |u~|^2/2);
    wave strengths of the acoustic waves (lam = u~_d -+ c~), the entropy wave and the two
    shear waves (lam = u~_d); eigenvectors of the Euler Jacobian at the Roe state."""
    g = P.gamma
    rL, rR = wL[0], wR[0]
    uL = [wL[1 + k] / rL for k in range(3)]
    uR = [wR[1 + k] / rR for k in range(3)]
    pL = (g - 1.0) * (wL[4] - 0.5 * rL * (uL[0] ** 2 + uL[1] ** 2 + uL[2] ** 2))
    pR = (g - 1.0) * (wR[4] - 0.5 * rR * (uR[0] ** 2 + uR[1] ** 2 + uR[2] ** 2))
    HL = (wL[4] + pL) / rL
    HR = (wR[4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    rt = sL * sR
    ut = [(sL * uL[k] + sR * uR[k]) / (sL + sR) for k in range(3)]
    Ht = (sL * HL + sR * HR) / (sL + sR)
    q2 = ut[0] ** 2 + ut[1] ** 2 + ut[2] ** 2
    c2 = (g - 1.0) * (Ht - 0.5 * q2)
    c = np.sqrt(c2)
    un = ut[d]
    dr, dp = rR - rL, pR - pL
    du = [uR[k] - uL[k] for k in range(3)]
    dun = du[d]
    a1 = (dp - rt * c * dun) / (2.0 * c2)
    a2 = dr - dp / c2
    a3 = (dp + rt * c * dun) / (2.0 * c2)
    delta = P.roe_delta * c
    l1 = _abs_fix(un - c, delta, signed)
    l2 = _abs_fix(un, delta, signed)
    l3 = _abs_fix(un + c, delta, signed)
    D = np.empty((5,) + np.shape(rL), dtype=np.result_type(wL, wR))
    D[0] = l1 * a1 + l2 * a2 + l3 * a3
    for k in range(3):
        n = 1.0 if k == d else 0.0
        D[1 + k] = (l1 * a1 * (ut[k] - c * n) + l2 * a2 * ut[k] + l3 * a3 * (ut[k] + c * n)
                    + l2 * rt * (du[k] - dun * n))
    D[4] = (l1 * a1 * (Ht - un * c) + l2 * a2 * 0.5 * q2 + l3 * a3 * (Ht + un * c)
            + l2 * rt * (ut[0] * du[0] + ut[1] * du[1] + ut[2] * du[2] - un * dun))
    return 0.5 * D


def _roe_face(w, d, P):
    """Roe dissipation at every face c + e_d/2 (left cell c)."""
    return roe_dissipation(w, _sh3(w, d, 1), d, P)


_CSTEP = 1e-30


def _roe_face_tangent(w, wd, d, P):
    """Directional derivative of _roe_face along wd, by complex step (exact to roundoff)."""
    wc = w + 1j * _CSTEP * wd
    return np.imag(roe_dissipation(wc, _sh3(wc, d, 1), d, P)) / _CSTEP


def _roe_face_jacobians(w, d, P):
    """JL[i, j], JR[i, j] = dD_i/dwL_j, dD_i/dwR_j at every face, by complex step."""
    wR = _sh3(w, d, 1)
    JL = np.empty((5, 5) + w.shape[1:])
    JR = np.empty((5, 5) + w.shape[1:])
    for j in range(5):
        e = np.zeros((5,) + (1,) * (w.ndim - 1))
        e[j] = _CSTEP
        JL[:, j] = np.imag(roe_dissipation(w + 1j * e, wR, d, P)) / _CSTEP
        JR[:, j] = np.imag(roe_dissipation(w, wR + 1j * e, d, P)) / _CSTEP
    return JL, JR


# ----------------------------------------------------------------------------------
# residual R(w): dw/dt = R(w), Eq. (e:vector) with the source s_i
# ----------------------------------------------------------------------------------
def face_flux(w, d, P: Params):
    """Total face flux Phi_d = (F_d(c) + F_d(c+e_d))/2 - F^v_d at the face c + e_d/2, minus
    the Roe dissipation when P.flux == "roe"."""
    F = euler_flux(w, d, P)
    Phi = 0.5 * (F + _sh3(F, d, 1)) - viscous_face_flux(w, d, P)
    if P.flux == "roe":
        Phi = Phi - _roe_face(w, d, P)
    return Phi


def residual(w, P: Params, s=None):
    """R(w) = -div(F - F^v) + s, in flux-difference form on the periodic box
    (Eq. e:vector and the source-term equation that follows it); with P.bc = "inout"
    the same on the box padded by the characteristic ghost columns."""
    if P.bc != "periodic":
        return _bounded_residual(w, P, s)
    R = np.zeros_like(w)
    for d in range(3):
        Phi = face_flux(w, d, P)
        R -= (Phi - _sh3(Phi, d, -1)) / P.dx[d]
    if s is not None:
        R = R + s
    return R


# ----------------------------------------------------------------------------------
# tangent (dR/dw) wdot, derived by hand (forward mode, same step order as residual)
# ----------------------------------------------------------------------------------
def primitives_tangent(w, wd, P: Params):
    rho, u, e, p = primitives(w, P)
    rhod = wd[0]
    ud = (wd[1:4] - u * rhod) / rho
    ed = (wd[4] - rhod * w[4] / rho) / rho - (u[0] * ud[0] + u[1] * ud[1] + u[2] * ud[2])
    pd = (P.gamma - 1.0) * (rhod * e + rho * ed)
    return rhod, ud, ed, pd


def residual_tangent(w, wd, P: Params):
    """(dR/dw) wd: the linearisation of residual(w) along wd (source is w-independent)."""
    if P.bc != "periodic":
        return _bounded_tangent(w, wd, P)
    rho, u, e, p = primitives(w, P)
    rhod, ud, ed, pd = primitives_tangent(w, wd, P)
    q = np.stack([u[0], u[1], u[2], e])
    qd = np.stack([ud[0], ud[1], ud[2], ed])
    Rd = np.zeros_like(w)
    for d in range(3):
        # Euler flux tangent
        Fd = np.empty_like(w)
        Fd[0] = wd[1 + d]
        for k in range(3):
            Fd[1 + k] = wd[1 + d] * u[k] + w[1 + d] * ud[k]
        Fd[1 + d] += pd
        Fd[4] = (wd[4] + pd) * u[d] + (w[4] + p) * ud[d]
        # viscous flux tangent
        g = face_gradient(q, d, P)
        gd = face_gradient(qd, d, P)
        sig = stress_row(g, d, P)
        sigd = stress_row(gd, d, P)
        uf = 0.5 * (q[0:3] + _sh3(q[0:3], d, 1))
        ufd = 0.5 * (qd[0:3] + _sh3(qd[0:3], d, 1))
        Fvd = np.zeros_like(w)
        Fvd[1:4] = sigd
        Fvd[4] = sum(ufd[j] * sig[j] + uf[j] * sigd[j] for j in range(3)) + P.alpha * gd[3, d]
        Phid = 0.5 * (Fd + _sh3(Fd, d, 1)) - Fvd
        if P.flux == "roe":
            Phid = Phid - _roe_face_tangent(w, wd, d, P)
        Rd -= (Phid - _sh3(Phid, d, -1)) / P.dx[d]
    return Rd


# ----------------------------------------------------------------------------------
# transpose (dR/dw)^T a, derived by hand (reverse mode through the same steps)
# ----------------------------------------------------------------------------------
def residual_transpose(w, a, P: Params):
    """(dR/dw)^T a: the exact transpose of the discrete residual.  This is the discrete
    counterpart of the A_kji, A^v_kji and D_kjil terms of the continuous adjoint
    equation (section "Unsteady adjoint"); the paper obtained it by automatic
    differentiation ("Implementation"), here each step of residual() is reversed by
    hand, last step first."""
    if P.bc != "periodic":
        return _bounded_transpose(w, a, P)
    rho, u, e, p = primitives(w, P)
    q = np.stack([u[0], u[1], u[2], e])
    gm1 = P.gamma - 1.0
    # adjoints of the cell quantities w (direct use), u, e, p, rho
    wb = np.zeros_like(w)
    ub = np.zeros_like(u)
    eb = np.zeros_like(e)
    pb = np.zeros_like(p)
    for d in range(3):
        # R -= (Phi(c) - Phi(c - e_d)) / dx  ->  Phi_bar(c) = (a(c + e_d) - a(c)) / dx
        Phib = (_sh3(a, d, 1) - a) / P.dx[d]
        if P.flux == "roe":
            # Phi -= D(w(c), w(c+e_d)): w_bar(c) -= JL^T Phi_bar, w_bar(c+e_d) -= JR^T Phi_bar
            JL, JR = _roe_face_jacobians(w, d, P)
            wb -= np.einsum("ij...,i...->j...", JL, Phib)
            wb -= _sh3(np.einsum("ij...,i...->j...", JR, Phib), d, -1)
        # Phi = (F(c) + F(c+e_d))/2 - Fv  ->  F_bar(c) = (Phi_bar(c) + Phi_bar(c-e_d))/2
        Fb = 0.5 * (Phib + _sh3(Phib, d, -1))
        Fvb = -Phib
        # reverse of the Euler flux: F0 = m_d; F_{1+k} = m_d u_k + p delta_dk;
        # F4 = (rhoE + p) u_d
        wb[1 + d] += Fb[0]
        for k in range(3):
            wb[1 + d] += Fb[1 + k] * u[k]
            ub[k] += Fb[1 + k] * w[1 + d]
        pb += Fb[1 + d]
        wb[4] += Fb[4] * u[d]
        pb += Fb[4] * u[d]
        ub[d] += Fb[4] * (w[4] + p)
        # reverse of the viscous face flux
        g = face_gradient(q, d, P)
        sig = stress_row(g, d, P)
        uf = 0.5 * (q[0:3] + _sh3(q[0:3], d, 1))
        sigb = np.empty_like(sig)
        ufb = np.empty_like(uf)
        for j in range(3):
            sigb[j] = Fvb[1 + j] + Fvb[4] * uf[j]
            ufb[j] = Fvb[4] * sig[j]
        gb = np.zeros_like(g)
        gb[3, d] = P.alpha * Fvb[4]
        for j in range(3):
            gb[j, d] += P.mu * sigb[j]
            gb[d, j] += P.mu * sigb[j]
        for m in range(3):
            gb[m, m] -= (2.0 / 3.0) * P.mu * sigb[d]
        # face velocity u_f = (u(c) + u(c+e_d))/2
        qb = np.zeros_like(q)
        qb[0:3] += 0.5 * (ufb + _sh3(ufb, d, -1))
        # face gradient (see face_gradient)
        for l in range(3):
            if l == d:
                qb += (_sh3(gb[:, l], d, -1) - gb[:, l]) / P.dx[d]
            else:
                Gb = 0.5 * (gb[:, l] + _sh3(gb[:, l], d, -1))
                qb += (_sh3(Gb, l, -1) - _sh3(Gb, l, 1)) / (2.0 * P.dx[l])
        ub += qb[0:3]
        eb += qb[3]
    # p = (gamma-1) rho e
    rhob = gm1 * e * pb
    eb = eb + gm1 * rho * pb
    # e = rhoE/rho - |u|^2/2
    wb[4] += eb / rho
    rhob -= eb * w[4] / rho ** 2
    ub = ub - eb * u
    # u = m / rho
    wb[1:4] += ub / rho
    rhob -= (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) / rho
    wb[0] += rhob
    return wb


# ----------------------------------------------------------------------------------
# RK4 in time: primal, tangent and the discrete adjoint of one step
# ----------------------------------------------------------------------------------
def rk4_step(w, P: Params, s=None):
    """Classical RK4 with constant dt.  Returns w^{n+1} and the stage states W1..W4."""
    dt = P.dt
    W1 = w
    k1 = residual(W1, P, s)
    W2 = w + 0.5 * dt * k1
    k2 = residual(W2, P, s)
    W3 = w + 0.5 * dt * k2
    k3 = residual(W3, P, s)
    W4 = w + dt * k3
    k4 = residual(W4, P, s)
    wn = w + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return wn, (W1, W2, W3, W4)


def rk4_tangent_step(w, wd, P: Params, s=None, sd=None):
    """Linearisation of rk4_step (primal source s) along (wd, sd): returns wd^{n+1}."""
    dt = P.dt
    _, (W1, W2, W3, W4) = rk4_step(w, P, s)
    add = (lambda x: x) if sd is None else (lambda x: x + sd)
    k1d = add(residual_tangent(W1, wd, P))
    W2d = wd + 0.5 * dt * k1d
    k2d = add(residual_tangent(W2, W2d, P))
    W3d = wd + 0.5 * dt * k2d
    k3d = add(residual_tangent(W3, W3d, P))
    W4d = wd + dt * k3d
    k4d = add(residual_tangent(W4, W4d, P))
    return wd + dt / 6.0 * (k1d + 2.0 * k2d + 2.0 * k3d + k4d)


def rk4_adjoint_step(w, lam, P: Params, s=None, nu=None):
    """Discrete adjoint of one RK4 step: given lam = dJ/dw^{n+1}, return
    (dw^{n+1}/dw^n)^T lam and the sum of the four stage seeds abar_i, whose inner
    product with a source direction gives the source sensitivity (the delta J =
    -int int w_hat delta s statement of section "Unsteady adjoint", in discrete form).

    With nu given, each stage product J_i^T abar_i also receives L_nu abar_i, the
    added adjoint viscosity of section "Energy analysis" (lambda sigma_1 delta_ki
    delta_jl term), with nu evaluated once per step.
    """
    dt = P.dt
    _, (W1, W2, W3, W4) = rk4_step(w, P, s)

    def JT(W, ab):
        g = residual_transpose(W, ab, P)
        if nu is not None:
            g = g + viscosity_apply(ab, nu, P)
        return g

    a4 = dt / 6.0 * lam
    g4 = JT(W4, a4)
    a3 = dt / 3.0 * lam + dt * g4
    g3 = JT(W3, a3)
    a2 = dt / 3.0 * lam + 0.5 * dt * g3
    g2 = JT(W2, a2)
    a1 = dt / 6.0 * lam + 0.5 * dt * g2
    g1 = JT(W1, a1)
    return lam + g1 + g2 + g3 + g4, a1 + a2 + a3 + a4


# ----------------------------------------------------------------------------------
# SSP-RK3, section "Numerical methods": the three-stage, third-order strong-stability-
# preserving Runge-Kutta method, written in its Shu-Osher form (each stage a convex
# combination of forward-Euler steps):
#     W2 = w + dt R(w)
#     W3 = 3/4 w + 1/4 (W2 + dt R(W2))
#     w' = 1/3 w + 2/3 (W3 + dt R(W3))
# ----------------------------------------------------------------------------------
def ssprk3_step(w, P: Params, s=None):
    """One SSP-RK3 step with constant dt.  Returns w^{n+1} and the stage states W1..W3."""
    dt = P.dt
    W1 = w
    W2 = w + dt * residual(W1, P, s)
    W3 = 0.75 * w + 0.25 * (W2 + dt * residual(W2, P, s))
    wn = w / 3.0 + 2.0 / 3.0 * (W3 + dt * residual(W3, P, s))
    return wn, (W1, W2, W3)


def ssprk3_tangent_step(w, wd, P: Params, s=None, sd=None):
    """Linearisation of ssprk3_step along (wd, sd): returns wd^{n+1}."""
    dt = P.dt
    _, (W1, W2, W3) = ssprk3_step(w, P, s)
    add = (lambda x: x) if sd is None else (lambda x: x + sd)
    W2d = wd + dt * add(residual_tangent(W1, wd, P))
    W3d = 0.75 * wd + 0.25 * (W2d + dt * add(residual_tangent(W2, W2d, P)))
    return wd / 3.0 + 2.0 / 3.0 * (W3d + dt * add(residual_tangent(W3, W3d, P)))


def ssprk3_adjoint_step(w, lam, P: Params, s=None, nu=None):
    """Discrete adjoint of one SSP-RK3 step, the Shu-Osher stages reversed by hand:
    given lam = dJ/dw^{n+1}, return (dw^{n+1}/dw^n)^T lam and the sum of the adjoints
    of the three stage residuals (the source sensitivity seeds, as in rk4_adjoint_step).
    nu adds L_nu to every stage product, as in rk4_adjoint_step."""
    dt = P.dt
    _, (W1, W2, W3) = ssprk3_step(w, P, s)

    def JT(W, ab):
        g = residual_transpose(W, ab, P)
        if nu is not None:
            g = g + viscosity_apply(ab, nu, P)
        return g

    # w' = w/3 + 2/3 W3 + 2/3 dt R(W3)
    wbar = lam / 3.0
    r3 = 2.0 / 3.0 * dt * lam
    W3bar = 2.0 / 3.0 * lam + JT(W3, r3)
    # W3 = 3/4 w + 1/4 W2 + 1/4 dt R(W2)
    wbar = wbar + 0.75 * W3bar
    r2 = 0.25 * dt * W3bar
    W2bar = 0.25 * W3bar + JT(W2, r2)
    # W2 = w + dt R(w)
    wbar = wbar + W2bar
    r1 = dt * W2bar
    wbar = wbar + JT(W1, r1)
    return wbar, r1 + r2 + r3


def step(w, P: Params, s=None):
    """One step of the scheme P.scheme: (w^{n+1}, stage states)."""
    return ssprk3_step(w, P, s) if P.scheme == "ssprk3" else rk4_step(w, P, s)


def tangent_step(w, wd, P: Params, s=None, sd=None):
    return (ssprk3_tangent_step if P.scheme == "ssprk3" else rk4_tangent_step)(w, wd, P, s, sd)


def adjoint_step(w, lam, P: Params, s=None, nu=None):
    return (ssprk3_adjoint_step if P.scheme == "ssprk3" else rk4_adjoint_step)(w, lam, P, s, nu)


# ----------------------------------------------------------------------------------
# pressure-loss objective, Eq. (e:pressure_loss)
# ----------------------------------------------------------------------------------
def stagnation_pressure(rho, m, rhoE, P: Params):
    """p_t = p (1 + (gamma-1)/2 M^2)^(gamma/(gamma-1)) from conservative values
    (Eq. e:pressure_loss), with M^2 = |u|^2 / c^2 and c^2 = gamma p / rho."""
    u2 = (m[0] ** 2 + m[1] ** 2 + m[2] ** 2) / rho ** 2
    p = (P.gamma - 1.0) * (rhoE - 0.5 * rho * u2)
    c2 = P.gamma * p / rho
    M2 = u2 / c2
    return p * (1.0 + 0.5 * (P.gamma - 1.0) * M2) ** (P.gamma / (P.gamma - 1.0))


def plane_state(w, P: Params):
    """Face state on the objective plane: the mean of the two cell columns around it."""
    i0 = P.plane_i
    return 0.5 * (w[..., (i0 - 1) % w.shape[-1]] + w[..., i0 % w.shape[-1]])


def objective(w, P: Params):
    """Instantaneous pressure loss J^n = [sum_f rho_f (p_t,in - p_t,f)] / [sum_f rho_f]
    / p_t,in over the plane's faces (Eq. e:pressure_loss, inner integrals; uniform face
    area cancels)."""
    wf = plane_state(w, P)
    pt = stagnation_pressure(wf[0], wf[1:4], wf[4], P)
    N = np.sum(wf[0] * (P.pt_in - pt))
    D = np.sum(wf[0])
    return N / D / P.pt_in


def objective_grad(w, P: Params):
    """dJ^n/dw (a field, nonzero on the two columns around the plane), by hand."""
    g = P.gamma
    wf = plane_state(w, P)
    rho, m, rE = wf[0], wf[1:4], wf[4]
    m2 = m[0] ** 2 + m[1] ** 2 + m[2] ** 2
    p = (g - 1.0) * (rE - 0.5 * m2 / rho)
    X = m2 / (rho * p)                    # = rho |u|^2 / p, so M^2 = X / gamma
    kap = 0.5 * (g - 1.0) / g
    base = 1.0 + kap * X
    ex = g / (g - 1.0)
    pt = p * base ** ex
    N = np.sum(rho * (P.pt_in - pt))
    D = np.sum(rho)
    # J = N / (D pt_in)
    Nb = 1.0 / (D * P.pt_in)
    Db = -N / (D ** 2 * P.pt_in)
    rhob = Nb * (P.pt_in - pt) + Db
    ptb = -Nb * rho
    # pt = p base^ex, base = 1 + kap X
    pb = ptb * base ** ex
    Xb = ptb * p * ex * base ** (ex - 1.0) * kap
    # X = m2 / (rho p)
    m2b = Xb / (rho * p)
    rhob = rhob - Xb * m2 / (rho ** 2 * p)
    pb = pb - Xb * m2 / (rho * p ** 2)
    # p = (g-1)(rE - m2/(2 rho))
    rEb = (g - 1.0) * pb
    m2b = m2b - (g - 1.0) * pb / (2.0 * rho)
    rhob = rhob + (g - 1.0) * pb * m2 / (2.0 * rho ** 2)
    wfb = np.empty_like(wf)
    wfb[0] = rhob
    for k in range(3):
        wfb[1 + k] = 2.0 * m[k] * m2b
    wfb[4] = rEb
    G = np.zeros_like(w)
    i0 = P.plane_i
    nx = w.shape[-1]
    G[..., (i0 - 1) % nx] += 0.5 * wfb
    G[..., i0 % nx] += 0.5 * wfb
    return G


# ----------------------------------------------------------------------------------
# characteristic inflow and outflow (section "Numerical methods": non-reflecting inlet
# and outlet; section "Energy analysis": the incoming characteristics are set on the
# inlet and outlet), and isothermal no-slip walls (the vane surface is isothermal).
# Inflow and outflow are the x-faces of the box, walls the y-faces; z stays periodic.
# Each boundary gets one ghost column holding the boundary state of the Riemann
# invariants of the x direction, R+- = u1 +- 2c/(gamma-1), with the entropy p/rho^gamma
# and the tangential velocity carried by the flow: at the outflow R+, the entropy and
# the tangential velocity come from the adjacent cell and R- from the far field; at the
# inflow R- comes from the adjacent cell and the rest from the far field (subsonic flow
# along +x).  The residual is the periodic residual of the padded box, cropped: every
# face next to a boundary, its tangential differences included, sees the ghost.  The
# functions below work on real or complex arrays, so the ghosts' Jacobians are taken by
# complex-step differentiation.
# ----------------------------------------------------------------------------------
def _periodic(P: Params):
    return dataclasses.replace(P, bc="periodic")


def characteristic_state(wc, P: Params, side):
    """Ghost (boundary) state next to the cells wc[5, ...] on side "in" (x = 0) or
    "out" (x = L_x), in conservative variables."""
    g = P.gamma
    k = 2.0 / (g - 1.0)
    rho = wc[0]
    u = wc[1:4] / rho
    p = (g - 1.0) * (wc[4] - 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    c = np.sqrt(g * p / rho)
    rf, uf1, uf2, uf3, pf = P.far
    cf = math.sqrt(g * pf / rf)
    if side == "out":
        Rp, Rm = u[0] + k * c, uf1 - k * cf
        ent, ut2, ut3 = p / rho ** g, u[1], u[2]
    elif side == "in":
        Rp, Rm = uf1 + k * cf, u[0] - k * c
        ent = pf / rf ** g + 0.0 * rho
        ut2, ut3 = uf2 + 0.0 * rho, uf3 + 0.0 * rho
    else:
        raise ValueError(side)
    ub = 0.5 * (Rp + Rm)
    cb = 0.25 * (g - 1.0) * (Rp - Rm)
    rhob = (cb * cb / (g * ent)) ** (1.0 / (g - 1.0))
    pb = rhob * cb * cb / g
    out = np.empty(wc.shape, dtype=np.result_type(wc, cb))
    out[0] = rhob
    out[1] = rhob * ub
    out[2] = rhob * ut2
    out[3] = rhob * ut3
    out[4] = pb / (g - 1.0) + 0.5 * rhob * (ub * ub + ut2 * ut2 + ut3 * ut3)
    return out


def wall_state(wc, P: Params, side):
    """Ghost state of an isothermal no-slip wall next to the cells wc[5, ...] on side
    "bottom" (y = 0) or "top" (y = L_y): the same density, the velocity reversed (the
    face velocity is zero) and e_g = 2 e_w - e (the face internal energy, so the face
    temperature, is the wall's), e_w = P.wall_e[0] or [1].  The mean of cell and ghost
    carries no mass through the wall."""
    ew = P.wall_e[0] if side == "bottom" else P.wall_e[1]
    rho = wc[0]
    u = wc[1:4] / rho
    e = wc[4] / rho - 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    eg = 2.0 * ew - e
    out = np.empty(wc.shape, dtype=wc.dtype)
    out[0] = rho
    out[1:4] = -wc[1:4]
    out[4] = rho * (eg + 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    return out


def _x_bounded(P: Params):
    return P.bc in ("inout", "inout_walls")


def _y_walls(P: Params):
    return P.bc in ("walls", "inout_walls")


def pad_x(w, P: Params):
    """w[5, nz, ny, nx] -> [5, nz, ny, nx + 2] with the inflow ghost column first and the
    outflow ghost column last."""
    return np.concatenate([characteristic_state(w[..., :1], P, "in"), w,
                           characteristic_state(w[..., -1:], P, "out")], axis=-1)


def pad_y(w, P: Params):
    """w[5, nz, ny, n] -> [5, nz, ny + 2, n] with the bottom wall's ghost row first and
    the top wall's last."""
    return np.concatenate([wall_state(w[..., :1, :], P, "bottom"), w,
                           wall_state(w[..., -1:, :], P, "top")], axis=-2)


def pad(w, P: Params):
    """The box with its ghost layers: x columns first, then y rows over them (so the
    corner ghosts are the walls' ghosts of the inflow and outflow ghosts)."""
    if _x_bounded(P):
        w = pad_x(w, P)
    if _y_walls(P):
        w = pad_y(w, P)
    return w


def _crop_cells(P: Params):
    """Index of the interior cells in a padded scalar field [nz, ny', nx']."""
    return (slice(None), slice(1, -1) if _y_walls(P) else slice(None),
            slice(1, -1) if _x_bounded(P) else slice(None))


def _crop(P: Params):
    return (slice(None),) + _crop_cells(P)


def _zero_pad(f, P: Params):
    width = [(0, 0)] * (f.ndim - 2) + [(1, 1) if _y_walls(P) else (0, 0), (1, 1) if _x_bounded(P) else (0, 0)]
    return np.pad(f, width)


def _cs_jacobian(fn, wc, h=1e-30):
    """J[i, k, ...] = d fn(wc)_i / d wc_k for a cell-local map, by complex-step
    differentiation (exact to roundoff)."""
    J = np.empty((5,) + wc.shape)
    for k in range(5):
        z = wc.astype(complex)
        z[k] += 1j * h
        J[:, k] = fn(z).imag / h
    return J


def ghost_jacobian(wc, P: Params, side, h=1e-30):
    """G[i, k, ...] = d ghost_i / d wc_k of a characteristic ("in", "out") or wall
    ("bottom", "top") ghost, by complex-step differentiation."""
    state = characteristic_state if side in ("in", "out") else wall_state
    return _cs_jacobian(lambda z: state(z, P, side), wc, h)


def _bounded_residual(w, P: Params, s=None):
    sp = None if s is None else _zero_pad(s, P)
    return residual(pad(w, P), _periodic(P), sp)[_crop(P)]


def _bounded_tangent(w, wd, P: Params):
    """(dR/dw) wd: the periodic tangent of the padded box along the padded direction
    (each ghost's Jacobian applied to the direction at its adjacent cells)."""
    if _x_bounded(P):
        Gi = ghost_jacobian(w[..., :1], P, "in")
        Go = ghost_jacobian(w[..., -1:], P, "out")
        wd = np.concatenate([np.einsum("ik...,k...->i...", Gi, wd[..., :1]), wd,
                             np.einsum("ik...,k...->i...", Go, wd[..., -1:])], axis=-1)
        w = pad_x(w, P)
    if _y_walls(P):
        Gb = ghost_jacobian(w[..., :1, :], P, "bottom")
        Gt = ghost_jacobian(w[..., -1:, :], P, "top")
        wd = np.concatenate([np.einsum("ik...,k...->i...", Gb, wd[..., :1, :]), wd,
                             np.einsum("ik...,k...->i...", Gt, wd[..., -1:, :])], axis=-2)
        w = pad_y(w, P)
    return residual_tangent(w, wd, _periodic(P))[_crop(P)]


def _bounded_transpose(w, a, P: Params):
    """(dR/dw)^T a by the chain rule through the padding: the periodic transpose of the
    padded box, then the wall rows' adjoints pulled back to their adjacent rows, then
    the inflow and outflow columns' to theirs, each with the transposed ghost Jacobian
    (the reverse of the order the padding was built in)."""
    wx = pad_x(w, P) if _x_bounded(P) else w
    b = residual_transpose(pad(w, P), _zero_pad(a, P), _periodic(P))
    if _y_walls(P):
        Gb = ghost_jacobian(wx[..., :1, :], P, "bottom")
        Gt = ghost_jacobian(wx[..., -1:, :], P, "top")
        out = b[..., 1:-1, :].copy()
        out[..., :1, :] += np.einsum("ik...,i...->k...", Gb, b[..., :1, :])
        out[..., -1:, :] += np.einsum("ik...,i...->k...", Gt, b[..., -1:, :])
        b = out
    if _x_bounded(P):
        Gi = ghost_jacobian(w[..., :1], P, "in")
        Go = ghost_jacobian(w[..., -1:], P, "out")
        out = b[..., 1:-1].copy()
        out[..., :1] += np.einsum("ik...,i...->k...", Gi, b[..., :1])
        out[..., -1:] += np.einsum("ik...,i...->k...", Go, b[..., -1:])
        b = out
    return b


# ----------------------------------------------------------------------------------
# whole trajectories: primal, tangent and adjoint with every state stored
# ----------------------------------------------------------------------------------
def primal_run(w0, P: Params, nsteps, s=None):
    """w^0 .. w^N and the time-averaged objective Jbar = (1/N) sum_{n=1..N} J(w^n)
    (Eq. e:pressure_loss with the time integral as a right-endpoint mean)."""
    ws = [w0]
    Jbar = 0.0
    for n in range(nsteps):
        wn, _ = step(ws[-1], P, s)
        ws.append(wn)
        Jbar += objective(wn, P) / nsteps
    return ws, Jbar


def adjoint_run(ws, P: Params, s=None, nu=None):
    """Backward sweep from the terminal condition (zero adjoint after the last step,
    section "Unsteady adjoint"): returns dJbar/dw^0 and the time sum of the stage
    seeds (for source sensitivities).  nu, when given, is a per-step callable
    nu(w^n) returning the adjoint-viscosity field, or a fixed field."""
    N = len(ws) - 1
    lam = np.zeros_like(ws[0])
    sbar = np.zeros_like(ws[0])
    for n in range(N, 0, -1):
        lam = lam + objective_grad(ws[n], P) / N
        nun = nu(ws[n - 1]) if callable(nu) else nu
        lam, sb = adjoint_step(ws[n - 1], lam, P, s, nun)
        sbar += sb
    return lam, sbar


def tangent_run(ws, wd0, P: Params, s=None, sd=None):
    """Forward tangent of Jbar along (wd0, sd) over a stored trajectory."""
    N = len(ws) - 1
    wd = wd0
    Jd = 0.0
    for n in range(N):
        wd = tangent_step(ws[n], wd, P, s, sd)
        Jd += np.sum(objective_grad(ws[n + 1], P) * wd) / N
    return Jd


# ----------------------------------------------------------------------------------
# added adjoint viscosity, section "Energy analysis" (stabilised adjoint equation)
# ----------------------------------------------------------------------------------
def viscosity_apply(a, nu, P: Params):
    """L_nu a = sum_d [nu_f+ (a(c+e_d) - a(c)) - nu_f- (a(c) - a(c-e_d))] / dx_d^2 for
    every component, nu_f the two-cell mean: the discrete div(nu grad a_i) of the
    lambda sigma_1 delta_ki delta_jl term, times the component's factor in P.nu_split.
    On a bounded box the boundary faces (inflow, outflow, walls) carry no flux."""
    out = np.zeros_like(a)
    for d in range(3):
        nup = 0.5 * (nu + _sh3(nu, d, 1))
        num = 0.5 * (nu + _sh3(nu, d, -1))
        if (d == 0 and _x_bounded(P)) or (d == 1 and _y_walls(P)):
            # no flux through the boundary faces (zero normal derivative)
            ax = 2 - d
            nup = np.moveaxis(nup.copy(), ax, -1)
            num = np.moveaxis(num.copy(), ax, -1)
            nup[..., -1] = 0.0
            num[..., 0] = 0.0
            nup = np.moveaxis(nup, -1, ax)
            num = np.moveaxis(num, -1, ax)
        out += (nup * (_sh3(a, d, 1) - a) - num * (a - _sh3(a, d, -1))) / P.dx[d] ** 2
    f_rho, f_mom, f_en = P.nu_split
    out[0] *= f_rho
    out[1:4] *= f_mom
    out[4] *= f_en
    return out


# ----------------------------------------------------------------------------------
# symmetrisation, growth matrix M and sigma_1 (section "Symmetrization" and
# "Energy analysis")
# ----------------------------------------------------------------------------------
def symmetrizer_S(rho, c, g):
    """S with delta v = S delta q, q = (rho, u1, u2, u3, p) (section "Symmetrization")."""
    S = np.zeros(rho.shape + (5, 5))
    S[..., 0, 0] = c / (math.sqrt(g) * rho)
    S[..., 1, 1] = S[..., 2, 2] = S[..., 3, 3] = 1.0
    S[..., 4, 0] = -c / (rho * math.sqrt(g * (g - 1.0)))
    S[..., 4, 4] = math.sqrt(g / (g - 1.0)) / (rho * c)
    return S


def primitive_jacobian_V(rho, u, g):
    """V with delta q = V delta w (section "Symmetrization"); rows 1..3 carry -u_k/rho
    in column 0, the derivative of u_k = m_k / rho."""
    V = np.zeros(rho.shape + (5, 5))
    V[..., 0, 0] = 1.0
    for k in range(3):
        V[..., 1 + k, 0] = -u[k] / rho
        V[..., 1 + k, 1 + k] = 1.0 / rho
        V[..., 4, 1 + k] = -(g - 1.0) * u[k]
    V[..., 4, 0] = 0.5 * (g - 1.0) * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    V[..., 4, 4] = g - 1.0
    return V


def symmetric_flux_matrix(u_j, c, j, g):
    """A_hat_{:j:} of section "Symmetrization": u_j I plus b = c/sqrt(g) coupling
    (v0, v_j) and a = sqrt((g-1)/g) c coupling (v_j, v4)."""
    b = c / math.sqrt(g)
    a = math.sqrt((g - 1.0) / g) * c
    A = np.zeros(np.shape(u_j) + (5, 5))
    for i in range(5):
        A[..., i, i] = u_j
    A[..., 0, 1 + j] = A[..., 1 + j, 0] = b
    A[..., 1 + j, 4] = A[..., 4, 1 + j] = a
    return A


def growth_matrix_generic(q, dq, g):
    """M = M1 - M2 from its definitions (section "Energy analysis"):
    M1_ki = 1/2 sum_{j,l} dAhat_kji/dq_l dq_l/dx_j and
    M2_ki = sum_{j,l,m} dAhat_kjl/dq_m S^-1_mi dv_l/dx_j with dv = S dq.
    q: (5, ...) primitive state, dq: (5, 3, ...) its gradient (dq[l, j] = dq_l/dx_j).
    dAhat/dq is taken by the exact chain rule through c = sqrt(g p / rho)."""
    rho, u, p = q[0], q[1:4], q[4]
    c = np.sqrt(g * p / rho)
    shp = rho.shape
    # dc/dq
    dc = np.zeros((5,) + shp)
    dc[0] = -c / (2.0 * rho)
    dc[4] = c / (2.0 * p)
    sb = 1.0 / math.sqrt(g)
    sa = math.sqrt((g - 1.0) / g)
    # dA[j, m] = dAhat_{:j:}/dq_m, shape (3, 5, ..., 5, 5)
    dA = np.zeros((3, 5) + shp + (5, 5))
    for j in range(3):
        for m in range(5):
            if m == 1 + j:
                for i in range(5):
                    dA[j, m, ..., i, i] = 1.0
            dA[j, m, ..., 0, 1 + j] += sb * dc[m]
            dA[j, m, ..., 1 + j, 0] += sb * dc[m]
            dA[j, m, ..., 1 + j, 4] += sa * dc[m]
            dA[j, m, ..., 4, 1 + j] += sa * dc[m]
    S = symmetrizer_S(rho, c, g)
    Sinv = np.linalg.inv(S)
    M1 = np.zeros(shp + (5, 5))
    for j in range(3):
        for m in range(5):
            M1 += 0.5 * dA[j, m] * dq[m, j][..., None, None]
    # dv_l/dx_j = S_lm dq_m/dx_j
    dv = np.einsum("...lm,mj...->lj...", S, dq)
    M2 = np.zeros(shp + (5, 5))
    for j in range(3):
        for m in range(5):
            # T_{k,l} = dAhat_kjl/dq_m ; contribution sum_l T_kl dv_l/dx_j * Sinv_mi
            Tv = np.einsum("...kl,l...->...k", dA[j, m], dv[:, j])
            M2 += Tv[..., :, None] * Sinv[..., m, None, :]
    return M1 - M2


def growth_matrix_closed(q, dq, db, da, g):
    """M = M1 - M2 from the closed forms printed in section "Energy analysis" with
    b = c/sqrt(g), a = sqrt((g-1)/g) c; db, da: (3, ...) gradients of b and a."""
    rho, p = q[0], q[4]
    c = np.sqrt(g * p / rho)
    b = c / math.sqrt(g)
    a = math.sqrt((g - 1.0) / g) * c
    div = dq[1, 0] + dq[2, 1] + dq[3, 2]
    shp = rho.shape
    M1 = np.zeros(shp + (5, 5))
    for i in range(5):
        M1[..., i, i] = 0.5 * div
    for j in range(3):
        M1[..., 0, 1 + j] = M1[..., 1 + j, 0] = 0.5 * db[j]
        M1[..., 1 + j, 4] = M1[..., 4, 1 + j] = 0.5 * da[j]
    M2 = np.zeros(shp + (5, 5))
    for j in range(3):
        M2[..., 0, 1 + j] = b / rho * dq[0, j]
        for k in range(3):
            M2[..., 1 + k, 1 + j] = dq[1 + k, j]
        M2[..., 4, 1 + j] = 2.0 / (g - 1.0) * da[j]
        M2[..., 1 + j, 4] = a / (2.0 * p) * dq[4, j]
    M2[..., 0, 4] = math.sqrt(g - 1.0) / 2.0 * div
    M2[..., 4, 4] = (g - 1.0) / 2.0 * div
    return M1 - M2


def _central(f, d, P):
    return (_sh3(f, d, 1) - _sh3(f, d, -1)) / (2.0 * P.dx[d])


def growth_matrix_field(w, P: Params):
    """Per-cell growth matrix M from central-difference gradients of rho, u_i, p, a, b
    (closed form, section "Energy analysis").  Shape (nz, ny, nx, 5, 5).  On a bounded
    box the differences at the boundary cells use the ghost states."""
    if P.bc != "periodic":
        return growth_matrix_field(pad(w, P), _periodic(P))[_crop_cells(P)]
    g = P.gamma
    rho, u, e, p = primitives(w, P)
    c = np.sqrt(g * p / rho)
    b = c / math.sqrt(g)
    a = math.sqrt((g - 1.0) / g) * c
    q = np.stack([rho, u[0], u[1], u[2], p])
    dq = np.stack([np.stack([_central(q[l], j, P) for j in range(3)]) for l in range(5)])
    db = np.stack([_central(b, j, P) for j in range(3)])
    da = np.stack([_central(a, j, P) for j in range(3)])
    return growth_matrix_closed(q, dq, db, da, g)


def sigma1_field(w, P: Params):
    """sigma_1, the largest singular value of M per cell (section "Energy analysis").
    For a 2D box (nz = 1) the (rho, u1, u2, p) block of M is used."""
    M = growth_matrix_field(w, P)
    if w.shape[1] == 1:
        idx = [0, 1, 2, 4]
        M = M[..., idx, :][..., :, idx]
    return np.linalg.svd(M, compute_uv=False)[..., 0]


def transform_T(w, P: Params):
    """T = S V per cell: delta v = T delta w (section "Symmetrization")."""
    g = P.gamma
    rho, u, e, p = primitives(w, P)
    c = np.sqrt(g * p / rho)
    return symmetrizer_S(rho, c, g) @ primitive_jacobian_V(rho, u, g)


def symmetric_adjoint(w, lam, P: Params):
    """v_hat with w_hat = T^T v_hat per cell (section "Symmetrization", boundedness)."""
    T = transform_T(w, P)
    lamc = np.moveaxis(lam, 0, -1)[..., None]
    vh = np.linalg.solve(np.swapaxes(T, -1, -2), lamc)[..., 0]
    return np.moveaxis(vh, -1, 0)


def adjoint_energy(w, lam, P: Params):
    """E_vhat = int v_hat . v_hat dV (section "Energy analysis", as a sum of squares)."""
    vh = symmetric_adjoint(w, lam, P)
    return float(np.sum(vh * vh) * P.dx[0] * P.dx[1] * P.dx[2])


def dot(a, b):
    """FP64 inner product over every element."""
    return float(np.sum(a * b))


def max_wave_speed(w, P: Params):
    """max over cells of |u| + c."""
    rho, u, e, p = primitives(w, P)
    c = np.sqrt(P.gamma * p / rho)
    return float(np.max(np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2) + c))


# ----------------------------------------------------------------------------------
# choice of the viscosity scaling factor (Conclusion: estimating the factor for a given
# problem is the method's first open question; results section, the table of adjoint
# and finite-difference sensitivities against the factor: too little viscosity leaves
# the adjoint growing, too much biases it, and in between the sensitivity hardly moves)
# ----------------------------------------------------------------------------------
def energy_efolds(E):
    """Growth of the adjoint energy over the second half of the backward sweep beyond
    what the objective source alone accounts for, in e-folds.  E[m] = E_vhat(w^m, lam^m)
    for m = 0..N (the sweep runs from m = N down to 0).  lam^m sums the sources of steps
    m..N, N - m + 1 bounded terms, pushed back by the adjoint propagator; when that
    propagator does not expand the energy norm (what the added viscosity is to ensure,
    section "Energy analysis") sqrt(E^m) grows at most linearly in N - m + 1, so the
    normalised energy E^m / (N - m + 1)^2 stays bounded and only exponential growth
    makes it rise.  With M = N // 2 the result is -M times the least-squares slope of
    ln(E[m] / (N - m + 1)^2) against m over m = 0..M: the fitted rise across the window
    as the adjoint runs backward from step M to step 0.  A non-positive or non-finite
    energy in the window gives +inf.  (A reading: the paper asks the energy to stay
    bounded without a test.)"""
    E = np.asarray(E, dtype=np.float64)
    N = E.shape[0] - 1
    M = N // 2
    if M < 1:
        raise ValueError("the window needs N >= 2")
    win = E[: M + 1]
    if not np.all(np.isfinite(win)) or np.any(win <= 0.0):
        return math.inf
    m = np.arange(M + 1, dtype=np.float64)
    y = np.log(win / (N - m + 1.0) ** 2)
    mc = m - m.mean()
    slope = float(np.sum(mc * (y - y.mean())) / np.sum(mc * mc))
    return -M * slope


def sensitivity_change(g_a, g_b):
    """Relative L2 change ||g_b - g_a|| / ||g_b|| of a sensitivity from one factor to the
    next larger one (over every element); 0 when both norms are 0, +inf when only
    ||g_b|| is."""
    g_a = np.asarray(g_a, dtype=np.float64)
    g_b = np.asarray(g_b, dtype=np.float64)
    d = math.sqrt(float(np.sum((g_b - g_a) ** 2)))
    nb = math.sqrt(float(np.sum(g_b * g_b)))
    if nb == 0.0:
        return 0.0 if d == 0.0 else math.inf
    return d / nb


def select_lambda(efolds, change, efold_tol, rel_tol):
    """Index of the smallest candidate factor i (candidates ascending, i < n - 1) whose
    adjoint energy does not grow by more than efold_tol e-folds over the window and
    whose sensitivity changes by at most rel_tol to the next candidate's; -1 if none.
    (A reading of the table and the conclusion: the smallest factor that damps the
    adjoint and sits on the plateau of the sensitivity.)"""
    for i in range(len(change)):
        if efolds[i] <= efold_tol and change[i] <= rel_tol:
            return i
    return -1


def estimate_lambda(w0, P: Params, nsteps, lambdas, s=None, tau=0.0, efold_tol=1.0, rel_tol=0.1):
    """Run the stabilised adjoint of an nsteps trajectory once per candidate factor
    (nu = lambda sigma_1(w^n) [sigma_1 > tau] for the step from w^n, none for lambda = 0)
    and apply select_lambda to the energy growth of each run and the relative change of
    the source sensitivity dJbar/ds between consecutive runs.  Returns (chosen index,
    efolds per candidate, change per consecutive pair, sbar per candidate, energy
    series E[m], m = 0..N, per candidate)."""
    ws, _ = primal_run(w0, P, nsteps, s)
    N = nsteps
    efolds, sbars, energies = [], [], []
    for lam_coef in lambdas:
        def nu_of(w, lam_coef=lam_coef):
            sig = sigma1_field(w, P)
            return lam_coef * sig * (sig > tau)
        # lam^N carries the objective source of step N; each reversed step n -> n - 1
        # then adds the source of step n - 1 (none for w^0), as in adjoint_run
        lam = objective_grad(ws[N], P) / N
        sbar = np.zeros_like(w0)
        E = np.zeros(N + 1)
        E[N] = adjoint_energy(ws[N], lam, P)
        for n in range(N, 0, -1):
            nun = nu_of(ws[n - 1]) if lam_coef > 0 else None
            lam, sb = adjoint_step(ws[n - 1], lam, P, s, nun)
            sbar += sb
            if n - 1 >= 1:
                lam = lam + objective_grad(ws[n - 1], P) / N
            E[n - 1] = adjoint_energy(ws[n - 1], lam, P)
        efolds.append(energy_efolds(E))
        sbars.append(sbar)
        energies.append(E)
    change = [sensitivity_change(sbars[i], sbars[i + 1]) for i in range(len(lambdas) - 1)]
    return select_lambda(efolds, change, efold_tol, rel_tol), efolds, change, sbars, energies
