"""Pins of the oracle's bounded boxes: characteristic inflow and outflow (section "Numerical
methods": non-reflecting inlet and outlet; section "Energy analysis": the incoming
characteristics are set there) and isothermal no-slip walls (section "Problem setup": the
vane surface is isothermal).  No GPU."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth

G = 1.4


def _params(nx, ny, nz, mu=0.01, dt=2e-3, flux="central", far=(1.0, 0.5, 0.0, 0.0, 1.0 / G)):
    return O.Params(gamma=G, mu=mu, dx=synth.box_shape(nx, ny, nz), dt=dt, bc="inout", far=far,
                    plane_i=(3 * nx) // 4, pt_in=1.0, flux=flux)


def _prim(w):
    rho = w[0]
    u = w[1:4] / rho
    p = (G - 1.0) * (w[4] - 0.5 * rho * np.sum(u * u, axis=0))
    return rho, u, p


def _invariants(w):
    rho, u, p = _prim(w)
    c = np.sqrt(G * p / rho)
    k = 2.0 / (G - 1.0)
    return u[0] + k * c, u[0] - k * c, p / rho ** G, u[1], u[2]


def test_uniform_far_field_stream_is_steady():
    """A stream equal to the far-field state makes every ghost equal to its neighbour,
    so the residual vanishes."""
    nx, ny, nz = 9, 4, 3
    rho = np.ones((nz, ny, nx))
    u = np.stack([0.5 * rho, 0.1 * rho, -0.2 * rho])
    w = synth._conservative(rho, u, rho / G, G)
    P = _params(nx, ny, nz, far=(1.0, 0.5, 0.1, -0.2, 1.0 / G))
    assert np.abs(O.residual(w, P)).max() <= 1e-14


def test_boundary_states_carry_the_right_invariants():
    """Outflow: R+, the entropy and the tangential velocity of the adjacent cell, R- of
    the far field.  Inflow: R- of the adjacent cell, R+, the entropy and the tangential
    velocity of the far field."""
    rng = np.random.default_rng(3)
    n = 50
    rho = 0.8 + 0.4 * rng.random(n)
    u = np.stack([0.2 + 0.4 * rng.random(n), 0.3 * rng.standard_normal(n), 0.3 * rng.standard_normal(n)])
    p = 0.5 + 0.4 * rng.random(n)
    wc = synth._conservative(rho, u, p, G)
    far = (1.1, 0.45, 0.05, -0.1, 0.75)
    P = _params(4, 4, 1, far=far)
    wf = synth._conservative(np.array([far[0]]), np.array(far[1:4])[:, None], np.array([far[4]]), G)
    I_c, I_f = _invariants(wc), _invariants(wf)
    out = _invariants(O.characteristic_state(wc, P, "out"))
    inn = _invariants(O.characteristic_state(wc, P, "in"))
    for got, want in zip(out, (I_c[0], I_f[1], I_c[2], I_c[3], I_c[4])):
        np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=1e-12, atol=1e-14)
    for got, want in zip(inn, (I_f[0], I_c[1], I_f[2], I_f[3], I_f[4])):
        np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("flux", ["central", "roe"])
def test_tangent_and_transpose_equal_fd_jacobian(flux):
    """Dense Jacobian of the bounded residual by central differences: the tangent and
    the transpose (periodic hand-derived operators on the padded box, ghosts pulled back
    through their complex-step Jacobians) reproduce J v and J^T a."""
    nx, ny, nz = 5, 4, 2
    w = synth.perturbed_uniform(nx, ny, nz, seed=11, amp=0.08)
    P = _params(nx, ny, nz, mu=0.05, flux=flux)
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
    scale = np.max(np.abs(J)) * 10
    np.testing.assert_allclose(O.residual_tangent(w, v, P).ravel(), J @ v.ravel(), atol=2e-7 * scale, rtol=0)
    np.testing.assert_allclose(O.residual_transpose(w, a, P).ravel(), J.T @ a.ravel(), atol=2e-7 * scale, rtol=0)
    # the boundary columns really differ from the periodic operator
    Pp = dataclasses.replace(P, bc="periodic")
    assert np.abs(O.residual_transpose(w, a, Pp) - O.residual_transpose(w, a, P)).max() > 1e-3 * scale / 10


def test_dot_product_identity_and_trajectory_gradient():
    """<a, J v> = <J^T a, v> to roundoff, and the adjoint of a bounded, sourced trajectory
    against central finite differences of Jbar (eps = 1e-6) along a random initial-state
    direction and a forcing shape."""
    nx, ny, nz = 12, 6, 1
    w0 = synth.isentropic_vortex(nx, ny, nz, noise=1e-3, seed=5)
    P = _params(nx, ny, nz, mu=0.01, dt=4e-3)
    v = synth.random_field(w0.shape, 3)
    a = synth.random_field(w0.shape, 4)
    lhs = O.dot(a, O.residual_tangent(w0, v, P))
    rhs = O.dot(O.residual_transpose(w0, a, P), v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(nx, ny, nz, n=4)[1]
    N = 6
    ws, _ = O.primal_run(w0, P, N, s)
    lam0, sbar = O.adjoint_run(ws, P, s)
    eps = 1e-6
    dw = synth.random_field(w0.shape, 12)
    fd = (O.primal_run(w0 + eps * dw, P, N, s)[1] - O.primal_run(w0 - eps * dw, P, N, s)[1]) / (2 * eps)
    assert abs(fd - O.dot(lam0, dw)) <= 1e-6 * abs(fd)
    ds = np.zeros_like(w0)
    ds[1] = synth.forcing_bumps(nx, ny, nz, n=4)[2]
    fd = (O.primal_run(w0, P, N, s + eps * ds)[1] - O.primal_run(w0, P, N, s - eps * ds)[1]) / (2 * eps)
    assert abs(fd - O.dot(sbar, ds)) <= 1e-6 * abs(fd)


def _pulse_energy_left(char_state):
    """Energy of the perturbation still in the box after a right-running acoustic pulse
    has crossed the outflow, relative to the pulse's initial energy (inviscid).  The
    pulse spans about 13 cells (sigma = 0.1 L_x on 128 cells): what the central scheme's
    dispersion leaves behind (a slow grid-scale tail) stays below 0.2% of the energy."""
    nx, ny, nz = 128, 2, 1
    rho0, u0, p0 = 1.0, 0.3, 1.0 / G
    c0 = math.sqrt(G * p0 / rho0)
    x = (np.arange(nx) + 0.5) / nx
    dp = 1e-3 * np.exp(-((x - 0.5) / 0.1) ** 2)
    shape = (nz, ny, nx)
    rho = rho0 + np.broadcast_to(dp / c0 ** 2, shape)
    u = np.stack([u0 + np.broadcast_to(dp / (rho0 * c0), shape), np.zeros(shape), np.zeros(shape)])
    p = p0 + np.broadcast_to(dp, shape)
    w = synth._conservative(np.array(rho), u, np.array(p), G)
    P = _params(nx, ny, nz, mu=0.0, dt=0.5 / nx / (u0 + c0), far=(rho0, u0, 0.0, 0.0, p0))
    e0 = float(np.sum(dp ** 2))
    steps = int(0.8 / P.dt)
    orig = O.characteristic_state
    try:
        O.characteristic_state = char_state
        for _ in range(steps):
            w, _ = O.rk4_step(w, P)
    finally:
        O.characteristic_state = orig
    _, _, pn = _prim(w)
    return float(np.sum((pn[0, 0] - p0) ** 2)) / e0


def test_outflow_lets_an_acoustic_pulse_leave():
    """The pulse crosses the characteristic outflow: more than 99.5% of its energy
    leaves the box.  A ghost held at the far-field state (a fixed-state boundary) keeps
    more than half of it in."""
    charac = _pulse_energy_left(O.characteristic_state)
    fixed = _pulse_energy_left(lambda wc, P, side: np.broadcast_to(
        synth._conservative(np.array([P.far[0]]), np.array(P.far[1:4])[:, None], np.array([P.far[4]]), G)
        .reshape((5,) + (1,) * (wc.ndim - 1)), wc.shape).copy())
    assert charac < 5e-3
    assert fixed > 0.5


def test_adjoint_viscosity_with_closed_inflow_and_outflow_faces():
    """The nu-Laplacian with no flux through the inflow and outflow faces stays symmetric
    and non-positive: <a, L b> = <L a, b> and <a, L a> <= 0."""
    nx, ny, nz = 7, 5, 3
    P = _params(nx, ny, nz)
    rng = np.random.default_rng(2)
    nu = 0.1 + rng.random((nz, ny, nx))
    a = rng.standard_normal((5, nz, ny, nx))
    b = rng.standard_normal((5, nz, ny, nx))
    La, Lb = O.viscosity_apply(a, nu, P), O.viscosity_apply(b, nu, P)
    assert abs(O.dot(a, Lb) - O.dot(La, b)) <= 1e-12 * abs(O.dot(a, Lb))
    assert O.dot(a, La) < 0.0
    # a field constant along x feels no boundary: only the y and z differences act
    c = np.broadcast_to(rng.standard_normal((5, nz, ny, 1)), a.shape).copy()
    Pp = dataclasses.replace(P, bc="periodic")
    np.testing.assert_allclose(O.viscosity_apply(c, np.ones_like(nu), P),
                               O.viscosity_apply(c, np.ones_like(nu), Pp), rtol=1e-13, atol=1e-13)


def test_sigma1_sees_the_ghosts():
    """sigma_1 of a uniform far-field stream is zero in every cell with the boundaries
    too; on a flow that differs from the far field the boundary columns' sigma_1 is
    taken with the ghost states (it differs from the periodic value) and the interior
    columns' is not."""
    nx, ny, nz = 8, 5, 3
    rho = np.ones((nz, ny, nx))
    w = synth._conservative(rho, np.stack([0.5 * rho, 0 * rho, 0 * rho]), rho / G, G)
    P = _params(nx, ny, nz)
    assert np.all(O.sigma1_field(w, P) == 0.0)
    w = synth.perturbed_uniform(nx, ny, nz, seed=5, amp=0.05)
    s_b = O.sigma1_field(w, P)
    s_p = O.sigma1_field(w, dataclasses.replace(P, bc="periodic"))
    np.testing.assert_allclose(s_b[..., 1:-1], s_p[..., 1:-1], rtol=1e-13)
    assert np.abs(s_b[..., [0, -1]] - s_p[..., [0, -1]]).max() > 1e-6


# ---- isothermal no-slip walls at y = 0 and y = L_y ------------------------------------
def _wall_params(nx, ny, nz, bc="walls", mu=0.02, e_w=(1.0 / 0.56, 1.0 / 0.56), **kw):
    return O.Params(gamma=G, mu=mu, dx=synth.box_shape(nx, ny, nz), dt=2e-3, bc=bc, wall_e=e_w,
                    far=kw.get("far", (1.0, 0.0, 0.0, 0.0, 1.0 / G)), plane_i=(3 * nx) // 4, pt_in=1.0)


@pytest.mark.parametrize("bc", ["walls", "inout_walls"])
def test_rest_at_the_wall_temperature_is_steady(bc):
    nx, ny, nz = 7, 6, 3
    rho = np.full((nz, ny, nx), 1.0)
    w = synth._conservative(rho, np.zeros((3,) + rho.shape), rho / G, G)
    P = _wall_params(nx, ny, nz, bc=bc, e_w=(1.0 / 0.56, 1.0 / 0.56))
    assert np.abs(O.residual(w, P)).max() <= 1e-13


def test_walls_pass_no_mass():
    """x and z periodic, walls in y: the mass residual sums to zero for any state."""
    nx, ny, nz = 6, 5, 4
    w = synth.perturbed_uniform(nx, ny, nz, seed=8, amp=0.1)
    P = _wall_params(nx, ny, nz, e_w=(1.5, 2.1))
    R = O.residual(w, P)
    assert abs(R[0].sum()) <= 1e-13 * np.abs(R[0]).sum()
    assert abs(R[4].sum()) > 1e-3 * np.abs(R[4]).sum()    # the walls exchange heat


def test_wall_heat_flux_and_pressure_closed_forms():
    """Rest, uniform rho and e with e != e_w: the wall face's heat flux is
    alpha (e - e_w) / (dy/2), so the wall row's energy residual is
    2 alpha (e_w - e) / dy^2; its y-momentum residual is the jump to the wall face's
    pressure, -(gamma-1) rho (e - e_w) / dy (bottom wall, outward normal -y)."""
    nx, ny, nz = 4, 6, 1
    rho0, e0, ew = 1.1, 1.8, 2.3
    rho = np.full((nz, ny, nx), rho0)
    w = synth._conservative(rho, np.zeros((3,) + rho.shape), (G - 1) * rho * e0, G)
    P = _wall_params(nx, ny, nz, e_w=(ew, e0))
    dy = P.dx[1]
    R = O.residual(w, P)
    np.testing.assert_allclose(R[4][:, 0], 2 * P.alpha * (ew - e0) / dy ** 2, rtol=1e-12)
    np.testing.assert_allclose(R[2][:, 0], -(G - 1) * rho0 * (e0 - ew) / dy, rtol=1e-12)
    np.testing.assert_allclose(R[:, :, 1:], 0.0, atol=1e-12)    # top wall at e0, interior at rest


def test_wall_drag_on_a_uniform_stream():
    """A uniform stream u1 = U at the wall temperature: the no-slip wall's shear stress
    mu (U - (-U)) / dy drags the wall rows, R_u1 = -2 mu U / dy^2 on both; the walls
    do no work (the face velocity is zero) and pass no heat."""
    nx, ny, nz = 5, 4, 2
    U = 0.3
    rho = np.ones((nz, ny, nx))
    u = np.stack([U * rho, 0 * rho, 0 * rho])
    w = synth._conservative(rho, u, rho / G, G)
    P = _wall_params(nx, ny, nz, e_w=(1.0 / 0.56, 1.0 / 0.56))
    dy = P.dx[1]
    R = O.residual(w, P)
    for row in (0, -1):
        np.testing.assert_allclose(R[1][:, row], -2 * P.mu * U / dy ** 2, rtol=1e-12)
        np.testing.assert_allclose(R[4][:, row], 0.0, atol=1e-12)
    np.testing.assert_allclose(R[:, :, 1:-1], 0.0, atol=1e-12)
    np.testing.assert_allclose(R[0], 0.0, atol=1e-12)


@pytest.mark.parametrize("bc,flux", [("walls", "central"), ("inout_walls", "central"), ("inout_walls", "roe")])
def test_wall_tangent_and_transpose_equal_fd_jacobian(bc, flux):
    nx, ny, nz = 4, 4, 2
    w = synth.perturbed_uniform(nx, ny, nz, seed=13, amp=0.08)
    P = _wall_params(nx, ny, nz, bc=bc, mu=0.05, e_w=(1.6, 2.0), far=(1.0, 0.5, 0.0, 0.0, 1.0 / G))
    P.flux = flux
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
    scale = np.max(np.abs(J)) * 10
    np.testing.assert_allclose(O.residual_tangent(w, v, P).ravel(), J @ v.ravel(), atol=2e-7 * scale, rtol=0)
    np.testing.assert_allclose(O.residual_transpose(w, a, P).ravel(), J.T @ a.ravel(), atol=2e-7 * scale, rtol=0)


def test_channel_trajectory_gradient():
    """Inflow, outflow and walls together: the adjoint of a sourced trajectory against
    central finite differences of Jbar (eps = 1e-6)."""
    nx, ny, nz = 12, 6, 1
    w0 = synth.isentropic_vortex(nx, ny, nz, noise=1e-3, seed=6)
    P = _wall_params(nx, ny, nz, bc="inout_walls", mu=0.01, e_w=(1.7, 1.9),
                     far=(1.0, 0.5, 0.0, 0.0, 1.0 / G))
    P.dt = 4e-3
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(nx, ny, nz, n=4)[1]
    N = 5
    ws, _ = O.primal_run(w0, P, N, s)
    lam0, sbar = O.adjoint_run(ws, P, s)
    eps = 1e-6
    dw = synth.random_field(w0.shape, 14)
    fd = (O.primal_run(w0 + eps * dw, P, N, s)[1] - O.primal_run(w0 - eps * dw, P, N, s)[1]) / (2 * eps)
    assert abs(fd - O.dot(lam0, dw)) <= 1e-6 * abs(fd)
    ds = np.zeros_like(w0)
    ds[1] = synth.forcing_bumps(nx, ny, nz, n=4)[3]
    fd = (O.primal_run(w0, P, N, s + eps * ds)[1] - O.primal_run(w0, P, N, s - eps * ds)[1]) / (2 * eps)
    assert abs(fd - O.dot(sbar, ds)) <= 1e-6 * abs(fd)


def test_adjoint_viscosity_with_closed_walls():
    nx, ny, nz = 6, 7, 3
    P = _wall_params(nx, ny, nz, bc="inout_walls")
    rng = np.random.default_rng(4)
    nu = 0.1 + rng.random((nz, ny, nx))
    a = rng.standard_normal((5, nz, ny, nx))
    b = rng.standard_normal((5, nz, ny, nx))
    La, Lb = O.viscosity_apply(a, nu, P), O.viscosity_apply(b, nu, P)
    assert abs(O.dot(a, Lb) - O.dot(La, b)) <= 1e-12 * abs(O.dot(a, Lb))
    assert O.dot(a, La) < 0.0
    # a field that varies only along z feels neither walls nor inflow and outflow
    c = np.broadcast_to(rng.standard_normal((5, nz, 1, 1)), a.shape).copy()
    np.testing.assert_allclose(O.viscosity_apply(c, np.ones_like(nu), P),
                               O.viscosity_apply(c, np.ones_like(nu), dataclasses.replace(P, bc="periodic")),
                               rtol=1e-13, atol=1e-13)
