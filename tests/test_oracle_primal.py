"""Pins of the oracle's primal residual, RK4 step and objective against what the
mathematics fixes (no GPU).  Each test is chosen so that a plausible slip in the
oracle (a dropped term, a sign, a transposed index) fails one of them."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth


def params_for(w, mu=0.01, dt=1e-3, gamma=1.4, Pr=0.72, mach=0.5):
    nz, ny, nx = w.shape[1:]
    pt_in = (1.0 / gamma) * (1.0 + 0.5 * (gamma - 1.0) * mach ** 2) ** (gamma / (gamma - 1.0))
    return O.Params(gamma=gamma, mu=mu, Pr=Pr, dx=synth.box_shape(nx, ny, nz), dt=dt,
                    plane_i=(3 * nx) // 4, pt_in=pt_in)


def uniform(nx, ny, nz, mach=0.7, gamma=1.4):
    rho = np.full((nz, ny, nx), 1.3)
    u = np.stack([np.full_like(rho, mach), np.full_like(rho, -0.2), np.full_like(rho, 0.1)])
    p = np.full_like(rho, 0.9 / gamma)
    return synth._conservative(rho, u, p, gamma)


def test_uniform_flow_residual_is_exactly_zero():
    """A uniform state is a steady solution: every face flux is identical, so R = 0
    bitwise (Eq. e:vector)."""
    for shp in [(6, 5, 4), (8, 8, 1)]:
        w = uniform(*shp)
        P = params_for(w, mu=0.05)
        R = O.residual(w, P)
        assert np.all(R == 0.0)


def test_primitive_and_euler_flux_closed_forms():
    """p = (gamma-1)(rho E - rho |u|^2/2) and the Euler flux columns (Eq. e:vector),
    checked on one cell against values worked out by hand."""
    g = 1.4
    rho, u, p = 2.0, np.array([0.3, -0.4, 0.5]), 1.5
    rhoE = p / (g - 1) + 0.5 * rho * np.dot(u, u)
    w = np.array([rho, rho * u[0], rho * u[1], rho * u[2], rhoE]).reshape(5, 1, 1, 1)
    P = O.Params(gamma=g)
    r, uu, e, pp = O.primitives(w, P)
    assert abs(pp.item() - p) < 1e-14
    assert abs(e.item() - p / ((g - 1) * rho)) < 1e-14
    for d in range(3):
        F = O.euler_flux(w, d, P)[:, 0, 0, 0]
        ref = np.array([rho * u[d], rho * u[d] * u[0], rho * u[d] * u[1], rho * u[d] * u[2],
                        (rhoE + p) * u[d]])
        ref[1 + d] += p
        np.testing.assert_allclose(F, ref, rtol=1e-15, atol=1e-15)


def test_viscous_flux_of_linear_shear_and_heat():
    """For a linear velocity u1 = s y (a periodic-compatible interior check) the face
    stress is mu s on x-faces' (1,2) entry; for a linear internal energy the heat flux
    is alpha de/dx.  Checked away from the periodic seam."""
    nx, ny, nz = 8, 16, 1
    g, mu, Pr = 1.4, 0.3, 0.72
    dx = (0.1, 0.1, 0.1)
    y = (np.arange(ny) + 0.5) * dx[1]
    x = (np.arange(nx) + 0.5) * dx[0]
    Y, X = np.meshgrid(y, x, indexing="ij")
    s, q = 0.7, 0.2
    rho = np.ones((nz, ny, nx))
    u = np.stack([s * Y[None], np.zeros_like(rho), np.zeros_like(rho)])
    e = 2.0 + q * X[None]
    p = (g - 1) * rho * e
    w = synth._conservative(rho, u, p, g)
    P = O.Params(gamma=g, mu=mu, Pr=Pr, dx=dx)
    Fv_x = O.viscous_face_flux(w, 0, P)      # x-faces between i and i+1
    Fv_y = O.viscous_face_flux(w, 1, P)      # y-faces between j and j+1
    sl = (0, slice(2, ny - 2), slice(1, nx - 2))
    # x-face: sigma_12 = mu du1/dy = mu s ; heat flux alpha de/dx = alpha q
    np.testing.assert_allclose(Fv_x[2][sl], mu * s, rtol=1e-12)
    np.testing.assert_allclose(Fv_x[1][sl], 0.0, atol=1e-12)
    uf = u[0][sl]
    np.testing.assert_allclose(Fv_x[4][sl], P.alpha * q + 0.0 * uf, rtol=1e-12)
    # y-face: sigma_21 = mu s, sigma_22 = 0, energy = u_f1 sigma_21
    np.testing.assert_allclose(Fv_y[1][sl], mu * s, rtol=1e-12)
    uf1 = 0.5 * (u[0] + np.roll(u[0], -1, axis=1))[sl]
    np.testing.assert_allclose(Fv_y[4][sl], uf1 * mu * s, rtol=1e-12)


@pytest.mark.parametrize("shape", [(7, 5, 3), (12, 9, 1), (5, 4, 6)])
def test_periodic_conservation(shape):
    """sum_cells R = 0 for mass, momentum and energy (flux-difference form on a periodic
    box telescopes), and the RK4 step conserves sum w to roundoff."""
    w = synth.perturbed_uniform(*shape, seed=3, amp=0.05)
    P = params_for(w, mu=0.02, dt=2e-3)
    R = O.residual(w, P)
    scale = np.max(np.abs(R), axis=(1, 2, 3))
    tot = np.sum(R, axis=(1, 2, 3))
    n = np.prod(shape)
    assert np.all(np.abs(tot) <= 1e-13 * n * np.maximum(scale, 1e-300))
    w1 = w
    for _ in range(5):
        w1, _ = O.rk4_step(w1, P)
    np.testing.assert_allclose(np.sum(w1, axis=(1, 2, 3)), np.sum(w, axis=(1, 2, 3)),
                               rtol=1e-13, atol=1e-13)


def test_galilean_shift_of_inviscid_flux():
    """Inviscid, the residual of a state that is a pure x-translation by one cell is the
    translated residual (the discrete operator commutes with periodic shifts)."""
    w = synth.perturbed_uniform(6, 5, 4, seed=5)
    P = params_for(w, mu=0.01)
    R = O.residual(w, P)
    Rs = O.residual(np.roll(w, 1, axis=3), P)
    np.testing.assert_allclose(Rs, np.roll(R, 1, axis=3), rtol=1e-13, atol=1e-13)


def _vortex_error(n, t_frac):
    mach = 0.5
    w0 = synth.isentropic_vortex(n, n, 1, mach=mach, noise=0.0)
    P = params_for(w0, mu=0.0, mach=mach)
    P.dt = 0.25 / n
    steps = int(round(t_frac / (mach * P.dt)))
    P.dt = t_frac / (mach * steps)
    w = w0
    for _ in range(steps):
        w, _ = O.rk4_step(w, P)
    wex = synth.isentropic_vortex(n, n, 1, mach=mach, noise=0.0, shift=t_frac)
    return math.sqrt(np.mean((w[0] - wex[0]) ** 2))


def test_inviscid_vortex_second_order_convergence():
    """Inviscid, the isentropic vortex is an exact solution that translates at the mean
    flow; the discrete error after a fixed time must fall at second order."""
    errs = [_vortex_error(n, 0.05) for n in (32, 64, 128)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 1.7 < rates[0] < 2.4 and 1.8 < rates[1] < 2.3, (errs, rates)


def test_stagnation_pressure_closed_forms():
    """p_t = p at rest; p_t/p = (1 + (g-1)/2)^(g/(g-1)) at Mach 1 (Eq. e:pressure_loss)."""
    g = 1.4
    P = O.Params(gamma=g)
    rho, p = np.array(1.7), np.array(0.8)
    zero = np.zeros(3)
    rhoE = p / (g - 1)
    assert abs(O.stagnation_pressure(rho, zero, rhoE, P) - p) < 1e-15
    c = math.sqrt(g * p / rho)
    m = np.array([rho * c, 0.0, 0.0])
    rhoE = p / (g - 1) + 0.5 * rho * c * c
    ratio = O.stagnation_pressure(rho, m, rhoE, P) / p
    assert abs(ratio - 1.2 ** 3.5) < 1e-13


def test_objective_uniform_and_gradient_by_fd():
    """J = 0 for the uniform free stream that defines p_t,in; dJ/dw (hand derived) agrees
    with central differences; dJ/dw is zero off the two plane columns."""
    g, mach = 1.4, 0.5
    shp = (8, 6, 3)
    rho = np.ones(shp[::-1])
    u = np.stack([np.full_like(rho, mach), 0 * rho, 0 * rho])
    w_u = synth._conservative(rho, u, np.full_like(rho, 1 / g), g)
    P = params_for(w_u, mach=mach)
    assert abs(O.objective(w_u, P)) < 1e-15
    w = synth.perturbed_uniform(*shp, seed=7, amp=0.08, mach=mach)
    G = O.objective_grad(w, P)
    cols = [(P.plane_i - 1) % shp[0], P.plane_i % shp[0]]
    off = np.delete(G, cols, axis=3)
    assert np.all(off == 0.0)
    rng = np.random.default_rng(0)
    for _ in range(6):
        idx = (rng.integers(5), rng.integers(shp[2]), rng.integers(shp[1]), rng.choice(cols))
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (O.objective(wp, P) - O.objective(wm, P)) / (2 * h)
        assert abs(fd - G[idx]) <= 1e-8 * max(abs(fd), 1e-6), (idx, fd, G[idx])


def test_viscous_flux_of_linear_compression_stokes_hypothesis():
    """u1 = s x (a uniform compression, div u = s): with zero bulk viscosity the normal
    stresses are 2 mu s - 2/3 mu s = 4/3 mu s along x and -2/3 mu s along y and z, and
    there is no shear stress (Eq. e:navier).  Checked away from the periodic seam."""
    nx, ny, nz = 12, 6, 5
    g, mu, Pr = 1.4, 0.3, 0.72
    dx = (0.1, 0.2, 0.15)
    x = (np.arange(nx) + 0.5) * dx[0]
    s = 0.4
    rho = np.ones((nz, ny, nx))
    u = np.stack([np.broadcast_to(s * x, rho.shape), np.zeros_like(rho), np.zeros_like(rho)])
    w = synth._conservative(rho, u, np.full_like(rho, 0.7), g)
    P = O.Params(gamma=g, mu=mu, Pr=Pr, dx=dx)
    interior = (slice(None), slice(None), slice(1, nx - 2))
    Fx, Fy, Fz = (O.viscous_face_flux(w, d, P) for d in range(3))
    np.testing.assert_allclose(Fx[1][interior], 4.0 / 3.0 * mu * s, rtol=1e-12)
    np.testing.assert_allclose(Fy[2][interior], -2.0 / 3.0 * mu * s, rtol=1e-12)
    np.testing.assert_allclose(Fz[3][interior], -2.0 / 3.0 * mu * s, rtol=1e-12)
    for F, d in ((Fx, 0), (Fy, 1), (Fz, 2)):
        for j in range(3):
            if j != d:
                np.testing.assert_allclose(F[1 + j][interior], 0.0, atol=1e-13)


def test_heat_flux_through_the_temperature():
    """The heat flux written as k dT/dx with k = mu c_p / Pr and T = e / c_v (any gas
    constant R: c_v = R / (gamma - 1), c_p = gamma c_v) for a linear internal energy at
    rest: the energy component of the x-face flux."""
    nx, ny, nz = 10, 4, 1
    g, mu, Pr, R = 1.4, 0.3, 0.72, 287.0
    dx = (0.1, 0.1, 0.1)
    x = (np.arange(nx) + 0.5) * dx[0]
    q = 0.25
    rho = np.full((nz, ny, nx), 1.3)
    e = np.broadcast_to(2.0 + q * x, rho.shape)
    w = synth._conservative(rho, np.zeros((3,) + rho.shape), (g - 1) * rho * e, g)
    P = O.Params(gamma=g, mu=mu, Pr=Pr, dx=dx)
    cv = R / (g - 1.0)
    cp = g * cv
    dTdx = q / cv
    Fx = O.viscous_face_flux(w, 0, P)
    np.testing.assert_allclose(Fx[4][..., 1:nx - 2], mu * cp / Pr * dTdx, rtol=1e-12)


def test_objective_closed_form_on_a_two_state_plane():
    """One plane face at rest (p_t = p) and one at Mach 1 (p_t = p (1.2)^3.5 for
    gamma = 1.4): J = [rho_a (p_t,in - p_a) + rho_b (p_t,in - 1.2^3.5 p_b)] / (rho_a +
    rho_b) / p_t,in, the density-weighted loss of Eq. (e:pressure_loss)."""
    g = 1.4
    nx, ny, nz = 8, 2, 1
    ra, pa, rb, pb = 1.0, 0.9, 2.0, 0.5
    rho = np.empty((nz, ny, nx))
    rho[:, 0], rho[:, 1] = ra, rb
    p = np.empty_like(rho)
    p[:, 0], p[:, 1] = pa, pb
    cb = math.sqrt(g * pb / rb)
    u = np.zeros((3,) + rho.shape)
    u[0][:, 1] = cb
    w = synth._conservative(rho, u, p, g)
    pt_in = 1.3
    P = O.Params(gamma=g, dx=synth.box_shape(nx, ny, nz), plane_i=6, pt_in=pt_in)
    expect = (ra * (pt_in - pa) + rb * (pt_in - 1.2 ** 3.5 * pb)) / (ra + rb) / pt_in
    assert O.objective(w, P) == pytest.approx(expect, rel=1e-13)
