"""The seeded input generators that feed both the oracle and the CUDA path (they hold no
solver arithmetic): each recipe has the properties its reading states."""
import math

import numpy as np
import pytest

from paper_1511_06959_gb300 import synth


def _primitives(w, g):
    rho = w[0]
    u = w[1:4] / rho
    p = (g - 1.0) * (w[4] - 0.5 * rho * np.sum(u * u, axis=0))
    return rho, u, p


@pytest.mark.parametrize("nz", [1, 3])
def test_isentropic_vortex(nz):
    """Shu-Yee vortex (beta = 5, R = L_x / 10) rescaled to sound speed 1: isentropic
    (p / rho^gamma = 1/gamma everywhere), the free stream far away, the temperature dip
    1 - (gamma-1) beta^2 / (8 gamma pi^2) e at the centre (Shu units), and the swirl
    speed beta / (2 pi) / sqrt(gamma) at r = R, its maximum; a column in 3D."""
    g, beta, mach = 1.4, 5.0, 0.5
    n = 64
    w = synth.isentropic_vortex(n, n, nz, mach=mach, beta=beta, noise=0.0, gamma=g)
    rho, u, p = _primitives(w, g)
    np.testing.assert_allclose(p / rho ** g, 1.0 / g, rtol=1e-12)
    corner = (0, 0, 0)
    assert abs(rho[corner] - 1.0) < 1e-9 and abs(u[0][corner] - mach) < 1e-6
    # every cell against the closed form (no noise)
    X, Y, _, (Lx, Ly, _) = synth._centres(n, n, nz)
    R = Lx / 10.0
    r2 = ((X - 0.5 * Lx) ** 2 + (Y - 0.5 * Ly) ** 2) / R ** 2
    T_shu = 1.0 - (g - 1.0) * beta ** 2 / (8.0 * g * math.pi ** 2) * np.exp(1.0 - r2)
    np.testing.assert_allclose(g * p / rho, T_shu, rtol=1e-12)   # T_shu = gamma p / rho here
    swirl = np.sqrt((u[0] - mach) ** 2 + u[1] ** 2)
    expect = beta / (2 * math.pi) * np.sqrt(r2) * np.exp(0.5 * (1.0 - r2)) / math.sqrt(g)
    np.testing.assert_allclose(swirl, expect, atol=1e-12)
    assert swirl.max() <= beta / (2 * math.pi) / math.sqrt(g) + 1e-12
    assert np.all(u[2] == 0.0)
    # seeded noise: reproducible, and a different seed differs
    a = synth.isentropic_vortex(16, 12, nz, noise=1e-3, seed=7)
    b = synth.isentropic_vortex(16, 12, nz, noise=1e-3, seed=7)
    c = synth.isentropic_vortex(16, 12, nz, noise=1e-3, seed=8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_solenoidal_turbulence():
    """Uniform rho = 1 and p = 1/gamma, mean velocity (mach, 0, 0), fluctuations with rms
    mach x rms over the three components, spectrally divergence-free, and only in the
    shells 2 <= |k| L_y / (2 pi) <= 16."""
    g, mach, rms = 1.4, 0.9, 0.1
    nx, ny, nz = 32, 16, 16
    w = synth.solenoidal_turbulence(nx, ny, nz, mach=mach, rms=rms, seed=2, gamma=g)
    rho, u, p = _primitives(w, g)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=0)
    np.testing.assert_allclose(p, 1.0 / g, rtol=1e-12)
    up = u - np.array([mach, 0.0, 0.0])[:, None, None, None]
    np.testing.assert_allclose(up.mean(axis=(1, 2, 3)), 0.0, atol=1e-14)
    assert math.sqrt(float(np.mean(up ** 2))) == pytest.approx(rms * mach, rel=1e-12)
    d = 1.0 / nx
    L = (nx * d, ny * d, nz * d)
    kx = np.fft.fftfreq(nx, d=1.0 / nx) * 2 * math.pi / L[0]
    ky = np.fft.fftfreq(ny, d=1.0 / ny) * 2 * math.pi / L[1]
    kz = np.fft.fftfreq(nz, d=1.0 / nz) * 2 * math.pi / L[2]
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    uh = np.fft.fftn(up, axes=(1, 2, 3))
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    assert np.abs(div).max() <= 1e-10 * (K * np.abs(uh).sum(axis=0)).max()
    kn = K * L[1] / (2 * math.pi)
    energy = np.sum(np.abs(uh) ** 2, axis=0)
    outside = (kn < 2 - 1e-9) | (kn > 16 + 1e-9)
    assert energy[outside].max() <= 1e-20 * energy.max()


@pytest.mark.parametrize("nz", [1, 8])
def test_forcing_bumps(nz):
    """64 Gaussian bumps of width 3 cells with peak 1 at x = L_x / 4: along y in 2D, on
    an 8 x 8 grid in (y, z) in 3D; periodic distances."""
    nx, ny = 32, 64
    phi = synth.forcing_bumps(nx, ny, nz, n=64)
    assert phi.shape == (64, nz, ny, nx)
    assert phi.max() <= 1.0 and phi.min() > 0.0
    X, Y, Z, (Lx, Ly, Lz) = synth._centres(nx, ny, nz)
    # each bump peaks at the cell nearest its centre, on the column x = L_x / 4
    for m in (0, 17, 63):
        k, j, i = np.unravel_index(np.argmax(phi[m]), phi[m].shape)
        assert abs(X[k, j, i] - 0.25 * Lx) <= 0.5 / nx + 1e-12
    # the profile along x through a peak is a Gaussian of width 3 cells
    k, j, i = np.unravel_index(np.argmax(phi[5]), phi[5].shape)
    row = phi[5][k, j]
    w = 3.0 / nx
    ratio = row[(i + 3) % nx] / row[i]
    dx0 = X[k, j, i] - 0.25 * Lx
    assert ratio == pytest.approx(math.exp(-0.5 * ((dx0 + 3.0 / nx) ** 2 - dx0 ** 2) / w ** 2), rel=1e-12)
    # distinct centres: no two bumps coincide
    peaks = {np.unravel_index(np.argmax(phi[m]), phi[m].shape) for m in range(64)}
    assert len(peaks) == 64


def test_kolmogorov_forcing_and_forced_start():
    """The Kolmogorov force acts on x-momentum only, with zero mean over y; the forced
    start is the stream plus the laminar shear profile (rho = 1, p = 1/gamma) and seeded
    noise of the stated relative size."""
    nx, ny, nz = 8, 32, 4
    s = synth.kolmogorov_forcing(nx, ny, nz, amp=0.7)
    assert s.shape == (5, nz, ny, nx)
    assert np.all(s[[0, 2, 3, 4]] == 0.0)
    assert abs(s[1].mean()) < 1e-15 and abs(np.abs(s[1]).max() - 0.7) < 0.01
    g = 1.4
    w = synth.forced_start(nx, ny, nz, mach=0.3, shear=0.2, noise=0.0, gamma=g)
    rho, u, p = _primitives(w, g)
    np.testing.assert_allclose(rho, 1.0)
    np.testing.assert_allclose(p, 1.0 / g, rtol=1e-12)
    y = (np.arange(ny) + 0.5) / nx
    prof = 0.3 + 0.2 * np.sin(2.0 * math.pi * y / (ny / nx))
    np.testing.assert_allclose(u[0][0, :, 0], prof, rtol=1e-12)
    wn = synth.forced_start(nx, ny, nz, mach=0.3, shear=0.2, noise=0.02, seed=3, gamma=g)
    _, un, _ = _primitives(wn, g)
    assert abs(np.std(un[1]) / (0.02 * 0.3) - 1.0) < 0.1
    assert np.array_equal(wn, synth.forced_start(nx, ny, nz, mach=0.3, shear=0.2, noise=0.02, seed=3, gamma=g))


def test_kolmogorov_amplitude_balances_the_discrete_viscous_term():
    """On the laminar profile u_1 = U0 sin(k y) (k = 2 pi / L_y) the forcing of amplitude
    mu k^2 U0 cancels the oracle's viscous x-momentum residual up to the three-point
    Laplacian's error: R_1 + s_1 = mu U0 (k^2 - (4 / dy^2) sin^2(k dy / 2)) sin(k y),
    about (k dy)^2 / 12 of the amplitude (mass and the other momenta stay at rest)."""
    from oracle import ns_oracle as O
    from tests.test_oracle_primal import params_for
    nx, ny, nz = 4, 32, 2
    U0, mu = 0.2, 0.01
    w = synth.forced_start(nx, ny, nz, mach=0.3, shear=U0, noise=0.0)
    dx = synth.box_shape(nx, ny, nz)
    Ly = ny * dx[1]
    amp = synth.kolmogorov_amplitude(U0, mu, Ly)
    s = synth.kolmogorov_forcing(nx, ny, nz, amp)
    P = params_for(w, mu=mu, dt=1e-3)
    R = O.residual(w, P, s)
    k, dy = 2.0 * math.pi / Ly, dx[1]
    y = (np.arange(ny) + 0.5) * dy
    exact = mu * U0 * (k * k - 4.0 / dy ** 2 * math.sin(0.5 * k * dy) ** 2) * np.sin(k * y)
    np.testing.assert_allclose(R[1][0, :, 0], exact, rtol=1e-6, atol=1e-12 * amp)
    assert abs(np.abs(R[1]).max() / amp - (k * dy) ** 2 / 12.0) < 0.01 * (k * dy) ** 2 / 12.0
    assert np.abs(R[0]).max() < 1e-12 and np.abs(R[2:4]).max() < 1e-12
