"""Seeded synthetic inputs shaped like the paper's transonic vane LES.

This module only builds input fields; it holds none of the solver's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  All fields are numpy
float64 in the conservative layout w[5, nz, ny, nx] (x fastest), w = (rho, rho u1,
rho u2, rho u3, rho E), in units where the free stream has rho = 1, p = 1/gamma
(so the sound speed is 1) and velocity = Mach number, and the box length along x
is 1.

Recipes (the paper's vane geometry and flow data are not available; these stand in
for them with the same flow character: Mach near 1, vortical structures, periodic
span):
  * isentropic_vortex: the Shu-Yee vortex of strength beta on a uniform flow at a
    given Mach number along x, radius unit R = L/10, centred in the box, written in
    Shu units (rho = p = T = 1 at infinity) and rescaled exactly to the units above
    (p -> p/gamma, u -> u/sqrt(gamma)); plus seeded Gaussian noise, relative in rho
    and absolute (times the Mach number) in each velocity component.
  * solenoidal_turbulence: uniform rho and p, mean flow along x plus a random-phase
    divergence-free velocity field with Fourier shells 2 <= |k| <= 16 (|k| counted in
    units of 2 pi / L_y), energy spectrum E(k) ~ k^(-5/3), scaled so that the rms of
    each fluctuating component is `rms` times the mean speed.
  * forcing_bumps: Gaussian source shapes acting on the x-momentum equation at
    x = 0.25 L_x, on a regular grid in (y, z) (or along y for a 2D box).
"""
from __future__ import annotations

import math

import numpy as np


def _conservative(rho, u, p, gamma):
    """(rho, u, p) -> w, the ideal-gas total energy rho E = p/(gamma-1) + rho |u|^2 / 2."""
    w = np.empty((5,) + rho.shape)
    w[0] = rho
    w[1:4] = rho * u
    w[4] = p / (gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return w


def box_shape(nx, ny, nz):
    """Cell sizes of a box of length 1 along x with cubic cells."""
    d = 1.0 / nx
    return (d, d, d)


def _centres(nx, ny, nz):
    d = 1.0 / nx
    x = (np.arange(nx) + 0.5) * d
    y = (np.arange(ny) + 0.5) * d
    z = (np.arange(nz) + 0.5) * d
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z, (nx * d, ny * d, nz * d)


def isentropic_vortex(nx, ny, nz=1, mach=0.5, beta=5.0, noise=1e-3, seed=1, gamma=1.4,
                      shift=0.0):
    """Shu-Yee isentropic vortex on a uniform flow (2D for nz = 1, a z-aligned column
    otherwise), with seeded noise.  `shift` moves the centre along x (in units of the
    box length) from the box centre.  Returns w[5, nz, ny, nx]."""
    X, Y, Z, (Lx, Ly, Lz) = _centres(nx, ny, nz)
    R = Lx / 10.0
    xc, yc = (0.5 + shift) * Lx, 0.5 * Ly
    # periodic nearest-image offsets
    dxv = (X - xc + 0.5 * Lx) % Lx - 0.5 * Lx
    dyv = (Y - yc + 0.5 * Ly) % Ly - 0.5 * Ly
    r2 = (dxv ** 2 + dyv ** 2) / R ** 2
    f = np.exp(0.5 * (1.0 - r2))
    # Shu units: rho = p = T = 1 at infinity, sound speed sqrt(gamma)
    du = -beta / (2.0 * math.pi) * (dyv / R) * f
    dv = beta / (2.0 * math.pi) * (dxv / R) * f
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * f ** 2
    rho = T ** (1.0 / (gamma - 1.0))
    p_shu = rho * T
    # rescale to free-stream sound speed 1
    u = np.stack([mach + du / math.sqrt(gamma), dv / math.sqrt(gamma), np.zeros_like(rho)])
    p = p_shu / gamma
    if noise > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        rho = rho * (1.0 + noise * rng.standard_normal(rho.shape))
        u = u + noise * mach * rng.standard_normal(u.shape)
        if nz == 1:
            u[2] = 0.0
    return _conservative(rho, u, p, gamma)


def solenoidal_turbulence(nx, ny, nz, mach=0.9, rms=0.1, seed=2, kmin=2, kmax=16,
                          gamma=1.4):
    """Uniform rho = 1, p = 1/gamma; u = mach e_x + random-phase solenoidal field."""
    d = 1.0 / nx
    Lx, Ly, Lz = nx * d, ny * d, nz * d
    rng = np.random.Generator(np.random.PCG64(seed))
    kx = np.fft.fftfreq(nx, d=1.0 / nx) * (2.0 * math.pi / Lx)
    ky = np.fft.fftfreq(ny, d=1.0 / ny) * (2.0 * math.pi / Ly)
    kz = np.fft.fftfreq(nz, d=1.0 / nz) * (2.0 * math.pi / Lz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kn = K * Ly / (2.0 * math.pi)          # shell index in units of 2 pi / L_y
    shell = (kn >= kmin) & (kn <= kmax)
    # an even axis's Nyquist plane has no mirror mode, so its real part would not stay
    # perpendicular to k: leave it empty (it lies outside the shells on the benchmark boxes)
    for axis, n in ((0, nz), (1, ny), (2, nx)):
        if n % 2 == 0:
            nyq = np.zeros(K.shape, dtype=bool)
            idx = [slice(None)] * 3
            idx[axis] = n // 2
            nyq[tuple(idx)] = True
            shell &= ~nyq
    amp = np.zeros_like(K)
    # 3D: |u_hat(k)|^2 ~ E(k) / k^2 with E ~ k^(-5/3)
    amp[shell] = kn[shell] ** (-11.0 / 6.0)
    uh = (rng.standard_normal((3,) + K.shape) + 1j * rng.standard_normal((3,) + K.shape))
    uh *= amp
    # project onto the plane normal to k (divergence free)
    Ks = np.where(K > 0, K, 1.0)
    kv = np.stack([KX, KY, KZ]) / Ks
    kdotu = np.sum(kv * uh, axis=0)
    uh -= kv * kdotu
    up = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    up -= up.mean(axis=(1, 2, 3), keepdims=True)
    cur = math.sqrt(float(np.mean(up ** 2)))
    if cur > 0.0:
        up *= rms * mach / cur
    rho = np.ones((nz, ny, nx))
    u = up.copy()
    u[0] += mach
    p = np.full((nz, ny, nx), 1.0 / gamma)
    return _conservative(rho, u, p, gamma)


def forcing_bumps(nx, ny, nz, n=64, width_cells=3.0):
    """Source shapes phi_m[n, nz, ny, nx] (x-momentum equation only): Gaussian bumps of
    width `width_cells` cells centred at x = 0.25 L_x on a sqrt(n) x sqrt(n) grid in
    (y, z) for a 3D box, or n points along y for a 2D box (nz = 1)."""
    X, Y, Z, (Lx, Ly, Lz) = _centres(nx, ny, nz)
    d = 1.0 / nx
    wdt = width_cells * d
    x0 = 0.25 * Lx

    def pdist(a, c, L):
        return (a - c + 0.5 * L) % L - 0.5 * L

    if nz == 1:
        centres = [(x0, (m + 0.5) * Ly / n, 0.5 * Lz) for m in range(n)]
    else:
        s = int(round(math.sqrt(n)))
        centres = [(x0, (i + 0.5) * Ly / s, (j + 0.5) * Lz / s)
                   for j in range(s) for i in range(s)]
    phi = np.empty((len(centres), nz, ny, nx))
    for m, (cx, cy, cz) in enumerate(centres):
        r2 = pdist(X, cx, Lx) ** 2 + pdist(Y, cy, Ly) ** 2
        if nz > 1:
            r2 = r2 + pdist(Z, cz, Lz) ** 2
        phi[m] = np.exp(-0.5 * r2 / wdt ** 2)
    return phi


def random_field(shape, seed, scale=1.0):
    """Seeded standard-normal field, for dot-product and parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)


def perturbed_uniform(nx, ny, nz, seed, amp=0.05, mach=0.5, gamma=1.4):
    """A smooth-ish random state near a uniform flow: every primitive gets a seeded
    relative perturbation of size amp (for operator tests on tiny grids)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = (nz, ny, nx)
    rho = 1.0 + amp * rng.standard_normal(shp)
    u = np.stack([mach + amp * rng.standard_normal(shp),
                  amp * rng.standard_normal(shp),
                  (amp * rng.standard_normal(shp)) if nz > 1 else np.zeros(shp)])
    p = (1.0 / gamma) * (1.0 + amp * rng.standard_normal(shp))
    return _conservative(rho, u, p, gamma)


def kolmogorov_amplitude(U0, mu, Ly, k=1):
    """Forcing amplitude that sustains the laminar profile u_1 = U0 sin(2 pi k y / L_y)
    against viscosity (mu (2 pi k / L_y)^2 U0; density 1)."""
    return U0 * mu * (2.0 * math.pi * k / Ly) ** 2


def kolmogorov_forcing(nx, ny, nz, amp, k=1):
    """A time-constant body force on the x-momentum equation, s_1 = amp sin(2 pi k y / L_y)
    (the other components zero): a Kolmogorov shear forcing that keeps a periodic box
    turbulent instead of decaying.  Its y-mean is zero, so it adds no net momentum."""
    X, Y, Z, (Lx, Ly, Lz) = _centres(nx, ny, nz)
    s = np.zeros((5, nz, ny, nx))
    s[1] = amp * np.sin(2.0 * math.pi * k * Y / Ly)
    return s


def forced_start(nx, ny, nz, mach=0.3, shear=0.0, k=1, noise=0.02, seed=5, gamma=1.4):
    """Initial state of a forced box: a stream of the given Mach number along x (rho = 1,
    p = 1/gamma, sound speed 1) carrying the shear profile shear sin(2 pi k y / L_y) that
    the Kolmogorov forcing sustains, with seeded noise of relative size noise (of the
    larger of mach and shear) on every velocity component, from which the shear layers'
    instability grows."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = (nz, ny, nx)
    X, Y, Z, (Lx, Ly, Lz) = _centres(nx, ny, nz)
    rho = np.ones(shp)
    a = noise * max(mach, shear)
    u = np.stack([mach + shear * np.sin(2.0 * math.pi * k * Y / Ly) + a * rng.standard_normal(shp),
                  a * rng.standard_normal(shp),
                  a * rng.standard_normal(shp) if nz > 1 else np.zeros(shp)])
    p = np.full(shp, 1.0 / gamma)
    return _conservative(rho, u, p, gamma)
