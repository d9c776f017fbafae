"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and evaluates input shapes (plane waves,
Gaussian envelopes) at the staggered positions of each field component.  It
contains none of the method's arithmetic (no stencil, no dispersion
relation): both the CUDA path and the oracle receive what it produces.
"""
from __future__ import annotations

import math

import numpy as np

# staggered offsets (x, y, z) of E_x, E_y, E_z, B_x, B_y, B_z in cell units (App. A)
OFFSETS = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5),
           (0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]


def positions(shape_xyz, comp, dx):
    """Coordinates (x, y, z) arrays of shape (nz, ny, nx) for field component `comp`."""
    nx, ny, nz = shape_xyz
    o = OFFSETS[comp]
    z, y, x = np.meshgrid((np.arange(nz) + o[2]) * dx[2], (np.arange(ny) + o[1]) * dx[1],
                          (np.arange(nx) + o[0]) * dx[0], indexing="ij")
    return x, y, z


def random_fields(shape_xyz, seed, scale=1.0):
    """Six independent standard-normal fields (nz, ny, nx), float64."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape_xyz
    return [scale * rng.standard_normal((nz, ny, nx)) for _ in range(6)]


def random_theta(seed, dims=3):
    """Coefficient draw: delta_i ~ U[-1/8, 0], beta_ij ~ U[-1/8, 1/8] (absent axes zero).

    The caller decides whether a draw is admissible (Eq. constraints)."""
    rng = np.random.default_rng(seed)
    beta = rng.uniform(-0.125, 0.125, (3, 3))
    delta = rng.uniform(-0.125, 0.0, 3)
    for i in range(3):
        beta[i, i] = 0.0
    for ax in range(dims, 3):
        beta[:, ax] = 0.0
        beta[ax, :] = 0.0
        delta[ax] = 0.0
    return beta, delta


def isotropic_theta(d_axial, d_perp, b_axial, b_perp):
    """Tied 3D coefficient set theta = (delta_x, delta_perp, beta_x, beta_perp):
    delta = (dx, dp, dp); beta_xy = beta_yx = beta_xz = beta_zx = b_axial; beta_yz = beta_zy = b_perp."""
    beta = np.array([[0.0, b_axial, b_axial], [b_axial, 0.0, b_perp], [b_axial, b_perp, 0.0]])
    delta = np.array([d_axial, d_perp, d_perp])
    return beta, delta


def plane_wave(shape_xyz, kvec, pol, dx, amplitude=1.0):
    """E = pol * cos(k . r) at each E component's own position; B = 0."""
    E = []
    for c in range(3):
        x, y, z = positions(shape_xyz, c, dx)
        E.append(amplitude * pol[c] * np.cos(kvec[0] * x + kvec[1] * y + kvec[2] * z))
    nx, ny, nz = shape_xyz
    zero = np.zeros((nz, ny, nx))
    return E + [zero, zero.copy(), zero.copy()]


def packet_x(shape_xyz, dx, x_center, sigma, wavelength, omega0, dt):
    """Plane packet moving along +x, uniform in y and z: E_z = g(x - xc) cos(k0 (x - xc)) at
    t = 0 and B_y = -g(x - xc + v dt/2) cos(k0 (x - xc) + omega0 dt/2) at t = -dt/2 (the
    leapfrog's B time), g a Gaussian of width sigma, k0 = 2 pi / wavelength and v = omega0 / k0.
    omega0 is the caller's angular frequency for k0 (it only sets the initial phase of B)."""
    nx, ny, nz = shape_xyz
    k0 = 2 * math.pi / wavelength
    v = omega0 / k0
    zero = np.zeros((nz, ny, nx))
    x, _, _ = positions(shape_xyz, 2, dx)
    Ez = np.exp(-((x - x_center) ** 2) / (2 * sigma ** 2)) * np.cos(k0 * (x - x_center))
    xb, _, _ = positions(shape_xyz, 4, dx)
    u = xb - x_center + 0.5 * v * dt
    By = -np.exp(-(u ** 2) / (2 * sigma ** 2)) * np.cos(k0 * (xb - x_center) + 0.5 * omega0 * dt)
    return [zero, zero.copy(), Ez, zero.copy(), By, zero.copy()]


def gaussian_pulse_2d(shape_xy, dx, center, waist, wavelength, seed=0, noise=1e-3):
    """2D TE pulse: stream function psi = exp(-r^2/waist^2) cos(2 pi x / wavelength) (+ seeded
    noise) sampled at the B_z positions; returned as psi (ny, nx).  Fields are derived from psi
    by the caller."""
    nx, ny = shape_xy
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid((np.arange(ny) + 0.5) * dx[1], (np.arange(nx) + 0.5) * dx[0], indexing="ij")
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    psi = np.exp(-r2 / waist ** 2) * np.cos(2 * math.pi * x / wavelength)
    return psi + noise * rng.standard_normal(psi.shape)


def pulse_ez_3d(shape_xyz, dx, x_center, sigma_x, waist, wavelength):
    """E_z pulse travelling along x: exp(-(x-xc)^2/(2 sigma_x^2)) exp(-r_perp^2/waist^2) cos(k x)."""
    nx, ny, nz = shape_xyz
    x, y, z = positions(shape_xyz, 2, dx)
    yc, zc = 0.5 * ny * dx[1], 0.5 * nz * dx[2]
    env = np.exp(-((x - x_center) ** 2) / (2 * sigma_x ** 2)) * \
        np.exp(-((y - yc) ** 2 + (z - zc) ** 2) / waist ** 2)
    return env * np.cos(2 * math.pi * x / wavelength)


def te_pulse(shape_xy, dx, center, waist, wavelength, dt, seed=0, noise=1e-3):
    """2D TE (E_x, E_y, B_z) Gaussian pulse moving along +x, plus seeded noise.

    E_y = exp(-|r - c|^2 / waist^2) cos(2 pi (x - c_x) / wavelength) at the E_y positions,
    B_z = the same profile evaluated half a time step ahead at the B_z positions (t = -dt/2),
    E_x = 0.  Shapes (1, ny, nx)."""
    nx, ny = shape_xy
    rng = np.random.default_rng(seed)

    def prof(x, y):
        return np.exp(-((x - center[0]) ** 2 + (y - center[1]) ** 2) / waist ** 2) * \
            np.cos(2 * math.pi * (x - center[0]) / wavelength)

    x, y, _ = positions((nx, ny, 1), 1, dx)
    Ey = prof(x, y) + noise * rng.standard_normal(x.shape)
    x, y, _ = positions((nx, ny, 1), 5, dx)
    Bz = prof(x + 0.5 * dt, y) + noise * rng.standard_normal(x.shape)
    zero = np.zeros((1, ny, nx))
    return [zero, Ey, zero.copy(), zero.copy(), zero.copy(), Bz]


def vacuum_probe_target(Ez0, dx, dt, nsteps, x_index):
    """Probe-plane target for the differentiable run: E_z(x_index, y, z, s dt), s = 1..nsteps, of
    the exact continuum (c = 1) vacuum solution that starts from E = (0, 0, Ez0), B = 0 on the
    periodic box.  Per Fourier mode the transverse part oscillates as cos(|k| t) and the
    longitudinal part stays; evaluated with FP64 FFTs.  Returns an array [nsteps, nz, ny]."""
    nz, ny, nx = Ez0.shape
    kx = 2 * math.pi * np.fft.fftfreq(nx, d=dx[0])
    ky = 2 * math.pi * np.fft.fftfreq(ny, d=dx[1])
    kz = 2 * math.pi * np.fft.fftfreq(nz, d=dx[2])
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    kn = np.sqrt(k2)
    with np.errstate(invalid="ignore", divide="ignore"):
        long_frac = np.where(k2 > 0, KZ ** 2 / k2, 1.0)   # z-component of the longitudinal projector
    F = np.fft.fftn(Ez0)
    # E_z at x = x_index for all (y, z): sum over k_x with the phase of the probe plane
    phase_x = np.exp(1j * kx * x_index * dx[0]) / nx
    out = np.empty((nsteps, nz, ny))
    A = F * (1.0 - long_frac)      # transverse part
    Bl = F * long_frac             # static longitudinal part
    static = np.tensordot(Bl, phase_x, axes=([2], [0]))
    for s in range(1, nsteps + 1):
        t = s * dt
        dyn = np.tensordot(A * np.cos(kn * t), phase_x, axes=([2], [0]))   # [nz, ny] in (kz, ky)
        plane = np.fft.ifft2(dyn + static, axes=(0, 1)) * 1.0
        out[s - 1] = plane.real
    return out


def angled_te_packet(nx, ny, angle, wavelength, sigma_u, sigma_v, center, dx=(1.0, 1.0)):
    """2D TE packet travelling at `angle` (radians from +x), continuum divergence-free:
    E = curl(psi z) = (d_y psi, -d_x psi) with psi = exp(-u^2/su^2 - v^2/sv^2) sin(k0 u)/k0,
    u, v the coordinates along / across the direction of travel, evaluated analytically at the
    E_x (i+1/2, j) and E_y (i, j+1/2) positions.  Returns (Ex, Ey), each [ny, nx]."""
    k0 = 2 * math.pi / wavelength
    ca, sa = math.cos(angle), math.sin(angle)

    def grads(x, y):
        u = (x - center[0]) * ca + (y - center[1]) * sa
        v = -(x - center[0]) * sa + (y - center[1]) * ca
        env = np.exp(-(u / sigma_u) ** 2 - (v / sigma_v) ** 2)
        psi_u = env * (np.cos(k0 * u) - 2 * u / sigma_u ** 2 * np.sin(k0 * u) / k0)
        psi_v = env * (-2 * v / sigma_v ** 2) * np.sin(k0 * u) / k0
        return psi_u * ca - psi_v * sa, psi_u * sa + psi_v * ca   # d/dx, d/dy

    y, x = np.meshgrid(np.arange(ny) * dx[1], (np.arange(nx) + 0.5) * dx[0], indexing="ij")
    _, dpsi_dy = grads(x, y)
    y, x = np.meshgrid((np.arange(ny) + 0.5) * dx[1], np.arange(nx) * dx[0], indexing="ij")
    dpsi_dx, _ = grads(x, y)
    return dpsi_dy, -dpsi_dx


def vacuum_target_2d(F0, dx, dt, nsteps, x_index):
    """One component of a continuum divergence-free 2D field under vacuum propagation
    (c = 1, initial B = 0): every Fourier mode oscillates as cos(|k| t).  Returns the values on
    the plane x = x_index for t = s dt, s = 1..nsteps: array [nsteps, ny]."""
    ny, nx = F0.shape
    kx = 2 * math.pi * np.fft.fftfreq(nx, d=dx[0])
    ky = 2 * math.pi * np.fft.fftfreq(ny, d=dx[1])
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kn = np.sqrt(KX ** 2 + KY ** 2)
    F = np.fft.fft2(F0)
    phase_x = np.exp(1j * kx * x_index * dx[0]) / nx
    out = np.empty((nsteps, ny))
    for s in range(1, nsteps + 1):
        col = (F * np.cos(kn * s * dt)) @ phase_x     # [ny] in k_y
        out[s - 1] = np.fft.ifft(col).real
    return out


def particles(shape_xyz, dx, n, seed, u_scale=1.0):
    """n macro-particles: positions uniform over the periodic box, momenta u = gamma v with
    standard-normal components times u_scale.  Arrays (3, n), float64."""
    rng = np.random.default_rng(seed)
    L = np.array([shape_xyz[a] * dx[a] for a in range(3)])[:, None]
    x = rng.uniform(0.0, 1.0, (3, n)) * L
    u = u_scale * rng.standard_normal((3, n))
    return x, u


def uniform_plasma(shape_xyz, dx, ppc, seed, u_th):
    """ppc particles in every cell, ordered cell by cell (x fastest), each uniformly placed
    inside its cell; thermal momenta u_th * N(0, 1) per component.  Arrays (3, n), float64."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape_xyz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64)
    base = np.repeat(cells, ppc, axis=1)
    x = (base + rng.uniform(0.0, 1.0, base.shape)) * np.asarray(dx, dtype=np.float64)[:, None]
    u = u_th * rng.standard_normal(base.shape)
    return x, u


def gaussian_bunch(n, center, sigma, direction, gamma, seed, dx=(1.0, 1.0, 1.0)):
    """n macro-particles of a relativistic bunch: positions Gaussian about `center` with
    widths sigma = (sigma_parallel, sigma_perp) (in cells, parallel = along `direction`),
    all with momentum u = sqrt(gamma^2 - 1) along the unit vector `direction`.  The draw is
    ordered by z cell, then y cell, then x position, so that neighbouring particles share
    cells, and still do after the bunch has drifted along x.  Arrays (3, n), float64,
    positions in the units of dx."""
    rng = np.random.default_rng(seed)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    # an orthonormal pair perpendicular to d
    a = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(d, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    s_par, s_perp = sigma
    r = rng.standard_normal((3, n))
    cells = (np.asarray(center, dtype=np.float64)[:, None] + s_par * r[0] * d[:, None]
             + s_perp * r[1] * e1[:, None] + s_perp * r[2] * e2[:, None])
    order = np.lexsort((cells[0], np.floor(cells[1]), np.floor(cells[2])))
    x = cells[:, order] * np.asarray(dx, dtype=np.float64)[:, None]
    u = np.repeat((math.sqrt(gamma * gamma - 1.0) * d)[:, None], n, axis=1)
    return x, u
