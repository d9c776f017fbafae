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
