"""Macro-particles coupled to the extended-stencil field solver -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain numpy, vectorised over
particles; every grid access wraps periodically.

The paper keeps Yee's stencil in Ampere's law so that a charge-conserving current
weighting (Esirkepov 2001, named in App. A) makes the discrete continuity equation
D_t rho + D . J = 0 hold exactly (App. A, numerical continuity equation); Gauss's law
D . E = rho (Sec. 2, Eq. divE) then holds at every step if it holds at the start.  Its
particle runs (Sec. 6) use the EPOCH code.  The paper does not state the particle shape
or the pusher; the readings taken here are:

  shape     first order (cloud in cell): node i of axis a carries the weight
            S_i(x) = max(0, 1 - |x / dx_a - i|)
  rho       at the nodes (i, j, k):  sum_p q S_i(x_p) S_j(y_p) S_k(z_p) / (dx dy dz)
  gather    each field component interpolated with the same first-order shape from its
            own staggered positions (E_x at (i+1/2, j, k), B_x at (i, j+1/2, k+1/2), ...
            as in ``oracle.fdtd``); B at the integer time level is the mean of
            B^{n-1/2} and B^{n+1/2}
  push      Boris's relativistic scheme in u = gamma v (c = 1): half electric kick,
            rotation about B, half electric kick; x^{n+1} = x^n + dt u^{n+1/2} / gamma
  current   Esirkepov's decomposition of the change of the particle's shape
            S1 - S0 (old and new position) into W_x + W_y + W_z, with
                W_x = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3)
            and cyclically; then  J_x(i+1/2) - J_x(i-1/2) = -q W_x(i) / (dt dy dz),
            summed from the low end of the particle's 4-node window (J_x stored at the
            E_x index).  A particle moves less than one cell per step (|v| < c and
            c dt < dx on every stable grid), so a 4-node window per axis holds both
            supports.

One PIC cycle (``pic_step``):
  B^{n+1/2} = B^{n-1/2} - dt D* x E^n            (extended Faraday, as ``oracle.fdtd.step``)
  gather E^n and B^n = (B^{n-1/2} + B^{n+1/2}) / 2 at x^n
  u^{n-1/2} -> u^{n+1/2} (Boris),  x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}
  J^{n+1/2} from x^n -> x^{n+1} (Esirkepov)
  E^{n+1} = E^n + dt (D x B^{n+1/2} - J^{n+1/2})  (Yee Ampere)
Positions are wrapped into [0, L) after the current is formed.
"""
from __future__ import annotations

import numpy as np

from . import fdtd as F

# staggered offsets (in cells) of E_x, E_y, E_z and B_x, B_y, B_z (x, y, z order)
E_OFFSETS = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]
B_OFFSETS = [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]


class Particles:
    """One species: positions x[3, n] (physical units), u[3, n] = gamma v (c = 1),
    macro-particle charge q and charge-to-mass ratio qm."""

    def __init__(self, x, u, q, qm):
        self.x = np.array(x, dtype=np.float64).reshape(3, -1)
        self.u = np.array(u, dtype=np.float64).reshape(3, -1)
        self.q, self.qm = float(q), float(qm)

    def copy(self):
        return Particles(self.x.copy(), self.u.copy(), self.q, self.qm)


def gamma(u):
    return np.sqrt(1.0 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)


def _shape_pair(xs, off):
    """Node index f and the two first-order weights (f, f+1) at grid coordinate xs - off."""
    gcoord = xs - off
    f = np.floor(gcoord)
    w1 = gcoord - f
    return f.astype(np.int64), 1.0 - w1, w1


def gather(Fc, off, x, dx):
    """Field component Fc (indexed [k, j, i], staggered by ``off`` cells) at the particle
    positions x[3, n]: the first-order weights of the two nearest positions per axis."""
    nz, ny, nx = Fc.shape
    fi, wx0, wx1 = _shape_pair(x[0] / dx[0], off[0])
    fj, wy0, wy1 = _shape_pair(x[1] / dx[1], off[1])
    fk, wz0, wz1 = _shape_pair(x[2] / dx[2], off[2])
    out = np.zeros(x.shape[1])
    for a, wa in ((0, wx0), (1, wx1)):
        for b, wb in ((0, wy0), (1, wy1)):
            for c, wc in ((0, wz0), (1, wz1)):
                v = Fc[(fk + c) % nz, (fj + b) % ny, (fi + a) % nx]
                out += wa * wb * wc * v
    return out


def boris(u, E, B, qm, dt):
    """Boris's relativistic push of u^{n-1/2} to u^{n+1/2} in the fields E, B at x^n."""
    h = 0.5 * qm * dt
    um = u + h * E
    g = gamma(um)
    t = h * B / g
    s = 2.0 * t / (1.0 + t[0] ** 2 + t[1] ** 2 + t[2] ** 2)
    up = um + np.cross(um, t, axis=0)
    upl = um + np.cross(up, s, axis=0)
    return upl + h * E


def _window(xs):
    """Base node (floor(xs) - 1) of the 4-node window and the first-order weights of grid
    coordinate xs on it (shape (4, n))."""
    base = np.floor(xs).astype(np.int64) - 1
    m = np.arange(4)[:, None]
    w = np.maximum(0.0, 1.0 - np.abs(xs[None, :] - (base[None, :] + m)))
    return base, w


def deposit_rho(p: Particles, shape, dx):
    """Charge density at the nodes from the first-order shape, periodic."""
    nz, ny, nx = shape
    rho = np.zeros(shape)
    fi, wx0, wx1 = _shape_pair(p.x[0] / dx[0], 0.0)
    fj, wy0, wy1 = _shape_pair(p.x[1] / dx[1], 0.0)
    fk, wz0, wz1 = _shape_pair(p.x[2] / dx[2], 0.0)
    vol = dx[0] * dx[1] * dx[2]
    for a, wa in ((0, wx0), (1, wx1)):
        for b, wb in ((0, wy0), (1, wy1)):
            for c, wc in ((0, wz0), (1, wz1)):
                np.add.at(rho, ((fk + c) % nz, (fj + b) % ny, (fi + a) % nx),
                          p.q * wa * wb * wc / vol)
    return rho


def esirkepov(x0, x1, q, shape, dx, dt):
    """J^{n+1/2} (three arrays, J_a at the E_a positions) of charges q moving from x0 to x1
    (both [3, n], x1 not wrapped; |x1 - x0| < one cell per axis)."""
    nz, ny, nx = shape
    n = [nx, ny, nz]
    bases, S0, dS = [], [], []
    for a in range(3):
        g0 = x0[a] / dx[a]
        g1 = x1[a] / dx[a]
        base, w0 = _window(g0)
        m = np.arange(4)[:, None]
        w1 = np.maximum(0.0, 1.0 - np.abs(g1[None, :] - (base[None, :] + m)))
        bases.append(base)
        S0.append(w0)
        dS.append(w1 - w0)
    J = [np.zeros(shape) for _ in range(3)]
    idx = np.arange(4)
    for a in range(3):
        b, c = [(1, 2), (0, 2), (0, 1)][a]
        # W_a[p, ma, mb, mc] over the windows of axes a, b, c
        Wa = dS[a].T[:, :, None, None] * (
            S0[b].T[:, None, :, None] * S0[c].T[:, None, None, :]
            + 0.5 * dS[b].T[:, None, :, None] * S0[c].T[:, None, None, :]
            + 0.5 * S0[b].T[:, None, :, None] * dS[c].T[:, None, None, :]
            + (1.0 / 3.0) * dS[b].T[:, None, :, None] * dS[c].T[:, None, None, :])
        Ja = -(q / (dt * dx[b] * dx[c])) * np.cumsum(Wa, axis=1)
        # node index of each window entry, per axis, broadcast to Ja's shape
        ia = (bases[a][:, None] + idx[None, :]) % n[a]
        ib = (bases[b][:, None] + idx[None, :]) % n[b]
        ic = (bases[c][:, None] + idx[None, :]) % n[c]
        full = [None, None, None]
        full[a] = ia[:, :, None, None]
        full[b] = ib[:, None, :, None]
        full[c] = ic[:, None, None, :]
        full = np.broadcast_arrays(*full, Ja)
        np.add.at(J[a], (full[2].ravel(), full[1].ravel(), full[0].ravel()), full[3].ravel())
    return J


def wrap_positions(x, shape, dx):
    nz, ny, nx = shape
    L = np.array([nx * dx[0], ny * dx[1], nz * dx[2]])[:, None]
    return np.mod(x, L)


def push(p: Particles, E, Bn, dx, dt):
    """Gather E, Bn at x^n, Boris push; returns (u^{n+1/2}, unwrapped x^{n+1})."""
    Ep = np.stack([gather(E[a], E_OFFSETS[a], p.x, dx) for a in range(3)])
    Bp = np.stack([gather(Bn[a], B_OFFSETS[a], p.x, dx) for a in range(3)])
    u1 = boris(p.u, Ep, Bp, p.qm, dt)
    x1 = p.x + dt * u1 / gamma(u1)
    return u1, x1


def pic_step(s: F.State, species, c: F.Coeffs, sponge=None):
    """One PIC cycle on state s (E^n, B^{n-1/2}) and the species list (x^n, u^{n-1/2}).
    ``sponge`` (the factor array of ``oracle.fdtd.sponge_factor``) multiplies B^{n+1/2}
    and E^{n+1} after their updates, as in ``oracle.fdtd.step``."""
    shape = s.E[0].shape
    f = F.faraday_rhs(s.E, c)
    B_half = [s.B[a] + c.dt * f[a] for a in range(3)]
    if sponge is not None:
        B_half = [b * sponge for b in B_half]
    Bn = [0.5 * (s.B[a] + B_half[a]) for a in range(3)]
    J = [np.zeros(shape) for _ in range(3)]
    for p in species:
        u1, x1 = push(p, s.E, Bn, c.dx, c.dt)
        Jp = esirkepov(p.x, x1, p.q, shape, c.dx, c.dt)
        for a in range(3):
            J[a] += Jp[a]
        p.u = u1
        p.x = wrap_positions(x1, shape, c.dx)
    s.B = B_half
    g = F.ampere_curl(s.B, c)
    s.E = [s.E[a] + c.dt * (g[a] - J[a]) for a in range(3)]
    if sponge is not None:
        s.E = [e * sponge for e in s.E]
    return s
