"""Leapfrog FDTD with the extended Faraday stencil, its adjoint, and diagnostics -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain numpy on periodic
grids; every neighbour access is an ``np.roll``.  Nothing here is blocked,
fused or reordered beyond the paper's update equations.

Layout and staggering (App. A, update equations)
-----------------------------------------------
Arrays are indexed ``[k, j, i]`` (z, y, x; x fastest) with shape (nz, ny, nx).
The integer index (i, j, k) of each component denotes the staggered position

    E_x (i+1/2, j, k)      B_x (i, j+1/2, k+1/2)
    E_y (i, j+1/2, k)      B_y (i+1/2, j, k+1/2)
    E_z (i, j, k+1/2)      B_z (i+1/2, j+1/2, k)

so every D*_a in Faraday's law is a forward difference along a (from E
positions to B positions) and every Yee D_a in Ampere's law is a backward
difference (from B positions to E positions).  Indices are periodic on all
axes.  Units c = mu0 = eps0 = 1, so c^2 dt = dt and mu0 J = J.

Grids with nz = 1 (or ny = nz = 1) are z-invariant (yz-invariant): every
difference along such an axis vanishes exactly, which reproduces the 2D (1D)
scheme provided the beta entries pointing along the missing axes are zero.

Optional absorbing sponge (a reading; the paper has none): after each half
update the fields in the outermost ``absorb_cells`` index layers along y and
z are multiplied by f(d) = 1 - sigma (d / L)^3, d = 1..L counted from the
inner edge of the layer.
"""
from __future__ import annotations

import math

import numpy as np

X, Y, Z = 0, 1, 2


def at(F, di=0, dj=0, dk=0):
    """F evaluated at (i+di, j+dj, k+dk), periodic."""
    return np.roll(F, shift=(-dk, -dj, -di), axis=(0, 1, 2))


def _off(axis, n):
    o = [0, 0, 0]
    o[axis] = n
    return o


def _plus(a, b):
    return [a[0] + b[0], a[1] + b[1], a[2] + b[2]]


class Coeffs:
    """beta_ij / delta_i of Eq. (D*) with alpha_i from Eq. (alpha); grid spacing and dt."""

    def __init__(self, beta, delta, dx, dt, alpha=None):
        """``alpha`` overrides Eq. (alpha); it is used only to run the scheme with
        coefficients as rounded to a lower working precision, where the rounded
        alpha no longer satisfies Eq. (alpha) exactly."""
        self.beta = np.array(beta, dtype=np.float64).reshape(3, 3)
        self.delta = np.array(delta, dtype=np.float64).reshape(3)
        self.dx = np.array(dx, dtype=np.float64).reshape(3)
        self.dt = float(dt)
        if alpha is not None:
            self.alpha = np.array(alpha, dtype=np.float64).reshape(3)
        else:
            self.alpha = np.array([
                1.0 - 2.0 * sum(self.beta[i, j] for j in range(3) if j != i) - 3.0 * self.delta[i]
                for i in range(3)])


# ----------------------------------------------------------------------------
# stencils
# ----------------------------------------------------------------------------


def dstar_taps(a, c: Coeffs):
    """The 12 taps of D*_a (Eq. D*) as (weight, offset) pairs, weights already divided by dx_a.

    Output position is +1/2 along a from the input's position:
      alpha_a (X[+1] - X[0]) + delta_a (X[+2] - X[-1])
      + beta_ab [(X[+1,+b] - X[0,+b]) + (X[+1,-b] - X[0,-b])]   for both transverse b.
    """
    inv = 1.0 / c.dx[a]
    taps = [(c.alpha[a] * inv, _off(a, 1)), (-c.alpha[a] * inv, _off(a, 0)),
            (c.delta[a] * inv, _off(a, 2)), (-c.delta[a] * inv, _off(a, -1))]
    for b in range(3):
        if b == a:
            continue
        for s in (1, -1):
            taps.append((c.beta[a, b] * inv, _plus(_off(a, 1), _off(b, s))))
            taps.append((-c.beta[a, b] * inv, _off(b, s)))
    return taps


def dstar(a, F, c: Coeffs):
    out = np.zeros_like(F)
    for w, o in dstar_taps(a, c):
        out += w * at(F, *o)
    return out


def dstar_T(a, G, c: Coeffs):
    """Transpose of ``dstar``: each tap F[c+o] -> out[c] becomes G[c] -> out[c+o]."""
    out = np.zeros_like(G)
    for w, o in dstar_taps(a, c):
        out += w * at(G, -o[0], -o[1], -o[2])
    return out


def dstar_dcoef(a, F, c: Coeffs):
    """d(D*_a F)/d(free coefficient) with alpha eliminated (Eq. alpha).

    Returns {("delta", a): ..., ("beta", a, b): ...}.  Since
    alpha_a = 1 - 2 sum_b beta_ab - 3 delta_a:
      d/d delta_a  = [(F[+2] - F[-1]) - 3 (F[+1] - F[0])] / dx_a
      d/d beta_ab  = [(F[+1,+b] - F[0,+b]) + (F[+1,-b] - F[0,-b]) - 2 (F[+1] - F[0])] / dx_a
    """
    inv = 1.0 / c.dx[a]
    axial = at(F, *_off(a, 1)) - F
    res = {("delta", a): inv * ((at(F, *_off(a, 2)) - at(F, *_off(a, -1))) - 3.0 * axial)}
    for b in range(3):
        if b == a:
            continue
        trans = 0.0
        for s in (1, -1):
            trans = trans + at(F, *_plus(_off(a, 1), _off(b, s))) - at(F, *_off(b, s))
        res[("beta", a, b)] = inv * (trans - 2.0 * axial)
    return res


def dyee(a, F, c: Coeffs):
    """Yee D_a (Ampere): backward difference (F[0] - F[-1]) / dx_a."""
    return (F - at(F, *_off(a, -1))) / c.dx[a]


def dyee_T(a, G, c: Coeffs):
    return (G - at(G, *_off(a, 1))) / c.dx[a]


def dyee_fwd(a, F, c: Coeffs):
    """Yee difference in the forward sense (F[+1] - F[0]) / dx_a, used by D.B."""
    return (at(F, *_off(a, 1)) - F) / c.dx[a]


# ----------------------------------------------------------------------------
# sponge
# ----------------------------------------------------------------------------


def sponge_profile(n, L, sigma):
    f = np.ones(n)
    if L <= 0:
        return f
    for m in range(L):
        d = L - m  # depth 1..L, deepest at the array edge
        f[m] = 1.0 - sigma * (d / L) ** 3
        f[n - 1 - m] = 1.0 - sigma * (d / L) ** 3
    return f


def sponge_factor(shape, L, sigma):
    nz, ny, nx = shape
    fy = sponge_profile(ny, L, sigma)
    fz = sponge_profile(nz, L, sigma)
    return fz[:, None, None] * fy[None, :, None] * np.ones(nx)[None, None, :]


# ----------------------------------------------------------------------------
# rigid bunch current (continuity-exact, App. A continuity equation)
# ----------------------------------------------------------------------------


def _Phi(x):
    """Standard normal CDF."""
    from scipy.special import erf
    return 0.5 * (1.0 + erf(np.asarray(x, dtype=np.float64) / math.sqrt(2.0)))


def _wrapd(x, L):
    return (x + 0.5 * L) % L - 0.5 * L


class Bunch:
    """Gaussian charge q moving rigidly along +x at speed v (a reading; the paper uses PIC).

    rho on nodes is the cell-integrated Gaussian divided by the cell volume;
    J_x at (i+1/2, j, k) between steps n and n+1 is chosen so that
    (rho^{n+1} - rho^n)/dt + D.J^{n+1/2} = 0 holds exactly (App. A).
    """

    def __init__(self, q, v, x0, y0, z0, sig_par, sig_perp):
        self.q, self.v = q, v
        self.x0, self.y0, self.z0 = x0, y0, z0
        self.sp, self.st = sig_par, sig_perp

    def _perp(self, shape, c):
        nz, ny, _ = shape
        jy = np.arange(ny) * c.dx[1]
        kz = np.arange(nz) * c.dx[2]
        Ly, Lz = ny * c.dx[1], nz * c.dx[2]
        dy = _wrapd(jy - self.y0, Ly)
        dz = _wrapd(kz - self.z0, Lz)
        gy = _Phi((dy + 0.5 * c.dx[1]) / self.st) - _Phi((dy - 0.5 * c.dx[1]) / self.st)
        gz = _Phi((dz + 0.5 * c.dx[2]) / self.st) - _Phi((dz - 0.5 * c.dx[2]) / self.st)
        return gz[:, None] * gy[None, :]

    def xc(self, n, c):
        return self.x0 + self.v * c.dt * n

    def rho(self, shape, n, c):
        nz, ny, nx = shape
        Lx = nx * c.dx[0]
        xi = np.arange(nx) * c.dx[0]
        d = _wrapd(xi - self.xc(n, c), Lx)
        gx = _Phi((d + 0.5 * c.dx[0]) / self.sp) - _Phi((d - 0.5 * c.dx[0]) / self.sp)
        vol = c.dx[0] * c.dx[1] * c.dx[2]
        return self.q * self._perp(shape, c)[:, :, None] * gx[None, None, :] / vol

    def Jx(self, shape, n, c):
        """J_x^{n+1/2} at (i+1/2, j, k) = q g_y g_z / (dy dz) * [G^n - G^{n+1}](x_{i+1/2}) / dt."""
        nz, ny, nx = shape
        Lx = nx * c.dx[0]
        xf = (np.arange(nx) + 0.5) * c.dx[0]
        # both cdf values are taken for the same periodic image of the bunch, so
        # their difference is a localised bump (no jump at the far side of the box)
        d = _wrapd(xf - self.xc(n, c), Lx)
        Gn = _Phi(d / self.sp)
        Gn1 = _Phi((d - (self.xc(n + 1, c) - self.xc(n, c))) / self.sp)
        return (self.q * self._perp(shape, c)[:, :, None] / (c.dx[1] * c.dx[2])
                * (Gn - Gn1)[None, None, :] / c.dt)


# ----------------------------------------------------------------------------
# forward step (App. A update equations)
# ----------------------------------------------------------------------------


class State:
    def __init__(self, E, B):
        self.E = [np.array(e, dtype=np.float64) for e in E]
        self.B = [np.array(b, dtype=np.float64) for b in B]

    def copy(self):
        return State([e.copy() for e in self.E], [b.copy() for b in self.B])

    def flat(self):
        return np.concatenate([a.ravel() for a in self.E + self.B])


def faraday_rhs(E, c: Coeffs):
    """-D* x E, component by component:  (D*_z E_y - D*_y E_z, D*_x E_z - D*_z E_x, D*_y E_x - D*_x E_y)."""
    return [dstar(Z, E[Y], c) - dstar(Y, E[Z], c),
            dstar(X, E[Z], c) - dstar(Z, E[X], c),
            dstar(Y, E[X], c) - dstar(X, E[Y], c)]


def ampere_curl(B, c: Coeffs):
    """Yee D x B:  (D_y B_z - D_z B_y, D_z B_x - D_x B_z, D_x B_y - D_y B_x)."""
    return [dyee(Y, B[Z], c) - dyee(Z, B[Y], c),
            dyee(Z, B[X], c) - dyee(X, B[Z], c),
            dyee(X, B[Y], c) - dyee(Y, B[X], c)]


def step(s: State, c: Coeffs, J=None, sponge=None):
    """One leapfrog step: B^{n+1/2} from E^n (extended stencil), then E^{n+1} from B^{n+1/2} (Yee)."""
    f = faraday_rhs(s.E, c)
    for a in range(3):
        s.B[a] = s.B[a] + c.dt * f[a]
        if sponge is not None:
            s.B[a] = s.B[a] * sponge
    g = ampere_curl(s.B, c)
    for a in range(3):
        src = 0.0 if J is None or J[a] is None else J[a]
        s.E[a] = s.E[a] + c.dt * (g[a] - src)
        if sponge is not None:
            s.E[a] = s.E[a] * sponge
    return s


def run(s: State, c: Coeffs, n, bunch: Bunch | None = None, n0=0, sponge=None, hook=None):
    """Advance n steps; ``bunch`` supplies J^{n+1/2} for absolute step index n0 + m."""
    shape = s.E[0].shape
    for m in range(n):
        J = None
        if bunch is not None:
            J = [bunch.Jx(shape, n0 + m, c), None, None]
        step(s, c, J, sponge)
        if hook is not None:
            hook(m + 1, s)
    return s


# ----------------------------------------------------------------------------
# adjoint step and coefficient gradient
# ----------------------------------------------------------------------------

COEF_KEYS = [("beta", a, b) for a in range(3) for b in range(3) if a != b] + \
            [("delta", a) for a in range(3)]


def adjoint_step(lam: State, E_n, c: Coeffs, grad: dict, sponge=None):
    """Transpose of one ``step`` (J drops out: it does not depend on the state).

    Forward: B1 = S(B0 + dt F E0); E1 = S(E0 + dt (G B1 - J)), F = -D* x, G = D x.
    Given lam = (lam_E, lam_B) attached to (E1, B1):
      l_E = S lam_E;  mu = S (lam_B + dt G^T l_E);
      lam_E <- l_E + dt F^T mu;  lam_B <- mu;
      dL/d theta += dt * <mu, (dF/d theta) E0>.
    ``E_n`` is the forward E^n of this step.  ``grad`` maps COEF_KEYS to floats.
    """
    lE = [l * sponge if sponge is not None else l for l in lam.E]
    # G^T: transpose of ampere_curl, component by component
    nu = [lam.B[X] + c.dt * (dyee_T(Z, lE[Y], c) - dyee_T(Y, lE[Z], c)),
          lam.B[Y] + c.dt * (dyee_T(X, lE[Z], c) - dyee_T(Z, lE[X], c)),
          lam.B[Z] + c.dt * (dyee_T(Y, lE[X], c) - dyee_T(X, lE[Y], c))]
    mu = [v * sponge if sponge is not None else v for v in nu]
    # coefficient gradient from (dF/d theta) E_n, with F E = faraday_rhs(E)
    pairs = [(X, Z, Y, +1), (X, Y, Z, -1),   # mu_x: +D*_z E_y - D*_y E_z
             (Y, X, Z, +1), (Y, Z, X, -1),   # mu_y: +D*_x E_z - D*_z E_x
             (Z, Y, X, +1), (Z, X, Y, -1)]   # mu_z: +D*_y E_x - D*_x E_y
    for comp, axis, field, sign in pairs:
        for key, val in dstar_dcoef(axis, E_n[field], c).items():
            grad[key] = grad.get(key, 0.0) + c.dt * sign * float(np.sum(mu[comp] * val))
    # F^T: transpose of faraday_rhs
    newE = [lE[X] + c.dt * (dstar_T(Y, mu[Z], c) - dstar_T(Z, mu[Y], c)),
            lE[Y] + c.dt * (dstar_T(Z, mu[X], c) - dstar_T(X, mu[Z], c)),
            lE[Z] + c.dt * (dstar_T(X, mu[Y], c) - dstar_T(Y, mu[X], c))]
    lam.E = newE
    lam.B = mu
    return lam


def grad_to_arrays(grad):
    gb = np.zeros((3, 3))
    gd = np.zeros(3)
    for key, v in grad.items():
        if key[0] == "beta":
            gb[key[1], key[2]] += v
        else:
            gd[key[1]] += v
    return gb, gd


# ----------------------------------------------------------------------------
# diagnostics (Sec. 2.1, 2.2; App. A continuity)
# ----------------------------------------------------------------------------


def div_star_B(B, c: Coeffs):
    """Eq. (divstarb): D* . B at (i+1/2, j+1/2, k+1/2)."""
    return dstar(X, B[X], c) + dstar(Y, B[Y], c) + dstar(Z, B[Z], c)


def div_yee_B(B, c: Coeffs):
    """Yee D . B at (i+1/2, j+1/2, k+1/2) (forward differences from B positions)."""
    return dyee_fwd(X, B[X], c) + dyee_fwd(Y, B[Y], c) + dyee_fwd(Z, B[Z], c)


def div_E(E, c: Coeffs):
    """Eq. (divE): D . E at the nodes (i, j, k) (backward differences)."""
    return dyee(X, E[X], c) + dyee(Y, E[Y], c) + dyee(Z, E[Z], c)


def energy(s: State, mask=None):
    tot = 0.0
    for a in range(3):
        e2 = s.E[a] ** 2 + s.B[a] ** 2
        tot += float(np.sum(e2 if mask is None else e2 * mask))
    return 0.5 * tot


def plane_wave_amplitude(F, kvec, dx, offset=(0.0, 0.0, 0.0)):
    """sum_cells F exp(-i k . x) with x the component's staggered position."""
    nz, ny, nx = F.shape
    x = (np.arange(nx) + offset[0]) * dx[0]
    y = (np.arange(ny) + offset[1]) * dx[1]
    z = (np.arange(nz) + offset[2]) * dx[2]
    ph = np.exp(-1j * kvec[0] * x)[None, None, :] * np.exp(-1j * kvec[1] * y)[None, :, None] \
        * np.exp(-1j * kvec[2] * z)[:, None, None]
    return complex(np.sum(F * ph))


def energy_moments(s: State, axis, dx):
    """Energy moments along one axis, for the packet centroid (Sec. 5, group velocity):
    (W, C, S) = sum over the six components and all cells of (1/2) F^2 dV (1, cos th, sin th),
    th = 2 pi (index_axis + o) / n_axis, o = 1/2 where the component is staggered along the axis
    (E_axis, and the two B components other than B_axis; App. A positions).
    The periodic centroid is atan2(S, C) n_axis dx_axis / (2 pi)."""
    fields = list(s.E) + list(s.B)
    n = fields[0].shape[2 - axis]
    dV = dx[0] * dx[1] * dx[2]
    W = C = S = 0.0
    for q, F in enumerate(fields):
        comp = q % 3
        staggered = (comp == axis) if q < 3 else (comp != axis)
        o = 0.5 if staggered else 0.0
        th = 2.0 * math.pi * (np.arange(n) + o) / n
        e = 0.5 * F * F * dV
        # sum over the two other axes, leaving a profile along `axis`
        prof = e.sum(axis=tuple(a for a in range(3) if a != 2 - axis))
        W += float(prof.sum())
        C += float(np.sum(prof * np.cos(th)))
        S += float(np.sum(prof * np.sin(th)))
    return W, C, S


def dt_of_courant(nu, dtmax):
    return nu * dtmax


def isclose_rel(a, b, tol):
    return abs(a - b) <= tol * max(abs(a), abs(b), 1e-300)


__all__ = ["Coeffs", "State", "Bunch", "step", "run", "adjoint_step", "grad_to_arrays",
           "div_star_B", "div_yee_B", "div_E", "energy", "plane_wave_amplitude", "energy_moments",
           "sponge_factor", "COEF_KEYS", "math"]
