"""Numerical dispersion relation, dispersion norm and CFL limit -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain numpy, written
from the paper, no blocking or fusion beyond what the formulas state.

Conventions
-----------
* ``beta`` is a 3x3 array, ``beta[i][j]`` = beta_ij of Eq. (D*): the
  coefficient of the transverse-neighbour taps of D*_i displaced along axis
  j.  The diagonal is unused.  ``delta[i]`` = delta_i.  alpha_i is never an
  input: it is eliminated with Eq. (alpha).
* ``dims`` = 1, 2 or 3.  Axes beyond ``dims`` carry no wave vector (k = 0)
  and their coefficients are ignored (treated as zero).
* Units: c = 1.

Readings of the paper taken here:
* App. B, final line: the paper prints ``+4 sum dx_j^2 beta_ij s_i^2 s_j^2``.
  The line before it has ``beta_ij/dx_i^2 (-1 + c_i + c_j - c_i c_j)``, which
  equals ``-4 dx_j^2 beta_ij s_i^2 s_j^2``; the minus sign is the one
  consistent with Eq. (dispersion_relation) and with NDFX being stable at
  c dt = dx.  ``S_reduced`` uses the minus sign.
* Eq. (norm) is taken unnormalised over the positive octant, evaluated with
  the midpoint rule on an N_x x N_y (x N_z) grid; in 2D the z integral and
  dz are dropped.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# coefficients
# ----------------------------------------------------------------------------


def clean_coeffs(beta, delta, dims):
    """Return (beta, delta) as float64 arrays with entries of absent axes zeroed.

    For dims < 3 the stencil has no taps along the missing axes, which is the
    same as setting the corresponding beta / delta entries to zero (Sec. 4:
    "the number of dimensions" is one of the choices fixing the stencil).
    """
    b = np.array(beta, dtype=np.float64).reshape(3, 3).copy()
    d = np.array(delta, dtype=np.float64).reshape(3).copy()
    for i in range(3):
        b[i, i] = 0.0
    for ax in range(dims, 3):
        b[:, ax] = 0.0
        b[ax, :] = 0.0
        d[ax] = 0.0
    return b, d


def alpha(beta, delta, dims=3):
    """Eq. (alpha): alpha_i = 1 - 2 sum_{j != i} beta_ij - 3 delta_i."""
    b, d = clean_coeffs(beta, delta, dims)
    return np.array([1.0 - 2.0 * (b[i].sum()) - 3.0 * d[i] for i in range(3)])


# ----------------------------------------------------------------------------
# dispersion relation
# ----------------------------------------------------------------------------


def s_sq(k, dx):
    """s_i^2 = sin^2(k_i dx_i / 2) / dx_i^2 (Sec. 3, abbreviations)."""
    return np.sin(0.5 * k * dx) ** 2 / dx ** 2


def S_paper(kx, ky, kz, beta, delta, dx, dims=3, alpha_override=None):
    """Right-hand side of Eq. (dispersion_relation): sum_i s_i^2 A_i, with A_i as printed.

    A_x = alpha_x + 2 beta_xy cos(k_y dy) + 2 beta_xz cos(k_z dz) + delta_x (1 + 2 cos(k_x dx)),
    and cyclically for y and z.  ``alpha_override`` replaces Eq. (alpha); it serves
    only to evaluate the relation for coefficients rounded to a working precision.
    """
    b, d = clean_coeffs(beta, delta, dims)
    a = alpha(b, d, dims) if alpha_override is None else np.asarray(alpha_override, dtype=np.float64)
    k = [np.asarray(kx, dtype=np.float64), np.asarray(ky, dtype=np.float64),
         np.asarray(kz, dtype=np.float64)]
    dxa = np.asarray(dx, dtype=np.float64)
    total = 0.0
    for i in range(dims):
        A = a[i] + d[i] * (1.0 + 2.0 * np.cos(k[i] * dxa[i]))
        for j in range(3):
            if j != i:
                A = A + 2.0 * b[i, j] * np.cos(k[j] * dxa[j])
        total = total + s_sq(k[i], dxa[i]) * A
    return total


def S_reduced(kx, ky, kz, beta, delta, dx, dims=3):
    """App. B reduced form (sign-corrected, see module docstring):

    s_omega^2 = sum_i s_i^2 (1 - 4 dx_i^2 delta_i s_i^2) - 4 sum_{i != j} dx_j^2 beta_ij s_i^2 s_j^2.
    """
    b, d = clean_coeffs(beta, delta, dims)
    k = [np.asarray(kx, dtype=np.float64), np.asarray(ky, dtype=np.float64),
         np.asarray(kz, dtype=np.float64)]
    dxa = np.asarray(dx, dtype=np.float64)
    s2 = [s_sq(k[i], dxa[i]) for i in range(3)]
    total = 0.0
    for i in range(dims):
        total = total + s2[i] * (1.0 - 4.0 * dxa[i] ** 2 * d[i] * s2[i])
    for i in range(dims):
        for j in range(dims):
            if i != j:
                total = total - 4.0 * dxa[j] ** 2 * b[i, j] * s2[i] * s2[j]
    return total


def omega_from_S(S, dt):
    """Invert s_omega^2 = S: omega = (2/dt) asin(dt sqrt(S))  (c = 1)."""
    arg = dt * np.sqrt(S)
    return 2.0 / dt * np.arcsin(arg)


def omega(kx, ky, kz, beta, delta, dt, dx, dims=3):
    return omega_from_S(S_paper(kx, ky, kz, beta, delta, dx, dims), dt)


# ----------------------------------------------------------------------------
# exact extremes of S over the Brillouin box, CFL limit (Eq. constraints)
# ----------------------------------------------------------------------------


def _quadratic_form(beta, delta, dx, dims):
    """S as a quadratic in u_i = s_i^2 in [0, 1/dx_i^2]:  S(u) = sum u - u^T Q u."""
    b, d = clean_coeffs(beta, delta, dims)
    dxa = np.asarray(dx, dtype=np.float64)
    Q = np.zeros((dims, dims))
    for i in range(dims):
        Q[i, i] = 4.0 * dxa[i] ** 2 * d[i]
        for j in range(dims):
            if i != j:
                # each unordered pair appears twice in u^T Q u
                Q[i, j] = 2.0 * (dxa[j] ** 2 * b[i, j] + dxa[i] ** 2 * b[j, i])
    ub = 1.0 / dxa[:dims] ** 2
    return Q, ub


def S_extremes(beta, delta, dx, dims=3):
    """Exact (min, max) of S over 0 <= k_i <= pi/dx_i.

    S is a quadratic in u = (s_x^2, s_y^2, s_z^2) over a box.  Every extremum
    lies at a point where each coordinate is either at a bound or free, with
    the gradient vanishing in the free coordinates.  All 3^dims such patterns
    are enumerated and their linear systems solved; singular systems are
    skipped (their extrema are then attained on a lower-dimensional face,
    which another pattern covers).
    """
    Q, ub = _quadratic_form(beta, delta, dx, dims)
    vals = []
    for pattern in itertools.product((0, 1, 2), repeat=dims):  # 0: lower, 1: upper, 2: free
        u = np.zeros(dims)
        free = [i for i in range(dims) if pattern[i] == 2]
        for i in range(dims):
            if pattern[i] == 1:
                u[i] = ub[i]
        if free:
            fixed = [i for i in range(dims) if pattern[i] != 2]
            A = 2.0 * Q[np.ix_(free, free)]
            rhs = np.ones(len(free))
            if fixed:
                rhs = rhs - 2.0 * Q[np.ix_(free, fixed)] @ u[fixed]
            if abs(np.linalg.det(A)) < 1e-14 * max(1.0, np.abs(A).max() ** len(free)):
                continue
            uf = np.linalg.solve(A, rhs)
            if np.any(uf < -1e-15) or np.any(uf > ub[free] * (1 + 1e-15)):
                continue
            u[free] = np.clip(uf, 0.0, ub[free])
        vals.append(u.sum() - u @ Q @ u)
    return min(vals), max(vals)


def dt_max(beta, delta, dx, dims=3):
    """Largest dt with dt^2 max_k S(k) <= 1 (right-hand inequality of Eq. constraints)."""
    _, smax = S_extremes(beta, delta, dx, dims)
    if smax <= 0:
        return math.inf
    return 1.0 / math.sqrt(smax)


def is_well_defined(beta, delta, dt, dx, dims=3, tol=1e-12):
    """Eq. (constraints): 0 <= dt^2 S <= 1 everywhere in the box."""
    smin, smax = S_extremes(beta, delta, dx, dims)
    return smin >= -tol and dt * dt * smax <= 1.0 + tol


# ----------------------------------------------------------------------------
# dispersion norm (Eq. norm) and its gradient
# ----------------------------------------------------------------------------

WEIGHT_UNIFORM = 0
WEIGHT_CONE_X = 1      # w = 1 inside a cone of half-angle `param` (radians) about +x
WEIGHT_GAUSS_Y = 2     # w = exp(-(k_y dy / param)^2), Eq. (norm_x_axis)


def weight(kx, ky, kz, kind, param, dx):
    if kind == WEIGHT_UNIFORM:
        return np.ones_like(kx)
    if kind == WEIGHT_CONE_X:
        kn = np.sqrt(kx * kx + ky * ky + kz * kz)
        return (kx >= kn * math.cos(param)).astype(np.float64)
    if kind == WEIGHT_GAUSS_Y:
        return np.exp(-(ky * dx[1] / param) ** 2)
    raise ValueError(kind)


def midpoint_grid(N, dx, dims):
    """Midpoint nodes k_i = (m + 1/2) pi / (N_i dx_i), m = 0..N_i-1, and the cell volume."""
    axes = []
    vol = 1.0
    for i in range(3):
        if i < dims:
            axes.append((np.arange(N[i]) + 0.5) * math.pi / (N[i] * dx[i]))
            vol *= math.pi / (N[i] * dx[i])
        else:
            axes.append(np.zeros(1))
    KZ, KY, KX = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return KX, KY, KZ, vol


def norm(beta, delta, dt, dx, N, dims=3, wkind=WEIGHT_UNIFORM, wparam=0.0):
    """Eq. (norm) by the midpoint rule: prod(dx) * sum w (omega - |k|)^2 * cell volume."""
    dxa = np.asarray(dx, dtype=np.float64)
    KX, KY, KZ, vol = midpoint_grid(N, dxa, dims)
    S = S_paper(KX, KY, KZ, beta, delta, dxa, dims)
    w = omega_from_S(S, dt)
    kn = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    wt = weight(KX, KY, KZ, wkind, wparam, dxa)
    return float(np.prod(dxa[:dims]) * vol * np.sum(wt * (w - kn) ** 2))


def norm_and_grad(beta, delta, dt, dx, N, dims=3, wkind=WEIGHT_UNIFORM, wparam=0.0):
    """Eq. (norm) and its closed-form gradient.

    Returns (f, g_beta[3,3], g_delta[3], g_dt).  Chain rule through
    omega = (2/dt) asin(dt sqrt S):
      d omega / d S  = 1 / (sqrt(S) sqrt(1 - dt^2 S)),
      d omega / d dt = -omega/dt + 2 sqrt(S) / (dt sqrt(1 - dt^2 S)),
    and from Eq. (dispersion_relation) with alpha eliminated by Eq. (alpha),
      dS/d beta_ij = s_i^2 * 2 (cos(k_j dx_j) - 1) = -4 dx_j^2 s_i^2 s_j^2,
      dS/d delta_i = s_i^2 * 2 (cos(k_i dx_i) - 1) = -4 dx_i^2 s_i^4.
    """
    dxa = np.asarray(dx, dtype=np.float64)
    KX, KY, KZ, vol = midpoint_grid(N, dxa, dims)
    K = [KX, KY, KZ]
    S = S_paper(KX, KY, KZ, beta, delta, dxa, dims)
    w = omega_from_S(S, dt)
    kn = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    wt = weight(KX, KY, KZ, wkind, wparam, dxa)
    pref = float(np.prod(dxa[:dims]) * vol)
    r = w - kn
    f = pref * float(np.sum(wt * r * r))
    root = np.sqrt(1.0 - dt * dt * S)
    dw_dS = 1.0 / (np.sqrt(S) * root)
    dw_ddt = -w / dt + 2.0 * np.sqrt(S) / (dt * root)
    common = 2.0 * wt * r
    s2 = [s_sq(K[i], dxa[i]) for i in range(3)]
    gb = np.zeros((3, 3))
    gd = np.zeros(3)
    for i in range(dims):
        for j in range(dims):
            if i != j:
                dS = s2[i] * 2.0 * (np.cos(K[j] * dxa[j]) - 1.0)
                gb[i, j] = pref * float(np.sum(common * dw_dS * dS))
        dS = s2[i] * 2.0 * (np.cos(K[i] * dxa[i]) - 1.0)
        gd[i] = pref * float(np.sum(common * dw_dS * dS))
    gdt = pref * float(np.sum(common * dw_ddt))
    return f, gb, gd, gdt


def norm_bruteforce(beta, delta, dt, dx, N, dims=3, wkind=WEIGHT_UNIFORM, wparam=0.0):
    """The same midpoint sum written as explicit Python loops (tiny N only)."""
    dxa = [float(v) for v in dx]
    b, d = clean_coeffs(beta, delta, dims)
    a = alpha(b, d, dims)
    total = 0.0
    ranges = [range(N[i]) if i < dims else range(1) for i in range(3)]
    h = [math.pi / (N[i] * dxa[i]) if i < dims else 0.0 for i in range(3)]
    for mz in ranges[2]:
        for my in ranges[1]:
            for mx in ranges[0]:
                k = [(mx + 0.5) * h[0], (my + 0.5) * h[1], (mz + 0.5) * h[2]]
                for i in range(dims, 3):
                    k[i] = 0.0
                S = 0.0
                for i in range(dims):
                    A = a[i] + d[i] * (1 + 2 * math.cos(k[i] * dxa[i]))
                    for j in range(3):
                        if j != i:
                            A += 2 * b[i, j] * math.cos(k[j] * dxa[j])
                    S += (math.sin(k[i] * dxa[i] / 2) / dxa[i]) ** 2 * A
                om = 2 / dt * math.asin(dt * math.sqrt(S))
                kn = math.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
                if wkind == WEIGHT_UNIFORM:
                    wt = 1.0
                elif wkind == WEIGHT_CONE_X:
                    wt = 1.0 if k[0] >= kn * math.cos(wparam) else 0.0
                else:
                    wt = math.exp(-(k[1] * dxa[1] / wparam) ** 2)
                total += wt * (om - kn) ** 2
    vol = 1.0
    for i in range(dims):
        vol *= h[i] * dxa[i]
    return total * vol


# ----------------------------------------------------------------------------
# phase / group velocity (Sec. 5)
# ----------------------------------------------------------------------------


def phase_velocity_extremes(beta, delta, dt, dx, n=1024, dims=2):
    """min and max of v_ph = omega/|k| over the box, on the grid k_i = pi m / (n dx_i), m = 1..n."""
    dxa = np.asarray(dx, dtype=np.float64)
    axes = [np.arange(1, n + 1) * math.pi / (n * dxa[i]) if i < dims else np.zeros(1)
            for i in range(3)]
    KZ, KY, KX = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    w = omega(KX, KY, KZ, beta, delta, dt, dxa, dims)
    v = w / np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    return float(v.min()), float(v.max())


def group_velocity(kvec, beta, delta, dt, dx, dims=3, h=1e-6):
    """grad_k omega by central differences of the closed form (Sec. 5, |v_g| = |d omega/dk|)."""
    kvec = np.asarray(kvec, dtype=np.float64)
    g = np.zeros(3)
    for i in range(dims):
        e = np.zeros(3)
        e[i] = h
        wp = omega(*(kvec + e), beta, delta, dt, dx, dims)
        wm = omega(*(kvec - e), beta, delta, dt, dx, dims)
        g[i] = (wp - wm) / (2 * h)
    return g


# ----------------------------------------------------------------------------
# group-velocity norm (a reading of the conclusions: "minimization of the numerical
# group velocity error"); not printed in the paper, so its values are pinned by closed
# forms, central differences and brute force only
# ----------------------------------------------------------------------------


def group_speed_terms(KX, KY, KZ, beta, delta, dt, dx, dims=3):
    """Per point: S, grad_k S (3 arrays) and |v_g| = |d omega/dk| = omega'(S) |grad_k S|,
    omega'(S) = 1 / (sqrt(S) sqrt(1 - dt^2 S)).  With alpha eliminated by Eq. (alpha),
    A_i = 1 + 2 sum_{j != i} beta_ij (c_j - 1) + 2 delta_i (c_i - 1), S = sum_i s_i^2 A_i, and
      dS/dk_m = sin(k_m dx_m) / (2 dx_m) A_m
                - 2 dx_m sin(k_m dx_m) (delta_m s_m^2 + sum_{i != m} beta_im s_i^2)."""
    b, d = clean_coeffs(beta, delta, dims)
    dxa = np.asarray(dx, dtype=np.float64)
    K = [KX, KY, KZ]
    s2 = [s_sq(K[i], dxa[i]) for i in range(3)]
    c = [np.cos(K[i] * dxa[i]) for i in range(3)]
    sn = [np.sin(K[i] * dxa[i]) for i in range(3)]
    A = []
    for i in range(3):
        a = 1.0 + 2.0 * d[i] * (c[i] - 1.0)
        for j in range(3):
            if j != i:
                a = a + 2.0 * b[i, j] * (c[j] - 1.0)
        A.append(a)
    S = sum(s2[i] * A[i] for i in range(dims))
    G = []
    for m in range(3):
        if m >= dims:
            G.append(np.zeros_like(S))
            continue
        t = d[m] * s2[m]
        for i in range(dims):
            if i != m:
                t = t + b[i, m] * s2[i]
        G.append(sn[m] / (2.0 * dxa[m]) * A[m] - 2.0 * dxa[m] * sn[m] * t)
    wS = 1.0 / (np.sqrt(S) * np.sqrt(1.0 - dt * dt * S))
    Gn = np.sqrt(G[0] ** 2 + G[1] ** 2 + G[2] ** 2)
    return dict(S=S, G=G, Gn=Gn, wS=wS, vg=wS * Gn, s2=s2, c=c, sn=sn, A=A)


def group_norm_and_grad(beta, delta, dt, dx, N, dims=3, wkind=WEIGHT_UNIFORM, wparam=0.0):
    """f_g = prod(dx) sum w (|v_g| - 1)^2 * cell volume on the midpoint grid of Eq. (norm), and
    its gradient.  Chain rule: with r = |v_g| - 1,
      d|v_g|/d theta = omega''(S) dS/dtheta |G| + omega'(S) (G . dG/dtheta) / |G|,
      omega''(S) = -omega'(S)^3 (1 - 2 dt^2 S) / 2,   d omega'(S)/d dt = omega'(S)^3 dt S^2,
      dS/d beta_ij = 2 s_i^2 (c_j - 1),  dS/d delta_i = 2 s_i^2 (c_i - 1),
      dG_m/d beta_ij = [m = i] sin(k_i dx_i)(c_j - 1)/dx_i - [m = j] 2 dx_j sin(k_j dx_j) s_i^2,
      dG_m/d delta_i = [m = i] (sin(k_i dx_i)(c_i - 1)/dx_i - 2 dx_i sin(k_i dx_i) s_i^2).
    Returns (f, g_beta[3,3], g_delta[3], g_dt)."""
    dxa = np.asarray(dx, dtype=np.float64)
    KX, KY, KZ, vol = midpoint_grid(N, dxa, dims)
    t = group_speed_terms(KX, KY, KZ, beta, delta, dt, dxa, dims)
    S, G, Gn, wS, vg = t["S"], t["G"], t["Gn"], t["wS"], t["vg"]
    s2, c, sn = t["s2"], t["c"], t["sn"]
    wt = weight(KX, KY, KZ, wkind, wparam, dxa)
    pref = float(np.prod(dxa[:dims]) * vol)
    r = vg - 1.0
    f = pref * float(np.sum(wt * r * r))
    wSS = -0.5 * wS ** 3 * (1.0 - 2.0 * dt * dt * S)
    common = 2.0 * wt * r
    gb = np.zeros((3, 3))
    gd = np.zeros(3)
    for i in range(dims):
        for j in range(dims):
            if i == j:
                continue
            dS = 2.0 * s2[i] * (c[j] - 1.0)
            GdG = G[i] * sn[i] * (c[j] - 1.0) / dxa[i] - G[j] * 2.0 * dxa[j] * sn[j] * s2[i]
            dv = wSS * dS * Gn + wS * GdG / Gn
            gb[i, j] = pref * float(np.sum(common * dv))
        dS = 2.0 * s2[i] * (c[i] - 1.0)
        GdG = G[i] * (sn[i] * (c[i] - 1.0) / dxa[i] - 2.0 * dxa[i] * sn[i] * s2[i])
        dv = wSS * dS * Gn + wS * GdG / Gn
        gd[i] = pref * float(np.sum(common * dv))
    gdt = pref * float(np.sum(common * wS ** 3 * dt * S * S * Gn))
    return f, gb, gd, gdt


def group_norm_fd(beta, delta, dt, dx, N, dims=3, wkind=WEIGHT_UNIFORM, wparam=0.0, h=1e-6):
    """The same sum with |v_g| from central differences of omega(k) (group_velocity), written
    as explicit loops over the points (small N only)."""
    dxa = np.asarray(dx, dtype=np.float64)
    KX, KY, KZ, vol = midpoint_grid(N, dxa, dims)
    wt = weight(KX, KY, KZ, wkind, wparam, dxa)
    total = 0.0
    for idx in np.ndindex(KX.shape):
        k = np.array([KX[idx], KY[idx], KZ[idx]])
        v = np.linalg.norm(group_velocity(k, beta, delta, dt, dxa, dims, h))
        total += wt[idx] * (v - 1.0) ** 2
    return float(np.prod(dxa[:dims]) * vol * total)


# ----------------------------------------------------------------------------
# constrained minimisation (Sec. 4): SLSQP, bounds cuboid, multistart grid
# ----------------------------------------------------------------------------


def minimise(unpack, x_bounds, starts, dx, N, dims=2, wkind=WEIGHT_UNIFORM, wparam=0.0,
             maxiter=200):
    """Minimise Eq. (norm) with SciPy SLSQP under Eq. (constraints), from every start point.

    ``unpack(x) -> (beta, delta, dt)`` maps the free-parameter vector to a
    full coefficient set; ``x_bounds`` is the search cuboid.  The constraints
    are 1 - dt^2 max S >= 0 and min S >= 0 (exact extremes).  Returns
    (best_x, best_f).
    """
    from scipy.optimize import minimize

    def obj(x):
        b, d, dt = unpack(x)
        if not is_well_defined(b, d, dt, dx, dims, tol=1e-9):
            return 1e3
        return norm(b, d, dt, dx, N, dims, wkind, wparam)

    def cfl(x):
        b, d, dt = unpack(x)
        _, smax = S_extremes(b, d, dx, dims)
        return 1.0 - dt * dt * smax

    def pos(x):
        b, d, _ = unpack(x)
        smin, _ = S_extremes(b, d, dx, dims)
        return smin

    best = (None, math.inf)
    for x0 in starts:
        if cfl(x0) < 0 or pos(x0) < 0:
            continue
        res = minimize(obj, np.asarray(x0, dtype=np.float64), method="SLSQP",
                       bounds=x_bounds,
                       constraints=[{"type": "ineq", "fun": cfl}, {"type": "ineq", "fun": pos}],
                       options={"maxiter": maxiter, "ftol": 1e-12})
        x = np.clip(res.x, [b[0] for b in x_bounds], [b[1] for b in x_bounds])
        if cfl(x) < -1e-9 or pos(x) < -1e-9:
            continue
        f = obj(x)
        if f < best[1]:
            best = (x, f)
    return best
