"""Pins of the dispersion-norm oracle against what the paper and the mathematics fix.

* Table 1 norms, Table 3 phase-velocity extremes, Table 2 ordering and the
  Fig. 3 value are the paper's printed numbers (tests/golden, cited there).
* The printed dispersion relation (Sec. 3) and the reduced App. B form are two
  different formulas; they must agree.
* The exact CFL limit is checked by brute force, the midpoint norm by explicit
  loops and by adaptive quadrature, the gradient by central differences.
* The SLSQP minimiser reproduces min.1 - min.4 of Table 1.
"""
import math

import numpy as np
import pytest

from oracle import dispersion as D

DX1 = [1.0, 1.0, 1.0]


def co2(b, dxx, dyy):
    beta = np.zeros((3, 3))
    beta[0, 1] = beta[1, 0] = b
    return beta, np.array([dxx, dyy, 0.0])


def rand_coeffs(rng, dims=3):
    beta = rng.uniform(-0.125, 0.125, (3, 3))
    delta = rng.uniform(-0.125, 0.0, 3)
    return D.clean_coeffs(beta, delta, dims)


def printed_match(value, printed_str, rel=0.05):
    """Equal at the printed precision, or within `rel` relative."""
    p = float(printed_str)
    if "e" in printed_str.lower():
        mant = printed_str.lower().split("e")[0]
        dec = len(mant.split(".")[1]) if "." in mant else 0
        half = 0.5 * 10 ** (-dec) * 10 ** int(printed_str.lower().split("e")[1])
    else:
        dec = len(printed_str.split(".")[1]) if "." in printed_str else 0
        half = 0.5 * 10 ** (-dec)
    return abs(value - p) <= half * (1 + 1e-9) or abs(value - p) <= rel * abs(p)


# ---------------------------------------------------------------- closed forms

def test_alpha_normalisation():
    beta = np.array([[0, 0.1, 0.02], [0.03, 0, -0.05], [0.07, 0.01, 0]])
    delta = np.array([-0.02, -0.04, 0.01])
    a = D.alpha(beta, delta, 3)
    assert a[0] == pytest.approx(1 - 2 * (0.1 + 0.02) - 3 * (-0.02))
    assert a[1] == pytest.approx(1 - 2 * (0.03 - 0.05) - 3 * (-0.04))
    assert a[2] == pytest.approx(1 - 2 * (0.07 + 0.01) - 3 * 0.01)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("dims", [2, 3])
def test_printed_and_reduced_forms_agree(seed, dims):
    """Sec. 3 dispersion relation vs App. B reduced form (sign-corrected) on random k, coefficients, dx."""
    rng = np.random.default_rng(seed)
    beta, delta = rand_coeffs(rng, dims)
    dx = rng.uniform(0.5, 2.0, 3)
    k = [rng.uniform(0, math.pi / dx[i], 200) if i < dims else np.zeros(200) for i in range(3)]
    a = D.S_paper(*k, beta, delta, dx, dims)
    b = D.S_reduced(*k, beta, delta, dx, dims)
    assert np.max(np.abs(a - b)) <= 1e-14 * max(1.0, np.max(np.abs(a)))


def test_reduced_form_printed_sign_is_a_typo():
    """With the '+' of App. B's last line, NDFX (beta = 1/8) could not run at c dt = dx.

    The paper states it does (Sec. 5, Table 1).  With the corrected '-' the
    maximum of S is exactly 1 at the zone corner, so dt_max = dx/c.
    """
    beta, delta = co2(0.125, 0, 0)
    S_corner = D.S_reduced(math.pi, math.pi, 0.0, beta, delta, DX1, 2)
    assert S_corner == pytest.approx(1.0, abs=1e-15)
    s2 = 1.0
    printed_sign = s2 + s2 + 4 * 2 * 0.125 * s2 * s2
    assert printed_sign > 1.5
    assert D.dt_max(beta, delta, DX1, 2) == pytest.approx(1.0, abs=1e-14)


def test_yee_limit_dispersion():
    """beta = delta = 0 gives alpha = 1 and the Yee relation s_w^2 = sum s_i^2 (Sec. 3)."""
    rng = np.random.default_rng(5)
    dx = rng.uniform(0.5, 2, 3)
    k = [rng.uniform(0, math.pi / dx[i], 100) for i in range(3)]
    S = D.S_paper(*k, np.zeros((3, 3)), np.zeros(3), dx, 3)
    yee = sum(np.sin(k[i] * dx[i] / 2) ** 2 / dx[i] ** 2 for i in range(3))
    assert np.allclose(S, yee, rtol=0, atol=1e-15)
    assert D.dt_max(np.zeros((3, 3)), np.zeros(3), dx, 3) == pytest.approx(
        1 / math.sqrt(sum(1 / dx ** 2)), rel=1e-14)


def test_1d_yee_is_dispersion_free_at_courant_one():
    """Sec. 3: in 1D the Yee scheme with c dt = dx has omega = c k exactly."""
    k = np.linspace(0.01, math.pi, 50)
    w = D.omega(k, 0 * k, 0 * k, np.zeros((3, 3)), np.zeros(3), 1.0, DX1, 1)
    assert np.max(np.abs(w - k)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("dims", [2, 3])
def test_exact_S_extremes_vs_bruteforce(seed, dims):
    rng = np.random.default_rng(100 + seed)
    beta, delta = rand_coeffs(rng, dims)
    dx = rng.uniform(0.5, 2.0, 3)
    smin, smax = D.S_extremes(beta, delta, dx, dims)
    n = 129 if dims == 3 else 1025
    ax = [np.linspace(0, math.pi / dx[i], n) if i < dims else np.zeros(1) for i in range(3)]
    KZ, KY, KX = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    S = D.S_paper(KX, KY, KZ, beta, delta, dx, dims)
    # the exact extremes bound the grid values and are approached by them
    assert S.max() <= smax * (1 + 1e-12) + 1e-15
    assert S.min() >= smin - 1e-12
    scale = max(1 / dx[i] ** 2 for i in range(dims))
    assert smax - S.max() <= 2e-3 * scale
    assert S.min() - smin <= 2e-3 * scale


# ---------------------------------------------------------------- the norm

@pytest.mark.parametrize("dims,N", [(2, (4, 4, 1)), (2, (8, 6, 1)), (3, (4, 3, 5))])
@pytest.mark.parametrize("wkind,wparam", [(D.WEIGHT_UNIFORM, 0.0), (D.WEIGHT_CONE_X, math.radians(30)),
                                          (D.WEIGHT_GAUSS_Y, 0.1)])
def test_norm_matches_bruteforce_loops(dims, N, wkind, wparam):
    rng = np.random.default_rng(7)
    beta, delta = rand_coeffs(rng, dims)
    dx = np.array([1.0, 1.3, 0.8])
    dt = 0.9 * D.dt_max(beta, delta, dx, dims)
    a = D.norm(beta, delta, dt, dx, N, dims, wkind, wparam)
    b = D.norm_bruteforce(beta, delta, dt, dx, N, dims, wkind, wparam)
    assert a == pytest.approx(b, rel=1e-13, abs=1e-300)


def test_norm_converges_to_adaptive_quadrature_2d():
    """Midpoint rule -> the integral of Eq. (norm) (scipy dblquad), Yee at 0.95/sqrt(2)."""
    from scipy.integrate import dblquad

    beta, delta = co2(0, 0, 0)
    dt = 0.95 / math.sqrt(2)

    def integrand(ky, kx):
        S = math.sin(kx / 2) ** 2 + math.sin(ky / 2) ** 2
        w = 2 / dt * math.asin(dt * math.sqrt(S))
        return (w - math.hypot(kx, ky)) ** 2

    ref, _ = dblquad(integrand, 0, math.pi, 0, math.pi, epsabs=1e-11, epsrel=1e-11)
    f256 = D.norm(beta, delta, dt, DX1, (256, 256, 1), 2)
    f64 = D.norm(beta, delta, dt, DX1, (64, 64, 1), 2)
    assert abs(f256 - ref) < abs(f64 - ref)
    assert f256 == pytest.approx(ref, rel=2e-4)


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("wkind,wparam", [(D.WEIGHT_UNIFORM, 0.0), (D.WEIGHT_CONE_X, math.radians(30))])
def test_norm_gradient_vs_central_differences(dims, wkind, wparam):
    rng = np.random.default_rng(11)
    beta, delta = rand_coeffs(rng, dims)
    dx = np.array([1.0, 1.2, 0.9])
    dt = 0.8 * D.dt_max(beta, delta, dx, dims)
    N = (24, 20, 16)
    f, gb, gd, gdt = D.norm_and_grad(beta, delta, dt, dx, N, dims, wkind, wparam)
    assert f == pytest.approx(D.norm(beta, delta, dt, dx, N, dims, wkind, wparam), rel=1e-14)
    h = 1e-6

    def fd(fun):
        return (fun(h) - fun(-h)) / (2 * h)

    for i in range(dims):
        for j in range(dims):
            if i == j:
                continue

            def fb(e, i=i, j=j):
                b = beta.copy()
                b[i, j] += e
                return D.norm(b, delta, dt, dx, N, dims, wkind, wparam)
            assert gb[i, j] == pytest.approx(fd(fb), rel=1e-6, abs=1e-9)

        def fdl(e, i=i):
            d = delta.copy()
            d[i] += e
            return D.norm(beta, d, dt, dx, N, dims, wkind, wparam)
        assert gd[i] == pytest.approx(fd(fdl), rel=1e-6, abs=1e-9)
    assert gdt == pytest.approx(fd(lambda e: D.norm(beta, delta, dt + e, dx, N, dims, wkind, wparam)),
                                rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- printed numbers

def test_table1_uniform_norms(golden):
    for name, nu, b, dxx, dyy, printed in golden("table1_uniform_norms.txt"):
        beta, delta = co2(float(b), float(dxx), float(dyy))
        f = D.norm(beta, delta, float(nu), DX1, (512, 512, 1), 2)
        assert printed_match(f, printed), (name, f, printed)
        assert D.is_well_defined(beta, delta, float(nu), DX1, 2, tol=5e-3), name


def test_table3_phase_velocity_extremes(golden):
    t1 = {r[0]: r for r in golden("table1_uniform_norms.txt")}
    for name, vmin, vmax in golden("table3_phase_velocity.txt"):
        _, nu, b, dxx, dyy, _ = t1[name]
        beta, delta = co2(float(b), float(dxx), float(dyy))
        lo, hi = D.phase_velocity_extremes(beta, delta, float(nu), DX1, 512, 2)
        assert abs(lo - float(vmin)) <= 0.015, (name, lo, vmin)
        assert abs(hi - float(vmax)) <= 0.015, (name, hi, vmax)


def test_table2_xaxis_weight_ordering(golden):
    """Table 2: only the ordering is pinned for all rows (Lehe and min.5 differ ~10x
    from the printed values under every reading tried); Yee and NDFX also by value."""
    vals = {}
    for name, nu, b, dxx, dyy, printed in golden("table2_xaxis_weight.txt"):
        beta, delta = co2(float(b), float(dxx), float(dyy))
        vals[name] = (D.norm(beta, delta, float(nu), DX1, (1024, 1024, 1), 2, D.WEIGHT_GAUSS_Y, 0.1),
                      float(printed))
    assert vals["min5"][0] < vals["Lehe"][0] < vals["Yee"][0]
    assert vals["NDFX"][0] < vals["min6"][0] < vals["Cowan"][0]
    assert vals["Yee"][0] == pytest.approx(vals["Yee"][1], rel=0.12)
    assert vals["NDFX"][0] == pytest.approx(vals["NDFX"][1], rel=0.05)


def test_fig3_aspect_ratio_yee(golden):
    (dxs, dys, frac, printed), = golden("fig3_aspect_ratio.txt")
    dx = [float(dxs), float(dys), 1.0]
    beta, delta = co2(0, 0, 0)
    dt = float(frac) * D.dt_max(beta, delta, dx, 2)
    f = D.norm(beta, delta, dt, dx, (512, 512, 1), 2)
    assert f == pytest.approx(float(printed), rel=0.01)


# ---------------------------------------------------------------- the minimiser

def _eqbeta_unpack(nu):
    def up(x):
        beta, delta = co2(x[0], x[0], x[0])
        return beta, delta, nu
    return up


@pytest.mark.parametrize("name", ["min2", "min3", "min4"])
def test_minimiser_reproduces_eqbeta_schemes(golden, name):
    """min.2-4: Eq. (beta) with delta_x = delta_y, fixed c dt/dx; one free parameter."""
    row = {r[0]: r for r in golden("table1_uniform_norms.txt")}[name]
    nu, printed_delta, printed_f = float(row[1]), float(row[3]), row[5]
    x, f = D.minimise(_eqbeta_unpack(nu), [(-0.125, 0.125)], [[-0.1], [0.0], [0.1]],
                      DX1, (256, 256, 1), 2)
    assert abs(x[0] - printed_delta) <= 0.002, (name, x)
    assert printed_match(f, printed_f), (name, f)


@pytest.mark.slow
def test_minimiser_reproduces_min1(golden):
    """min.1: beta_xy = beta_yx, delta_x = delta_y and dt free (3 parameters)."""
    row = {r[0]: r for r in golden("table1_uniform_norms.txt")}["min1"]

    def up(x):
        beta, delta = co2(x[0], x[1], x[1])
        return beta, delta, x[2]
    starts = [[b, d, n] for b in (-0.1, 0.05, 0.2) for d in (-0.1, 0.1) for n in (0.3, 0.8)]
    x, f = D.minimise(up, [(-0.125, 0.25), (-0.125, 0.125), (0.05, 1.0)], starts, DX1, (256, 256, 1), 2)
    assert abs(x[0] - float(row[2])) <= 0.002
    assert abs(x[1] - float(row[3])) <= 0.002
    assert abs(x[2] - float(row[1])) <= 0.002
    assert printed_match(f, row[5])


def _co2(bxy, byx, dx_, dy_):
    b = np.zeros((3, 3))
    b[0, 1], b[1, 0] = bxy, byx
    return b, np.array([dx_, dy_, 0.0])


def test_minimiser_reproduces_ndfx_with_dt_at_dx_over_c():
    """Sec. 5 (reproducing published stencils): with c dt = dx as the lower bound of the time step
    (so c dt = dx), the minimum of Eq. (norm) is Pukhov's NDFX scheme, beta = 1/8, delta = 0,
    from several feasible starts."""
    def up(x):
        b, d = _co2(x[0], x[0], x[1], x[1])
        return b, d, x[2]
    bounds = [(-0.125, 0.25), (-0.125, 0.125), (1.0, 1.0)]
    for start in ([0.0625, 0.0625, 1.0], [0.2, 0.0, 1.0], [0.15, 0.02, 1.0]):
        x, f = D.minimise(up, bounds, [start], [1, 1, 1], (64, 64, 1), 2)
        assert abs(x[0] - 0.125) <= 0.002 and abs(x[1]) <= 0.002, (start, x)


def test_minimiser_reproduces_lehe_with_delta_y_pinned_at_zero():
    """Sec. 5: delta_y held at zero and c dt / dx = 0.96 (read as the time step pinned at the bound;
    with a free lower bound the minimum moves to c dt / dx ~ 0.68) give Lehe's scheme,
    beta = 1/8 and delta_x = -0.021 (Table 1)."""
    def up(x):
        b, d = _co2(x[0], x[0], x[1], x[2])
        return b, d, x[3]
    bounds = [(-0.125, 0.25), (-0.125, 0.125), (-1e-6, 1e-6), (0.96, 0.96)]
    starts = [[b, d, 0.0, 0.96] for b in (0.0, 0.1, 0.2) for d in (-0.1, 0.0)]
    x, f = D.minimise(up, bounds, starts, [1, 1, 1], (64, 64, 1), 2)
    assert abs(x[0] - 0.125) <= 0.002 and abs(x[1] + 0.021) <= 0.002, x


# ---------------------------------------------------------------- group-velocity norm

def _rand_set(seed, dims=3):
    rng = np.random.default_rng(seed)
    b = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            if i != j:
                b[i, j] = rng.uniform(-0.06, 0.06)
    d = rng.uniform(-0.08, 0.0, 3)
    return b, d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_group_speed_matches_central_differences(seed):
    """|d omega/dk| from the analytic grad_k S equals central differences of omega(k)."""
    b, d = _rand_set(seed)
    dx = [1.0, 1.1, 0.9]
    dt = 0.8 * D.dt_max(b, d, dx, 3)
    rng = np.random.default_rng(seed + 10)
    for _ in range(5):
        k = rng.uniform(0.05, 2.6, 3)
        t = D.group_speed_terms(*(np.array(v) for v in k), b, d, dt, dx, 3)
        assert float(t["vg"]) == pytest.approx(np.linalg.norm(D.group_velocity(k, b, d, dt, dx, 3)),
                                               rel=1e-8)


def test_group_norm_vanishes_for_1d_yee_at_courant_one():
    """1D Yee with c dt = dx propagates every wavenumber at exactly c: v_g = 1, f_g = 0."""
    b, d = np.zeros((3, 3)), np.zeros(3)
    f, gb, gd, gdt = D.group_norm_and_grad(b, d, 1.0, [1.0, 1.0, 1.0], (256, 1, 1), 1)
    assert f < 1e-24


def test_group_norm_yee_2d_closed_form():
    """Yee in 2D: |v_g|^2 = (sin^2(kx dx)/(4 dx^2) + sin^2(ky dy)/(4 dy^2)) / (S (1 - dt^2 S)),
    S = sin^2(kx dx/2)/dx^2 + sin^2(ky dy/2)/dy^2, summed here independently."""
    dx = [1.0, 0.7, 1.0]
    dt = 0.9 / math.sqrt(1 / dx[0] ** 2 + 1 / dx[1] ** 2)
    N = (40, 30, 1)
    tot = 0.0
    for my in range(N[1]):
        for mx in range(N[0]):
            kx = (mx + 0.5) * math.pi / (N[0] * dx[0])
            ky = (my + 0.5) * math.pi / (N[1] * dx[1])
            S = math.sin(kx * dx[0] / 2) ** 2 / dx[0] ** 2 + math.sin(ky * dx[1] / 2) ** 2 / dx[1] ** 2
            g2 = math.sin(kx * dx[0]) ** 2 / (4 * dx[0] ** 2) + math.sin(ky * dx[1]) ** 2 / (4 * dx[1] ** 2)
            tot += (math.sqrt(g2 / (S * (1 - dt * dt * S))) - 1.0) ** 2
    ref = tot * (math.pi / N[0]) * (math.pi / N[1])
    f, *_ = D.group_norm_and_grad(np.zeros((3, 3)), np.zeros(3), dt, dx, N, 2)
    assert f == pytest.approx(ref, rel=1e-12)


def test_group_norm_matches_difference_quotient_loops():
    b, d = _rand_set(3)
    dx = [1.0, 1.1, 0.9]
    dt = 0.8 * D.dt_max(b, d, dx, 3)
    f, *_ = D.group_norm_and_grad(b, d, dt, dx, (6, 5, 4), 3)
    assert f == pytest.approx(D.group_norm_fd(b, d, dt, dx, (6, 5, 4), 3), rel=1e-7)


@pytest.mark.parametrize("dims,wkind,wparam", [(3, D.WEIGHT_UNIFORM, 0.0), (2, D.WEIGHT_CONE_X, 0.6),
                                               (2, D.WEIGHT_GAUSS_Y, 0.3)])
def test_group_norm_gradient_vs_central_differences(dims, wkind, wparam):
    b, d = _rand_set(4)
    b, d = D.clean_coeffs(b, d, dims)
    dx = [1.0, 1.1, 0.9]
    dt = 0.8 * D.dt_max(b, d, dx, dims)
    N = (12, 10, 8)
    f, gb, gd, gdt = D.group_norm_and_grad(b, d, dt, dx, N, dims, wkind, wparam)
    h = 1e-6

    def F(bb, dd, tt):
        return D.group_norm_and_grad(bb, dd, tt, dx, N, dims, wkind, wparam)[0]
    for i in range(dims):
        for j in range(dims):
            if i != j:
                bp, bm = b.copy(), b.copy()
                bp[i, j] += h
                bm[i, j] -= h
                assert gb[i, j] == pytest.approx((F(bp, d, dt) - F(bm, d, dt)) / (2 * h), rel=1e-6, abs=1e-9)
        dp, dm = d.copy(), d.copy()
        dp[i] += h
        dm[i] -= h
        assert gd[i] == pytest.approx((F(b, dp, dt) - F(b, dm, dt)) / (2 * h), rel=1e-6, abs=1e-9)
    assert gdt == pytest.approx((F(b, d, dt + h) - F(b, d, dt - h)) / (2 * h), rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- the cone weight (Sec. 4)
# Sec. 4 weights the norm by a function that is non-zero only inside a cone of directions; the
# oracle reads it as w = 1 where k_x >= |k| cos(theta) (a cone of half-angle theta about +x).
# These pins check that reading against closed-form volumes and moments of the cone inside the
# positive octant [0, pi]^dims, and the weighted norm against a quadrature in cone-adapted
# coordinates that never evaluates the weight function.  For tan(theta) <= 1 the cone's cross
# section at k_x is a quarter disk (3D) or a segment (2D) of radius k_x tan(theta) <= pi, which
# stays inside the box.


def _cone_sums(N, dims, theta, wfun=None):
    """Midpoint sums of w, w k_x, w k_y over the box, with the oracle's grid and weight."""
    wfun = wfun or (lambda KX, KY, KZ: D.weight(KX, KY, KZ, D.WEIGHT_CONE_X, theta, np.ones(3)))
    KX, KY, KZ, vol = D.midpoint_grid(N, np.ones(3), dims)
    w = wfun(KX, KY, KZ)
    return w.sum() * vol, (w * KX).sum() * vol, (w * KY).sum() * vol


def _cone_closed_forms(dims, theta):
    """Volume, first moment along x and along y of the cone inside the box."""
    t = math.tan(theta)
    pi = math.pi
    if dims == 3:
        # quarter disk of radius R = k_x t: area pi R^2 / 4, moment of k_y = R^3 / 3
        return pi / 4 * t * t * pi ** 3 / 3, pi / 4 * t * t * pi ** 4 / 4, t ** 3 / 3 * pi ** 4 / 4
    # segment 0 <= k_y <= k_x t: length R, moment of k_y = R^2 / 2
    return t * pi ** 2 / 2, t * pi ** 3 / 3, t * t * pi ** 3 / 6


@pytest.mark.parametrize("dims,N,tol", [(2, (512, 512, 1), 1e-4), (3, (96, 96, 96), 5e-4)])
@pytest.mark.parametrize("deg", [30.0, 20.0])
def test_cone_weight_volume_and_moments_closed_form(dims, N, tol, deg):
    th = math.radians(deg)
    got = _cone_sums(N, dims, th)
    ref = _cone_closed_forms(dims, th)
    for g, r in zip(got, ref):
        assert g == pytest.approx(r, rel=tol)
    # the midpoint sums converge to the closed forms
    coarse = _cone_sums(tuple(max(1, n // 4) for n in N), dims, th)
    assert abs(got[0] - ref[0]) <= abs(coarse[0] - ref[0]) + 1e-12


def _gauss_cone(f, theta, dims, n=64):
    """Integral of f(kx, ky, kz) over the cone inside the box, by Gauss-Legendre in cone
    coordinates: k_x in [0, pi]; 3D: k_y = r cos(phi), k_z = r sin(phi), r in [0, k_x t],
    phi in [0, pi/2] (Jacobian r); 2D: k_y in [0, k_x t]."""
    x, wq = np.polynomial.legendre.leggauss(n)
    t = math.tan(theta)
    kx = 0.5 * math.pi * (x + 1)
    wkx = 0.5 * math.pi * wq
    if dims == 2:
        KX = kx[:, None]
        R = KX * t
        KY = 0.5 * R * (x[None, :] + 1)
        W = wkx[:, None] * 0.5 * R * wq[None, :]
        return float(np.sum(W * f(KX, KY, 0.0 * KX)))
    KX = kx[:, None, None]
    R = KX * t
    r = 0.5 * R * (x[None, :, None] + 1)
    phi = 0.25 * math.pi * (x[None, None, :] + 1)
    W = wkx[:, None, None] * (0.5 * R * wq[None, :, None]) * (0.25 * math.pi * wq[None, None, :]) * r
    return float(np.sum(W * f(KX, r * np.cos(phi), r * np.sin(phi))))


@pytest.mark.parametrize("dims,N,tol", [(2, (1024, 1024, 1), 2e-4), (3, (128, 128, 128), 2e-3)])
def test_cone_weighted_norm_matches_cone_quadrature(dims, N, tol):
    """Eq. (norm) with the cone weight, on an anisotropic coefficient set (so the cone's axis
    matters), against the same integral taken only over the cone."""
    th = math.radians(30.0)
    beta = np.zeros((3, 3))
    delta = np.zeros(3)
    beta[0, 1], beta[1, 0], delta[0], delta[1] = 0.11, -0.02, -0.09, -0.03
    if dims == 3:
        beta[0, 2], beta[2, 0], beta[1, 2], beta[2, 1], delta[2] = 0.05, 0.07, -0.04, 0.01, -0.06
    dx = np.ones(3)
    dt = 0.9 * D.dt_max(beta, delta, dx, dims)

    def integrand(kx, ky, kz):
        S = D.S_paper(kx, ky, kz, beta, delta, dx, dims)
        return (D.omega_from_S(S, dt) - np.sqrt(kx * kx + ky * ky + kz * kz)) ** 2

    ref = _gauss_cone(integrand, th, dims)
    assert ref == pytest.approx(_gauss_cone(integrand, th, dims, n=96), rel=1e-10)
    got = D.norm(beta, delta, dt, dx, N, dims, D.WEIGHT_CONE_X, th)
    assert got == pytest.approx(ref, rel=tol)
    # the same scheme weighted by a cone about +y gives a different value (the axis is pinned)
    def swapped(kx, ky, kz):
        return integrand(ky, kx, kz)
    assert abs(_gauss_cone(swapped, th, dims) / ref - 1) > 20 * tol


@pytest.mark.parametrize("mistake", ["axis_y", "sin_for_cos", "degrees", "strict_complement"])
def test_cone_pins_catch_planted_mistakes(mistake):
    """Plausible misreadings of the cone weight each fail the closed-form pins above."""
    th = math.radians(30.0)

    def wrong(KX, KY, KZ):
        kn = np.sqrt(KX * KX + KY * KY + KZ * KZ)
        if mistake == "axis_y":
            return (KY >= kn * math.cos(th)).astype(np.float64)
        if mistake == "sin_for_cos":
            return (KX >= kn * math.sin(th)).astype(np.float64)
        if mistake == "degrees":
            return (KX >= kn * math.cos(30.0)).astype(np.float64)
        return (KX < kn * math.cos(th)).astype(np.float64)

    for dims, N in [(2, (256, 256, 1)), (3, (48, 48, 48))]:
        got = _cone_sums(N, dims, th, wrong)
        ref = _cone_closed_forms(dims, th)
        assert max(abs(g / r - 1) for g, r in zip(got, ref)) > 0.05, (dims, mistake)
