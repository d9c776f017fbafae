"""Pins of the FDTD oracle against what the paper and the mathematics fix.

* Plane waves advance with the closed-form numerical dispersion relation
  (Sec. 3): for transverse E and any coefficients, the projected amplitudes
  obey a_{n+1} + a_{n-1} = 2 cos(omega dt) a_n exactly.
* 1D Yee at c dt = dx shifts a pulse by one cell per step (Sec. 3).
* D*.B is conserved for any coefficients (Sec. 2.1); Yee D.B only under
  Eq. (beta) (Sec. 2.2) -- with a negative case.
* Discrete continuity (App. A): with the rigid-bunch current,
  D.E^n = rho^n - rho^0 when E^0 = 0.
* The adjoint is the transpose (dot-product test) and its coefficient
  gradient matches central differences of the forward map.
"""
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import fdtd as F


def rand_state(rng, shape):
    return F.State([rng.standard_normal(shape) for _ in range(3)],
                   [rng.standard_normal(shape) for _ in range(3)])


def stable_coeffs(rng, dims=3):
    while True:
        beta = rng.uniform(-0.125, 0.125, (3, 3))
        delta = rng.uniform(-0.125, 0.0, 3)
        beta, delta = D.clean_coeffs(beta, delta, dims)
        smin, _ = D.S_extremes(beta, delta, [1, 1, 1], dims)
        if smin >= 0:
            return beta, delta


# ---------------------------------------------------------------- dispersion

def _positions(shape, comp, dx):
    nz, ny, nx = shape
    off = [[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5]][comp]
    z, y, x = np.meshgrid((np.arange(nz) + off[2]) * dx[2], (np.arange(ny) + off[1]) * dx[1],
                          (np.arange(nx) + off[0]) * dx[0], indexing="ij")
    return x, y, z


@pytest.mark.parametrize("direction,pol", [((1, 0, 0), (0, 0, 1)), ((1, 1, 0), (0, 0, 1)),
                                           ((1, 1, 1), (1, -1, 0)), ((0, 1, 0), (1, 0, 0))])
@pytest.mark.parametrize("seed", [0, 1])
def test_plane_wave_follows_dispersion_relation(direction, pol, seed):
    rng = np.random.default_rng(seed)
    beta, delta = stable_coeffs(rng)
    shape = (8, 8, 8)
    dx = np.array([1.0, 1.0, 1.0])
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    c = F.Coeffs(beta, delta, dx, dt)
    m = 2
    k = np.array(direction, dtype=np.float64) * 2 * math.pi * m / shape[2]
    E = []
    for a in range(3):
        x, y, z = _positions(shape, a, dx)
        E.append(pol[a] * np.cos(k[0] * x + k[1] * y + k[2] * z))
    s = F.State(E, [np.zeros(shape)] * 3)
    comp = int(np.argmax(np.abs(pol)))
    amps = [F.plane_wave_amplitude(s.E[comp], k, dx)]
    for _ in range(40):
        F.step(s, c)
        amps.append(F.plane_wave_amplitude(s.E[comp], k, dx))
    a = np.array(amps)
    w = D.omega(*k, beta, delta, dt, dx, 3)
    resid = a[2:] + a[:-2] - 2 * math.cos(w * dt) * a[1:-1]
    assert np.max(np.abs(resid)) <= 1e-11 * np.max(np.abs(a))
    # and a wrong frequency is detected
    resid_bad = a[2:] + a[:-2] - 2 * math.cos(1.001 * w * dt) * a[1:-1]
    assert np.max(np.abs(resid_bad)) > 1e-6 * np.max(np.abs(a))


def test_yee_1d_courant_one_is_exact_shift():
    nx = 64
    shape = (1, 1, nx)
    i = np.arange(nx)
    g = lambda idx: np.exp(-(((idx - 20 + nx / 2) % nx - nx / 2) / 4.0) ** 2)  # noqa: E731
    Ey = g(i)[None, None, :]
    Bz = g(i + 1)[None, None, :]  # B_z at (i+1/2), time -1/2: right-moving wave
    z = np.zeros(shape)
    s = F.State([z, Ey, z], [z, z, Bz])
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), [1, 1, 1], 1.0)
    F.run(s, c, 1000)
    expect = g(i - 1000)[None, None, :]
    assert np.max(np.abs(s.E[1] - expect)) < 1e-12
    # with delta_x != 0 the same run is dispersive
    s2 = F.State([z, Ey, z], [z, z, Bz])
    d = np.array([-0.05, 0, 0])
    c2 = F.Coeffs(np.zeros((3, 3)), d, [1, 1, 1], 0.99 * D.dt_max(np.zeros((3, 3)), d, [1, 1, 1], 1))
    F.run(s2, c2, 200)
    assert np.max(np.abs(s2.E[1] - g(i - 200)[None, None, :])) > 1e-3


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_div_star_B_conserved_any_coefficients(seed):
    rng = np.random.default_rng(seed)
    beta, delta = stable_coeffs(rng)
    shape = (6, 7, 8)
    dx = rng.uniform(0.7, 1.3, 3)
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    c = F.Coeffs(beta, delta, dx, dt)
    s = rand_state(rng, shape)
    d0 = F.div_star_B(s.B, c)
    F.run(s, c, 20)
    d1 = F.div_star_B(s.B, c)
    assert np.max(np.abs(d1 - d0)) < 1e-11 * np.max(np.abs(d0))


def test_yee_div_B_conserved_iff_eq_beta():
    rng = np.random.default_rng(4)
    shape = (6, 7, 8)
    dx = [1.0, 1.0, 1.0]
    # Eq. (beta): beta_ij = delta_j
    delta = np.array([-0.03, -0.05, -0.02])
    beta = np.array([[0, delta[1], delta[2]], [delta[0], 0, delta[2]], [delta[0], delta[1], 0]])
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    c = F.Coeffs(beta, delta, dx, dt)
    s = rand_state(rng, shape)
    d0 = F.div_yee_B(s.B, c)
    F.run(s, c, 20)
    assert np.max(np.abs(F.div_yee_B(s.B, c) - d0)) < 1e-11 * np.max(np.abs(d0))
    # min.1-like coefficients violate Eq. (beta): Yee D.B drifts
    beta2 = np.zeros((3, 3))
    beta2[0, 1] = beta2[1, 0] = 0.11
    delta2 = np.array([-0.125, -0.125, 0.0])
    c2 = F.Coeffs(beta2, delta2, dx, 0.9 * D.dt_max(beta2, delta2, dx, 2))
    s2 = rand_state(rng, shape)
    e0 = F.div_yee_B(s2.B, c2)
    F.run(s2, c2, 20)
    assert np.max(np.abs(F.div_yee_B(s2.B, c2) - e0)) > 1e-2 * np.max(np.abs(e0))


def test_continuity_with_rigid_bunch():
    shape = (12, 12, 32)
    dx = np.array([1.0, 1.0, 1.0])
    beta, delta = stable_coeffs(np.random.default_rng(9))
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    c = F.Coeffs(beta, delta, dx, dt)
    b = F.Bunch(q=1.0, v=0.999, x0=8.0, y0=6.0, z0=6.0, sig_par=2.0, sig_perp=2.5)
    z = np.zeros(shape)
    s = F.State([z, z, z], [z, z, z])
    rho0 = b.rho(shape, 0, c)
    F.run(s, c, 15, bunch=b)
    lhs = F.div_E(s.E, c)
    rhs = b.rho(shape, 15, c) - rho0
    assert np.max(np.abs(rhs)) > 1e-3
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs)) + 1e-14


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("sponge", [False, True])
def test_adjoint_dot_product(sponge):
    rng = np.random.default_rng(21)
    shape = (20, 20, 8) if sponge else (5, 6, 7)
    beta, delta = stable_coeffs(rng)
    dx = rng.uniform(0.8, 1.2, 3)
    c = F.Coeffs(beta, delta, dx, 0.9 * D.dt_max(beta, delta, dx, 3))
    sp = F.sponge_factor(shape, 4, 0.3) if sponge else None
    u, v = rand_state(rng, shape), rand_state(rng, shape)
    Mu = F.step(u.copy(), c, None, sp)
    lam = F.adjoint_step(v.copy(), u.E, c, {}, sp)
    lhs, rhs = np.dot(Mu.flat(), v.flat()), np.dot(u.flat(), lam.flat())
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_adjoint_gradient_vs_central_differences():
    rng = np.random.default_rng(22)
    shape = (5, 6, 7)
    beta, delta = stable_coeffs(rng)
    dx = np.array([1.0, 1.1, 0.9])
    dt = 0.8 * D.dt_max(beta, delta, dx, 3)
    u, v = rand_state(rng, shape), rand_state(rng, shape)
    n = 4

    def loss(b, d):
        s = u.copy()
        F.run(s, F.Coeffs(b, d, dx, dt), n)
        return float(np.dot(s.flat(), v.flat()))

    c = F.Coeffs(beta, delta, dx, dt)
    states = [u.copy()]
    for _ in range(n):
        states.append(F.step(states[-1].copy(), c))
    lam, g = v.copy(), {}
    for m in range(n - 1, -1, -1):
        F.adjoint_step(lam, states[m].E, c, g)
    gb, gd = F.grad_to_arrays(g)
    h = 1e-5
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            bp, bm = beta.copy(), beta.copy()
            bp[i, j] += h
            bm[i, j] -= h
            fd = (loss(bp, delta) - loss(bm, delta)) / (2 * h)
            assert gb[i, j] == pytest.approx(fd, rel=1e-7, abs=1e-7)
        dp, dm = delta.copy(), delta.copy()
        dp[i] += h
        dm[i] -= h
        fd = (loss(beta, dp) - loss(beta, dm)) / (2 * h)
        assert gd[i] == pytest.approx(fd, rel=1e-7, abs=1e-7)


def _centroid(m, n):
    W, C, S = m
    return (math.atan2(S, C) * n / (2 * math.pi)) % n


def test_energy_moments_pins():
    """Packet centroid moments (Sec. 5 group velocity measurement): a single excited cell sits at
    its component's staggered position (App. A), W is the field energy, and translating the
    fields by m cells moves the centroid by exactly m (mod n)."""
    nz, ny, nx = 3, 4, 40
    dx = [1.0, 1.0, 1.0]
    # E_y at i = 10 is not staggered along x; E_x and B_z are (offset 1/2); B_x is not
    for comp, want in [(1, 10.0), (0, 10.5), (5, 10.5), (3, 10.0)]:
        f = [np.zeros((nz, ny, nx)) for _ in range(6)]
        f[comp][1, 2, 10] = 3.0
        st = F.State(f[:3], f[3:])
        m = F.energy_moments(st, 0, dx)
        assert m[0] == pytest.approx(4.5)
        assert _centroid(m, nx) == pytest.approx(want, abs=1e-12)
    # along y: B_x is staggered along y, E_y too, E_x is not
    f = [np.zeros((nz, ny, nx)) for _ in range(6)]
    f[3][0, 1, 5] = 1.0
    assert _centroid(F.energy_moments(F.State(f[:3], f[3:]), 1, dx), ny) == pytest.approx(1.5)
    rng = np.random.default_rng(3)
    f = [rng.standard_normal((nz, ny, nx)) for _ in range(6)]
    st = F.State(f[:3], f[3:])
    m0 = F.energy_moments(st, 0, [0.5, 2.0, 1.0])
    assert m0[0] == pytest.approx(F.energy(st) * 1.0, rel=1e-12)
    for shift in (1, 7, 39):
        g = [np.roll(a, shift, axis=2) for a in f]
        m = F.energy_moments(F.State(g[:3], g[3:]), 0, [0.5, 2.0, 1.0])
        d = (_centroid(m, nx) - _centroid(m0, nx)) % nx
        assert d == pytest.approx(shift, abs=1e-9)


def test_packet_centroid_moves_at_group_velocity():
    """Sec. 5: a Gaussian packet (sigma 32, lambda 16) on the oracle's leapfrog moves at the
    closed-form group velocity d omega / d k_x of Eq. (dispersion_relation) (a seeded extended
    coefficient set, whose v_g exceeds 1 by 1.3 %), measured by the energy centroid."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from gpu_util import admissible_theta
    from paper_1710_06829_gb300 import inputs
    beta, delta = admissible_theta(1)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    k0 = 2 * math.pi / 16
    w0 = D.omega(k0, 0.0, 0.0, beta, delta, dt, dx, 3)
    h = 1e-5
    vg = (D.omega(k0 + h, 0, 0, beta, delta, dt, dx, 3) - D.omega(k0 - h, 0, 0, beta, delta, dt, dx, 3)) / (2 * h)
    nx = 512
    f = inputs.packet_x((nx, 2, 2), dx, 160.0, 32.0, 16.0, w0, dt)
    st = F.State([a.copy() for a in f[:3]], [a.copy() for a in f[3:]])
    c = F.Coeffs(beta, delta, dx, dt)
    ts, xs, prev = [], [], None
    for s in range(0, 201, 20):
        if s:
            F.run(st, c, 20)
        x = _centroid(F.energy_moments(st, 0, dx), nx)
        if prev is not None:
            x += round((prev - x) / nx) * nx
        prev = x
        ts.append(s * dt)
        xs.append(x)
    v = np.polyfit(ts, xs, 1)[0]
    assert vg > 1.005                      # the set is superluminal at lambda = 16 ...
    assert abs(v / vg - 1) < 2e-4          # ... and the packet follows d omega / d k


@pytest.mark.parametrize("sigma", [0.3, 0.5])
@pytest.mark.parametrize("scheme", ["yee", "extended"])
def test_sponge_reflects_and_transmits_below_1e3(sigma, scheme):
    """The absorbing layer (a reading; the paper has none): a Gaussian pulse (width 8, wavelength
    16) meets a 16-cell layer at normal incidence; after 300 time units the reflected energy
    (back in the interior behind the start) and the energy that crossed both layers of the
    periodic y axis (ahead of the start) are each below 1e-3 of the initial energy."""
    ny, nx, L, dt = 400, 4, 16, 0.5
    if scheme == "yee":
        beta, delta = np.zeros((3, 3)), np.zeros(3)
    else:
        beta = np.array([[0, 0.05, 0.05], [0.05, 0, 0.02], [0.05, 0.02, 0]])
        delta = np.array([-0.03, -0.03, -0.03])
    c = F.Coeffs(beta, delta, [1, 1, 1], dt)
    y = np.arange(ny).astype(float)
    yc, w, lam = 200.0, 8.0, 16.0
    prof = lambda yy: np.exp(-((yy - yc) / w) ** 2) * np.cos(2 * np.pi * (yy - yc) / lam)
    Ex = np.repeat(prof(y)[None, :, None], nx, axis=2)
    Bz = -np.repeat(prof(y + 0.5 + 0.5 * dt)[None, :, None], nx, axis=2)   # moving along +y
    s = F.State([Ex, 0 * Ex, 0 * Ex], [0 * Ex, 0 * Ex, Bz])
    sponge = np.ones((1, ny, nx)) * F.sponge_profile(ny, L, sigma)[None, :, None]
    e0 = F.energy(s)
    for _ in range(600):
        F.step(s, c, None, sponge)
    refl = np.zeros((1, ny, nx))
    refl[:, 220:ny - L, :] = 1
    trans = np.zeros((1, ny, nx))
    trans[:, L:200, :] = 1
    assert F.energy(s, refl) / e0 < 1e-3
    assert F.energy(s, trans) / e0 < 1e-3
