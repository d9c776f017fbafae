"""Pins of the particle-coupling oracle against what the paper and the mathematics fix.

* Gather: first-order interpolation reproduces fields linear in position exactly, at every
  component's own staggered positions (a half-cell slip of any offset fails).
* Boris push: in a uniform B the momentum turns by exactly 2 atan(|t|) per step about B with
  |u| and u.B kept (the scheme's closed form); in a uniform E, u grows by q/m dt E exactly.
* Esirkepov current: the discrete continuity equation (App. A) holds to rounding for random
  moves in every direction; each particle's current integrates to q dx/dt; a move along x on
  the nodes of y and z gives the textbook one-dimensional face currents.
* The PIC cycle keeps D.E - rho at its initial value (Sec. 2, Eq. divE with App. A), for
  extended coefficients, two mobile species and a non-zero initial field; a cold plasma
  oscillates at the plasma frequency (a sign error anywhere in gather, push, current or
  Ampere law turns the oscillation into growth or shifts it).
"""
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import fdtd as F
from oracle import pic as P


def _interior_points(rng, n, shape, dx, margin=1.5):
    nz, ny, nx = shape
    lo = margin
    return np.stack([rng.uniform(lo, nx - 1 - lo, n) * dx[0], rng.uniform(lo, ny - 1 - lo, n) * dx[1],
                     rng.uniform(lo, nz - 1 - lo, n) * dx[2]])


@pytest.mark.parametrize("comp", range(6))
def test_gather_reproduces_linear_fields(comp):
    rng = np.random.default_rng(3)
    shape = (9, 10, 12)
    dx = np.array([0.7, 1.1, 0.9])
    off = (P.E_OFFSETS + P.B_OFFSETS)[comp]
    k, j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    # the component's staggered positions, written out here: ((i + ox) dx, (j + oy) dy, (k + oz) dz)
    X, Y, Z = (i + off[0]) * dx[0], (j + off[1]) * dx[1], (k + off[2]) * dx[2]
    f = lambda x, y, z: 0.3 + 1.7 * x - 0.6 * y + 0.25 * z
    Fc = f(X, Y, Z)
    x = _interior_points(rng, 200, shape, dx)
    got = P.gather(Fc, off, x, dx)
    assert np.max(np.abs(got - f(x[0], x[1], x[2]))) < 1e-12


def test_boris_uniform_B_rotates_by_the_closed_form_angle():
    qm, dt, B0 = -1.0, 0.4, 2.5
    u = np.array([[0.8], [0.0], [0.3]])
    E = np.zeros((3, 1))
    B = np.array([[0.0], [0.0], [B0]])
    g = math.sqrt(1 + 0.8 ** 2 + 0.3 ** 2)
    tau = 0.5 * qm * dt * B0 / g
    n = 37
    for _ in range(n):
        u = P.boris(u, E, B, qm, dt)
    assert abs(math.hypot(u[0, 0], u[1, 0]) - 0.8) < 1e-13
    assert abs(u[2, 0] - 0.3) < 1e-14
    # u -> u + 2 u x t to first order: for t along +z the rotation is clockwise
    angle = math.atan2(u[1, 0], u[0, 0])
    expect = -2.0 * n * math.atan(tau)
    assert abs(math.remainder(angle - expect, 2 * math.pi)) < 1e-12


def test_boris_uniform_E_kicks_by_q_over_m_dt_E():
    rng = np.random.default_rng(4)
    u = rng.standard_normal((3, 50))
    E = rng.standard_normal((3, 50))
    qm, dt = 0.7, 0.3
    u1 = P.boris(u, E, np.zeros((3, 50)), qm, dt)
    assert np.max(np.abs(u1 - (u + qm * dt * E))) < 1e-14


def _random_moves(rng, n, shape, dx):
    nz, ny, nx = shape
    x0 = np.stack([rng.uniform(0, nx * dx[0], n), rng.uniform(0, ny * dx[1], n),
                   rng.uniform(0, nz * dx[2], n)])
    d = rng.uniform(-0.99, 0.99, (3, n)) * np.asarray(dx)[:, None]
    return x0, x0 + d


def test_esirkepov_satisfies_discrete_continuity():
    """(rho^{n+1} - rho^n)/dt + D.J^{n+1/2} = 0 (App. A) for moves in every direction,
    across the periodic seams."""
    rng = np.random.default_rng(5)
    shape = (8, 9, 10)
    dx = np.array([1.0, 0.8, 1.3])
    dt = 0.37
    x0, x1 = _random_moves(rng, 400, shape, dx)
    q = 0.9
    J = P.esirkepov(x0, x1, q, shape, dx, dt)
    r0 = P.deposit_rho(P.Particles(x0, np.zeros_like(x0), q, 1.0), shape, dx)
    r1 = P.deposit_rho(P.Particles(P.wrap_positions(x1, shape, dx), np.zeros_like(x0), q, 1.0),
                       shape, dx)
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), dx, dt)
    res = (r1 - r0) / dt + F.div_E(J, c)
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(r0)) / dt
    # and the charge itself is conserved by the shape
    vol = dx.prod()
    assert abs(r1.sum() * vol - 400 * q) < 1e-10


def test_esirkepov_current_integrates_to_q_velocity():
    rng = np.random.default_rng(6)
    shape = (6, 7, 8)
    dx = np.array([0.9, 1.0, 1.2])
    dt = 0.5
    vol = dx.prod()
    for _ in range(20):
        x0, x1 = _random_moves(rng, 1, shape, dx)
        J = P.esirkepov(x0, x1, -1.3, shape, dx, dt)
        for a in range(3):
            assert abs(J[a].sum() * vol - (-1.3) * (x1[a, 0] - x0[a, 0]) / dt) < 1e-12


def test_esirkepov_one_dimensional_face_currents():
    """A move along x with y, z on nodes: the current through face i+1/2 is q/(dt dy dz)
    times the drop of the charge fraction on the nodes at or left of i."""
    shape = (5, 6, 12)
    dx = np.array([1.0, 1.0, 1.0])
    dt, q = 0.5, 2.0
    # from grid coordinate 4.3 (cell 4) to 5.6 (cell 5): crosses node 5
    x0 = np.array([[4.3], [2.0], [3.0]])
    x1 = np.array([[5.6], [2.0], [3.0]])
    J = P.esirkepov(x0, x1, q, shape, dx, dt)
    expect = np.zeros(shape)
    expect[3, 2, 4] = q * (5.0 - 4.3) / dt     # face 4.5: fraction left drops from 0.7 to 0
    expect[3, 2, 5] = q * (5.6 - 5.0) / dt     # face 5.5: from 1 to 0.4
    assert np.max(np.abs(J[0] - expect)) < 1e-14
    assert np.max(np.abs(J[1])) == 0.0 and np.max(np.abs(J[2])) == 0.0


def _stable(rng):
    while True:
        beta = rng.uniform(-0.1, 0.1, (3, 3))
        np.fill_diagonal(beta, 0.0)
        delta = rng.uniform(-0.04, 0.02, 3)
        dx = np.array([1.0, 1.1, 0.9])
        try:
            dtm = D.dt_max(beta, delta, dx, 3)
        except Exception:
            continue
        if np.isfinite(dtm) and dtm > 0.2:
            return beta, delta, dx, 0.6 * dtm


def test_pic_cycle_conserves_gauss_law():
    rng = np.random.default_rng(7)
    shape = (6, 7, 8)
    beta, delta, dx, dt = _stable(rng)
    c = F.Coeffs(beta, delta, dx, dt)
    s = F.State([0.1 * rng.standard_normal(shape) for _ in range(3)],
                [np.zeros(shape) for _ in range(3)])
    nz, ny, nx = shape
    L = np.array([nx * dx[0], ny * dx[1], nz * dx[2]])[:, None]
    ne = 300
    elec = P.Particles(rng.uniform(0, 1, (3, ne)) * L, rng.standard_normal((3, ne)), -0.05, -1.0)
    ions = P.Particles(rng.uniform(0, 1, (3, ne)) * L, 0.1 * rng.standard_normal((3, ne)), 0.05, 0.02)

    def gauss(st, sp):
        return F.div_E(st.E, c) - sum(P.deposit_rho(p, shape, dx) for p in sp)

    g0 = gauss(s, [elec, ions])
    E0 = [e.copy() for e in s.E]
    for _ in range(12):
        P.pic_step(s, [elec, ions], c)
    g1 = gauss(s, [elec, ions])
    assert np.max(np.abs(g1 - g0)) < 1e-12 * (1.0 + np.max(np.abs(g0)))
    # the charges moved the field (the check is not vacuous)
    assert max(np.max(np.abs(s.E[a] - E0[a])) for a in range(3)) > 1e-3


def test_cold_plasma_oscillates_at_the_plasma_frequency():
    """Uniform electrons (16 per cell) on a fixed neutralising background, a small velocity
    perturbation at the longest wavelength: the field mode oscillates at omega_p (within the
    first-order-shape and leapfrog corrections, below 1 % at k dx = 2 pi / 32)."""
    nx, ppc = 32, 16
    shape = (1, 1, nx)
    dx = np.array([1.0, 1.0, 1.0])
    dt = 0.5
    wp = 0.25
    q = -wp ** 2 / ppc            # n q^2 / m = wp^2 with q/m = -1, n = ppc per unit volume
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), dx, dt)
    xs = (np.arange(nx * ppc) + 0.5) / ppc
    k = 2 * np.pi / nx
    u = np.zeros((3, xs.size))
    u[0] = 1e-3 * np.sin(k * xs)
    elec = P.Particles(np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)]), u, q, -1.0)
    s = F.State([np.zeros(shape) for _ in range(3)], [np.zeros(shape) for _ in range(3)])
    rho_bg = -P.deposit_rho(elec, shape, dx)      # neutralising background: rho_total = 0, E = 0
    xf = np.arange(nx) + 0.5                       # E_x positions
    amp = []
    for _ in range(130):
        P.pic_step(s, [elec], c)
        amp.append(float(np.sum(s.E[0][0, 0] * np.sin(k * xf))))
    amp = np.array(amp)
    t = (np.arange(amp.size) + 1) * dt
    zc = [t[i] - amp[i] * dt / (amp[i + 1] - amp[i]) for i in range(amp.size - 1)
          if amp[i] == 0 or amp[i] * amp[i + 1] < 0]
    assert len(zc) >= 3
    omega = 2 * np.pi / (zc[2] - zc[0])
    assert abs(omega / wp - 1) < 0.01, omega
    # bounded: the amplitude neither grows nor decays over two periods
    half = amp.size // 2
    assert 0.9 < np.max(np.abs(amp[half:])) / np.max(np.abs(amp[:half])) < 1.1
    # Gauss's law with the background
    res = F.div_E(s.E, c) - P.deposit_rho(elec, shape, dx) - rho_bg
    assert np.max(np.abs(res)) < 1e-13


def _one_particle_step(E, B, x, u, c, qm=-1.0):
    s = F.State(E, B)
    p = P.Particles(x, u, 1e-30, qm)      # a test charge: its own current is negligible
    P.pic_step(s, [p], c)
    return p


def _rotate(v, axis, theta):
    """Rodrigues' rotation of v about the unit vector axis by theta."""
    return (v * math.cos(theta) + np.cross(axis, v) * math.sin(theta)
            + axis * np.dot(axis, v) * (1 - math.cos(theta)))


def test_push_kicks_with_E_at_the_E_positions():
    """E = (a x, b y, c z) has no curl away from the periodic seam, so B stays zero at the
    particle and the push is the exact kick q/m dt E(x_p)."""
    shape = (10, 11, 12)
    dx = np.array([0.9, 1.0, 1.1])
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), dx, 0.3)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    E = [0.7 * (i + 0.5) * dx[0], -0.4 * (j + 0.5) * dx[1], 0.2 * (k + 0.5) * dx[2]]
    B = [np.zeros(shape) for _ in range(3)]
    x = np.array([[5.3], [4.9], [6.2]])
    u = np.array([[0.2], [-0.1], [0.4]])
    p = _one_particle_step(E, B, x, u, c)
    kick = -1.0 * c.dt * np.array([0.7 * x[0, 0], -0.4 * x[1, 0], 0.2 * x[2, 0]])
    assert np.max(np.abs(p.u[:, 0] - (u[:, 0] + kick))) < 1e-13
    g = math.sqrt(1 + np.sum(p.u ** 2))
    assert np.max(np.abs(p.x[:, 0] - (x[:, 0] + c.dt * p.u[:, 0] / g))) < 1e-13


def test_push_rotates_about_B_at_the_B_positions():
    """E = 0 keeps B fixed; each B component linear in position is read at its own staggered
    positions; the momentum turns about B(x_p) by 2 atan(|t|), t = q/m dt B / (2 gamma)."""
    shape = (10, 11, 12)
    dx = np.array([1.0, 0.9, 1.2])
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), dx, 0.35)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    lin = lambda x, y, z, a: [0.3 + 0.1 * x - 0.05 * z, -0.2 + 0.07 * y + 0.02 * x,
                              0.5 - 0.04 * z + 0.03 * y][a]
    B = []
    for a, off in enumerate(P.B_OFFSETS):
        B.append(lin((i + off[0]) * dx[0], (j + off[1]) * dx[1], (k + off[2]) * dx[2], a))
    E = [np.zeros(shape) for _ in range(3)]
    x = np.array([[4.4], [5.1], [6.7]])
    u = np.array([[1.2], [-0.5], [0.8]])
    p = _one_particle_step(E, B, x, u, c, qm=-1.0)
    Bp = np.array([lin(x[0, 0], x[1, 0], x[2, 0], a) for a in range(3)])
    g = math.sqrt(1 + np.sum(u ** 2))
    t = 0.5 * (-1.0) * c.dt * Bp / g
    tn = np.linalg.norm(t)
    expect = _rotate(u[:, 0], t / tn, -2 * math.atan(tn))
    assert np.max(np.abs(p.u[:, 0] - expect)) < 1e-13


def test_push_uses_time_centred_B():
    """B^{n-1/2} = -B^{n+1/2} (a standing wave at its magnetic node in time): B at the
    integer level vanishes and a fast particle gets the pure electric kick, no rotation."""
    shape = (8, 8, 16)
    dx = np.array([1.0, 1.0, 1.0])
    rng = np.random.default_rng(8)
    beta, delta = np.zeros((3, 3)), np.zeros(3)
    beta[0, 1] = beta[0, 2] = 0.1
    c = F.Coeffs(beta, delta, dx, 0.4)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    E = [np.zeros(shape), 0.8 * np.cos(2 * np.pi * i / 16) + 0.1 * rng.standard_normal(shape),
         np.zeros(shape)]
    f = F.faraday_rhs(E, c)
    B = [-0.5 * c.dt * f[a] for a in range(3)]
    x = np.array([[7.3], [3.6], [4.2]])
    u = np.array([[3.0], [0.5], [-0.4]])
    p = _one_particle_step(E, B, x, u, c)
    Ey = P.gather(E[1], P.E_OFFSETS[1], x, dx)[0]
    assert np.max(np.abs(p.u[:, 0] - (u[:, 0] + np.array([0.0, -c.dt * Ey, 0.0])))) < 1e-13
    # with B^{n+1/2} alone the rotation would be visible
    assert np.max(np.abs(B[2])) * c.dt * 3.0 > 1e-3


def test_boris_is_kick_rotate_kick():
    """Uniform E and B together: half kick, a rotation by 2 atan(|t|) about t = q/m dt B /
    (2 gamma^-) with gamma^- taken after the first half kick, half kick (Rodrigues' form)."""
    rng = np.random.default_rng(9)
    qm, dt = -1.0, 0.45
    for _ in range(10):
        u, E, B = (rng.standard_normal(3) * s for s in (2.0, 1.0, 1.5))
        h = 0.5 * qm * dt
        um = u + h * E
        t = h * B / math.sqrt(1 + um @ um)
        tn = np.linalg.norm(t)
        expect = _rotate(um, t / tn, -2 * math.atan(tn)) + h * E
        got = P.boris(u[:, None], E[:, None], B[:, None], qm, dt)[:, 0]
        assert np.max(np.abs(got - expect)) < 1e-13
