"""GPU diagnostics (fdtd_diagnostic, fdtd_divergence) against the oracle, and the
measurements they support: phase velocity from simulated plane waves (Sec. 3, 5) and the
divergence invariants of Sec. 2.1/2.2 at full size."""
import math

import numpy as np
import pytest

from gpu_util import admissible_theta, rounded_coeffs
from oracle import dispersion as D
from oracle import fdtd as F

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402


def make(shape, dtype="f64", seed=3, **kw):
    beta, delta = admissible_theta(seed)
    dx = [1.0, 1.1, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, **kw)
    fields = inputs.random_fields(shape, seed=seed + 10)
    sm.set_state([torch.from_numpy(f) for f in fields])
    return sm, F.Coeffs(beta, delta, dx, dt), fields


@pytest.mark.parametrize("shape", [(64, 16, 12), (36, 10, 7)])
def test_divergences_match_oracle(shape):
    sm, c, fields = make(shape)
    sm.step(3)
    st = [t.cpu().numpy() for t in sm.get_state()]
    for which, ref in [(L.FDTD_DIV_STAR_B, F.div_star_B(st[3:], c)), (L.FDTD_DIV_YEE_B, F.div_yee_B(st[3:], c)),
                       (L.FDTD_DIV_E, F.div_E(st[:3], c))]:
        got = sm.divergence(which).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), which
    sm.close()


def test_energy_window_and_plane_wave_match_oracle():
    shape = (64, 16, 12)
    sm, c, fields = make(shape)
    sm.step(2)
    st = [t.cpu().numpy() for t in sm.get_state()]
    nx, ny, nz = shape
    x_lo, x_len, margin = 50, 30, 2   # wraps around x
    mask = np.zeros((nz, ny, nx))
    xs = [(x_lo + i) % nx for i in range(x_len)]
    mask[margin:nz - margin, margin:ny - margin, :][:, :, xs] = 1.0
    ref_e = F.energy(F.State(st[:3], st[3:]), mask) * np.prod(c.dx)
    got_e = float(sm.energy(x_lo, x_len, margin).item())
    assert got_e == pytest.approx(ref_e, rel=1e-12)
    k = np.array([2 * math.pi * 3 / (nx * c.dx[0]), 2 * math.pi / (ny * c.dx[1]), 0.0])
    offs = inputs.OFFSETS
    for comp in range(6):
        ref = F.plane_wave_amplitude(st[comp], k, c.dx, offs[comp])
        got = sm.plane_wave(comp, k).cpu().numpy()
        scale = np.sum(np.abs(st[comp]))
        assert abs(complex(got[0], got[1]) - ref) <= 1e-12 * scale
    sm.close()


@pytest.mark.parametrize("direction,pol,lam", [((1, 0, 0), (0, 0, 1), 4), ((1, 0, 0), (0, 0, 1), 32),
                                               ((1, 1, 0), (0, 0, 1), 8), ((1, 1, 1), (1, -1, 0), 16)])
def test_measured_phase_velocity_matches_dispersion_relation_256(direction, pol, lam):
    """256^3 FP32: omega from the simulated plane wave (recurrence fit) vs Eq. dispersion_relation."""
    n = 256
    shape = (n, n, n)
    dx = [1.0, 1.0, 1.0]
    beta, delta = admissible_theta(1)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    dvec = np.array(direction, dtype=np.float64)
    m = max(1, round(n / (lam * np.linalg.norm(dvec))))
    kvec = dvec * 2 * math.pi * m / n
    fields = inputs.plane_wave(shape, kvec, pol, dx)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f32")
    sm.set_state([torch.from_numpy(f.astype(np.float32)) for f in fields])
    comp = int(np.argmax(np.abs(pol)))
    amps = []
    for _ in range(200):
        amps.append(sm.plane_wave(comp, kvec).cpu().numpy())
        sm.step(1)
    sm.close()
    a = np.array([complex(x, y) for x, y in amps])
    # a_{s+1} + a_{s-1} = 2 cos(omega dt) a_s: least squares for cos(omega dt)
    lhs = a[2:] + a[:-2]
    rhs = 2 * a[1:-1]
    cw = float(np.real(np.vdot(rhs, lhs) / np.vdot(rhs, rhs)))
    w_sim = math.acos(cw) / dt
    c32 = rounded_coeffs(beta, delta, dx, dt, 3, np.float32)
    kk = [kvec[i] * dx[i] / c32.dx[i] for i in range(3)]
    S32 = float(D.S_paper(*kk, c32.beta, c32.delta, c32.dx, 3, alpha_override=c32.alpha))
    w_ref = 2 / dt * math.asin(dt * math.sqrt(S32))
    assert abs(w_sim / w_ref - 1) < 2e-6
    # and the measured phase velocity differs from c as the closed form says
    vph = w_sim / np.linalg.norm(kvec)
    assert abs(vph - D.omega(*kvec, beta, delta, dt, dx, 3) / np.linalg.norm(kvec)) < 1e-5


def test_div_star_B_conserved_full_size_and_yee_div_B_is_not():
    """Sec. 2.1: D*.B is conserved for any coefficients; Sec. 2.2: Yee D.B only under Eq. (beta)."""
    n = 256
    shape = (n, n, n)
    beta, delta = admissible_theta(2)
    dt = 0.95 * D.dt_max(beta, delta, [1, 1, 1], 3)
    sm = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32")
    sm.set_state([torch.from_numpy(f.astype(np.float32)) for f in inputs.random_fields(shape, 4)])
    d0 = sm.divergence(L.FDTD_DIV_STAR_B)
    y0 = sm.divergence(L.FDTD_DIV_YEE_B)
    sm.step(100)
    d1 = sm.divergence(L.FDTD_DIV_STAR_B)
    y1 = sm.divergence(L.FDTD_DIV_YEE_B)
    sm.close()
    drift = float((d1 - d0).abs().max() / d0.abs().max())
    ydrift = float((y1 - y0).abs().max() / y0.abs().max())
    assert drift < 1e-4          # FP32 round-off over 100 steps
    assert ydrift > 1e-2         # the random coefficients violate Eq. (beta)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_energy_moments_match_oracle(dtype):
    shape = (64, 16, 12)
    sm, c, fields = make(shape, dtype=dtype)
    sm.step(2)
    st = [t.cpu().numpy().astype(np.float64) for t in sm.get_state()]
    for axis in range(3):
        ref = np.array(F.energy_moments(F.State(st[:3], st[3:]), axis, c.dx))
        got = sm.energy_moments(axis).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0], axis
    sm.close()


def test_packet_group_velocity_fp32_512():
    """Sec. 5: the energy centroid of a Gaussian packet (sigma 32, lambda 16) along x moves at
    the group velocity d omega / d k_x of Eq. (dispersion_relation); FP32, 512 x 8 x 8, 400
    steps, a seeded extended coefficient set at Courant 0.95.  The finite-packet bias is
    O((sigma k)^-2) times the curvature of v_g; the oracle run of the same packet measures
    2.6e-5; the bound is 5e-4."""
    nx = 512
    shape = (nx, 8, 8)
    dx = [1.0, 1.0, 1.0]
    beta, delta = admissible_theta(1)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    lam, sigma, xc = 16.0, 32.0, 160.0
    k0 = 2 * math.pi / lam
    w0 = D.omega(k0, 0.0, 0.0, beta, delta, dt, dx, 3)
    h = 1e-5
    vg = (D.omega(k0 + h, 0.0, 0.0, beta, delta, dt, dx, 3) -
          D.omega(k0 - h, 0.0, 0.0, beta, delta, dt, dx, 3)) / (2 * h)
    fields = inputs.packet_x(shape, dx, xc, sigma, lam, w0, dt)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f32")
    sm.set_state([torch.from_numpy(f.astype(np.float32)) for f in fields])
    ts, xs = [], []
    prev = None
    for s in range(0, 401, 20):
        if s:
            sm.step(20)
        W, C, Sn = (float(v) for v in sm.energy_moments(0).cpu())
        x = math.atan2(Sn, C) * nx / (2 * math.pi)
        if prev is not None:   # unwrap the periodic centroid
            x += round((prev - x) / nx) * nx
        prev = x
        ts.append(s * dt)
        xs.append(x)
    sm.close()
    v_meas = np.polyfit(ts, xs, 1)[0]
    assert abs(v_meas / vg - 1) < 5e-4
    W, C, Sn = F.energy_moments(F.State(fields[:3], fields[3:]), 0, dx)   # initial, oracle
    assert abs(xs[0] - math.atan2(Sn, C) * nx / (2 * math.pi)) < 1e-3
