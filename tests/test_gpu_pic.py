"""GPU PIC cycle (fdtd_pic_step, fdtd_deposit_rho) against the particle oracle.

* Several cycles with extended coefficients, random fields and two mobile species: fields
  and particles element by element against ``oracle.pic`` (FP64 and FP32, with and without
  the absorbing layer), on grids that are not multiples of any tile; scattered particles
  (every lane on its own) and particles in blocks of 32 sharing a cell (the warp-shared
  gather and deposit), with a ragged last warp.
* Gauss's law D.E - rho (Eq. divE with App. A's continuity equation) stays at its initial
  value on the GPU, FP64 and FP32.
* Closed forms on the GPU path: the Boris rotation angle in a uniform B; a cold plasma
  oscillates at the plasma frequency, cycle by cycle equal to the oracle.
* The bunch workload at full size (512 x 256 x 256, absorbing layers, the launch
  configuration bench.py times): Gauss's law away from the layers, the first-cycle
  positions of sampled particles, and E after the first cycle in a sampled box against the
  oracle's Esirkepov current of every particle that reaches it.
* Edge cases: empty species, a non-finite particle (left unchanged, FDTD_ENONFINITE at
  sync), argument errors.
"""
import math

import numpy as np
import pytest

from gpu_util import admissible_theta, exact_coeffs, rounded_coeffs
from oracle import dispersion as D
from oracle import fdtd as F
from oracle import pic as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402

TD = {"f64": (torch.float64, np.float64), "f32": (torch.float32, np.float32)}


def _to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=TD[dtype][0])


def _periodic_diff(a, b, L):
    return (a - b + 0.5 * L) % L - 0.5 * L


def _case(shape_xyz, seed, dx=(1.0, 1.1, 0.9), frac=0.8):
    beta, delta = admissible_theta(seed)
    dt = frac * D.dt_max(beta, delta, dx, 3)
    fields = [0.1 * f for f in inputs.random_fields(shape_xyz, seed=seed + 1)]
    xe, ue = inputs.particles(shape_xyz, dx, 700, seed=seed + 2, u_scale=1.0)
    xi, ui = inputs.particles(shape_xyz, dx, 300, seed=seed + 3, u_scale=0.05)
    species = [(xe, ue, -0.02, -1.0), (xi, ui, 0.03, 0.01)]
    return beta, delta, list(dx), dt, fields, species


def _clustered(shape_xyz, dx, seed, ncell=37, per=32, extra=13):
    """Particles in blocks of `per` sharing one cell (the warp-uniform path of the push), in
    cell order, plus a ragged block of `extra`; momenta small enough to stay near the cell."""
    rng = np.random.default_rng(seed)
    cells = np.stack([rng.integers(0, shape_xyz[a], ncell) for a in range(3)])
    base = np.repeat(cells, per, axis=1)
    x = (base + rng.uniform(0.02, 0.98, base.shape)) * np.asarray(dx)[:, None]
    xe, _ = inputs.particles(shape_xyz, dx, extra, seed=seed + 1)
    x = np.concatenate([x, xe], axis=1)
    u = 0.3 * rng.standard_normal(x.shape)
    return x, u


@pytest.mark.parametrize("dtype,absorb,clustered", [("f64", 0, False), ("f32", 0, False),
                                                    ("f64", 3, False), ("f64", 0, True),
                                                    ("f32", 2, True)])
def test_pic_cycles_match_oracle(dtype, absorb, clustered):
    shape = (20, 13, 11)
    beta, delta, dx, dt, fields, species = _case(shape, seed=11)
    if clustered:
        xc, uc = _clustered(shape, dx, seed=12)
        species = [(xc, uc, -0.02, -1.0)] + species[1:]
    npd = TD[dtype][1]
    # the oracle starts from the values the device holds
    fields = [f.astype(npd).astype(np.float64) for f in fields]
    species = [(x.astype(npd).astype(np.float64), u.astype(npd).astype(np.float64), q, qm)
               for x, u, q, qm in species]
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, absorb_cells=absorb,
                      absorb_sigma=0.5)
    sm.set_state([_to_dev(f, dtype) for f in fields])
    sps = [S.Species(_to_dev(x, dtype), _to_dev(u, dtype), q, qm) for x, u, q, qm in species]
    steps = 4
    sm.pic_step(steps, sps)
    sm.sync()
    got = [t.cpu().numpy().astype(np.float64) for t in sm.get_state()]
    c = exact_coeffs(beta, delta, dx, dt, 3) if dtype == "f64" else \
        rounded_coeffs(beta, delta, dx, dt, 3, np.float32)
    sponge = F.sponge_factor((shape[2], shape[1], shape[0]), absorb, 0.5) if absorb else None
    st = F.State(fields[:3], fields[3:])
    ref = [P.Particles(x, u, q, qm) for x, u, q, qm in species]
    for _ in range(steps):
        P.pic_step(st, ref, c, sponge)
    want = st.E + st.B
    scale = max(np.max(np.abs(w)) for w in want)
    tol = 1e-12 if dtype == "f64" else 2e-5
    for a in range(6):
        assert np.max(np.abs(got[a] - want[a])) <= tol * scale, a
    Lbox = np.array([shape[a] * dx[a] for a in range(3)])[:, None]
    for sp, r in zip(sps, ref):
        gx = sp.x.cpu().numpy().astype(np.float64)
        gu = sp.u.cpu().numpy().astype(np.float64)
        assert np.all((gx >= 0) & (gx <= Lbox))
        ptol = 1e-12 if dtype == "f64" else 2e-5
        assert np.max(np.abs(_periodic_diff(gx, r.x, Lbox))) <= ptol * np.max(Lbox)
        assert np.max(np.abs(gu - r.u)) <= ptol * max(1.0, np.max(np.abs(r.u)))
    sm.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gauss_law_is_kept(dtype):
    shape = (40, 24, 20)
    beta, delta = admissible_theta(5)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype)
    sm.set_state([_to_dev(0.05 * f, dtype) for f in inputs.random_fields(shape, seed=6)[:3]] +
                 [None, None, None])
    xe, ue = inputs.particles(shape, dx, 20000, seed=7, u_scale=2.0)
    xi, ui = inputs.particles(shape, dx, 20000, seed=8, u_scale=0.02)
    sps = [S.Species(_to_dev(xe, dtype), _to_dev(ue, dtype), -0.01, -1.0),
           S.Species(_to_dev(xi, dtype), _to_dev(ui, dtype), 0.01, 1.0 / 1836)]

    def residual():
        rho = sm.deposit_rho(sps).double()
        return sm.divergence(L.FDTD_DIV_E) - rho, rho

    r0, rho0 = residual()
    E0 = [t.clone() for t in sm.get_state()[:3]]
    sm.pic_step(30, sps)
    sm.sync()
    r1, _ = residual()
    drift = float((r1 - r0).abs().max())
    scale = float(rho0.abs().max())
    assert drift <= (1e-11 if dtype == "f64" else 2e-4) * scale, (drift, scale)
    moved = max(float((a - b).abs().max()) for a, b in zip(sm.get_state()[:3], E0))
    assert moved > 1e-3
    sm.close()


def test_boris_rotation_in_uniform_B_on_gpu():
    """A test charge in a uniform B_z (a static solution: E stays zero) turns by exactly
    2 atan(|t|) per cycle, |u| and u_z kept (FP64)."""
    shape = (16, 16, 16)
    dx = [1.0, 1.0, 1.0]
    dt = 0.4
    sm = S.Simulation(shape, dx, dt, np.zeros((3, 3)), np.zeros(3), dims=3, dtype="f64")
    B0 = 1.7
    bz = torch.full((16, 16, 16), B0, dtype=torch.float64, device="cuda")
    sm.set_state([None, None, None, None, None, bz])
    u0 = np.array([[0.9], [0.0], [0.4]])
    sp = S.Species(_to_dev(np.array([[5.3], [7.1], [2.2]]), "f64"), _to_dev(u0, "f64"), 1e-30, 1.0)
    n = 25
    sm.pic_step(n, [sp])
    sm.sync()
    u = sp.u.cpu().numpy()[:, 0]
    g = math.sqrt(1 + 0.9 ** 2 + 0.4 ** 2)
    tau = 0.5 * 1.0 * dt * B0 / g
    assert abs(math.hypot(u[0], u[1]) - 0.9) < 1e-13 and abs(u[2] - 0.4) < 1e-14
    angle = math.atan2(u[1], u[0])
    assert abs(math.remainder(angle + 2.0 * n * math.atan(tau), 2 * math.pi)) < 1e-12
    sm.close()


def test_cold_plasma_oscillation_matches_oracle():
    """The oracle's cold-plasma case on a 32 x 2 x 2 grid (y, z invariant), 16 electrons per
    cell on a neutralising background: the E_x mode, cycle by cycle, equals the oracle's
    and oscillates at omega_p."""
    nx, ny, nz, ppc = 32, 2, 2, 16
    shape = (nx, ny, nz)
    dx = [1.0, 1.0, 1.0]
    dt, wp = 0.5, 0.25
    q = -wp ** 2 / ppc
    ncell = nx * ny * nz
    rng = np.random.default_rng(0)
    xs = (np.arange(ncell * ppc) % (nx * ppc) + 0.5) / ppc
    pos = np.stack([xs, rng.uniform(0, ny, xs.size), rng.uniform(0, nz, xs.size)])
    k = 2 * np.pi / nx
    u = np.zeros((3, xs.size))
    u[0] = 1e-3 * np.sin(k * pos[0])
    sm = S.Simulation(shape, dx, dt, np.zeros((3, 3)), np.zeros(3), dims=3, dtype="f64")
    sm.set_state([None] * 6)
    sp = S.Species(_to_dev(pos, "f64"), _to_dev(u, "f64"), q, -1.0)
    st = F.State([np.zeros((nz, ny, nx))] * 3, [np.zeros((nz, ny, nx))] * 3)
    ref = [P.Particles(pos, u, q, -1.0)]
    c = F.Coeffs(np.zeros((3, 3)), np.zeros(3), dx, dt)
    xf = np.arange(nx) + 0.5
    amp_g, amp_o = [], []
    for _ in range(120):
        sm.pic_step(1, [sp])
        P.pic_step(st, ref, c)
        ex = sm.get_state()[0].cpu().numpy()
        amp_g.append(float(np.sum(ex * np.sin(k * xf))))
        amp_o.append(float(np.sum(st.E[0] * np.sin(k * xf))))
    amp_g, amp_o = np.array(amp_g), np.array(amp_o)
    assert np.max(np.abs(amp_g - amp_o)) <= 1e-10 * np.max(np.abs(amp_o))
    t = (np.arange(amp_g.size) + 1) * dt
    zc = [t[i] - amp_g[i] * dt / (amp_g[i + 1] - amp_g[i]) for i in range(amp_g.size - 1)
          if amp_g[i] * amp_g[i + 1] < 0]
    omega = 2 * np.pi / (zc[2] - zc[0])
    assert abs(omega / wp - 1) < 0.01
    sm.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_deposit_rho_matches_oracle(dtype):
    """Charge density at the nodes (first-order shape), two species, positions anywhere in the
    box and a few outside it (wrapped), on a ragged grid."""
    shape = (20, 13, 11)
    dx = [1.0, 1.1, 0.9]
    sm = S.Simulation(shape, dx, 0.3, np.zeros((3, 3)), np.zeros(3), dims=3, dtype=dtype)
    xe, ue = inputs.particles(shape, dx, 1001, seed=41)
    xi, ui = inputs.particles(shape, dx, 333, seed=42)
    Lbox = np.array([shape[a] * dx[a] for a in range(3)])[:, None]
    xi[:, :7] += Lbox * np.array([[1], [-1], [2]])          # outside the box: wrapped first
    npd = TD[dtype][1]
    xe, xi = xe.astype(npd).astype(np.float64), xi.astype(npd).astype(np.float64)
    sps = [S.Species(_to_dev(xe, dtype), _to_dev(ue, dtype), -0.7, -1.0),
           S.Species(_to_dev(xi, dtype), _to_dev(ui, dtype), 1.3, 0.01)]
    got = sm.deposit_rho(sps).double().cpu().numpy()
    sm.sync()
    grid = (shape[2], shape[1], shape[0])
    ref = (P.deposit_rho(P.Particles(xe, ue, -0.7, -1.0), grid, dx) +
           P.deposit_rho(P.Particles(P.wrap_positions(xi, grid, dx), ui, 1.3, 0.01), grid, dx))
    tol = 1e-13 if dtype == "f64" else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    sm.close()


# ---- the bunch workload at full size ----------------------------------------------------

BUNCH_SHAPE = (512, 256, 256)
BUNCH_N = 1 << 22


def bunch_inputs():
    """The bench's PIC workload: 512 x 256 x 256, 16-cell absorbing layers, Yee-free extended
    coefficients (seeded), a gamma = 10 electron bunch of 2^22 macro-particles with
    sigma_par = 4, sigma_perp = 8 cells moving along +x, unit total charge."""
    beta, delta = admissible_theta(0)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    x, u = inputs.gaussian_bunch(BUNCH_N, (64.0, 128.0, 128.0), (4.0, 8.0), (1.0, 0.0, 0.0), 10.0,
                                 seed=21)
    return beta, delta, dx, dt, x, u, -1.0 / BUNCH_N


def test_bunch_full_size_first_cycle_and_gauss_law():
    beta, delta, dx, dt, x, u, q = bunch_inputs()
    nx, ny, nz = BUNCH_SHAPE
    sm = S.Simulation(BUNCH_SHAPE, dx, dt, beta, delta, dims=3, dtype="f32", absorb_cells=16,
                      absorb_sigma=0.5)
    sm.set_state([None] * 6)
    x32 = x.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    sp = S.Species(_to_dev(x32, "f32"), _to_dev(u32, "f32"), q, -1.0)
    sm.pic_step(1, [sp])
    sm.sync()
    # fields start at zero: the first push is free flight, x1 = x0 + dt u / gamma
    rng = np.random.default_rng(1)
    idx = rng.choice(BUNCH_N, 4096, replace=False)
    gx = sp.x[:, idx].cpu().numpy().astype(np.float64)
    want = x32[:, idx] + dt * u32[:, idx] / P.gamma(u32[:, idx])
    assert np.max(np.abs(gx - want)) <= 1e-4
    # B^{1/2} = 0, so E^1 = -dt J^{1/2}; a sampled box on the bunch's flank (tens of particles
    # per cell) against the oracle current of every particle whose window reaches it
    lo = np.array([71, 139, 125])
    box = np.array([4, 4, 4])
    near = np.all((x32 >= (lo - 3)[:, None]) & (x32 < (lo + box + 3)[:, None]), axis=0)
    x1 = x32[:, near] + dt * u32[:, near] / P.gamma(u32[:, near])
    J = P.esirkepov(x32[:, near], x1, q, (nz, ny, nx), dx, dt)
    E = sm.get_state()[:3]
    sl = (slice(lo[2], lo[2] + box[2]), slice(lo[1], lo[1] + box[1]), slice(lo[0], lo[0] + box[0]))
    for a in range(3):
        got = E[a][sl].cpu().numpy().astype(np.float64)
        ref = -dt * J[a][sl]
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(-dt * J[0][sl])), a
    # Gauss's law after a few more cycles, away from the absorbing layers (ions stay behind:
    # a fixed background of the initial electron density)
    rho_bg = -sm.deposit_rho([S.Species(_to_dev(x32, "f32"), _to_dev(u32, "f32"), q, -1.0)])
    sm.pic_step(9, [sp])
    sm.sync()
    r = (sm.divergence(L.FDTD_DIV_E) - sm.deposit_rho([sp]).double() - rho_bg.double())
    inner = r[20:-20, 20:-20, :]
    assert float(inner.abs().max()) <= 2e-4 * float(rho_bg.abs().max())
    sm.close()


# ---- edge cases -----------------------------------------------------------------------


def test_empty_species_is_a_field_step():
    shape = (16, 8, 8)
    beta, delta = admissible_theta(2)
    dx = [1.0, 1.0, 1.0]
    dt = 0.8 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=3)
    a = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    b = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    for sm in (a, b):
        sm.set_state([_to_dev(f, "f64") for f in fields])
    empty = S.Species(torch.empty((3, 0), dtype=torch.float64, device="cuda"),
                      torch.empty((3, 0), dtype=torch.float64, device="cuda"), 1.0, 1.0)
    a.pic_step(3, [empty])
    a.pic_step(2, [])
    b.step(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert float((x - y).abs().max()) <= 1e-13 * max(1.0, float(y.abs().max()))
    a.close()
    b.close()


def test_nonfinite_particle_is_reported_and_left_unchanged():
    shape = (16, 8, 8)
    sm = S.Simulation(shape, [1, 1, 1], 0.4, np.zeros((3, 3)), np.zeros(3), dims=3, dtype="f32")
    sm.set_state([None] * 6)
    x = np.array([[1.5, float("nan"), 3.5], [2.5, 2.5, 2.5], [1.0, 1.0, 1.0]])
    u = np.array([[0.1, 0.1, float("inf")], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    sp = S.Species(_to_dev(x, "f32"), _to_dev(u, "f32"), 0.1, 1.0)
    sm.pic_step(1, [sp])
    with pytest.raises(L.FdtdError) as e:
        sm.sync()
    assert e.value.status == L.FDTD_ENONFINITE
    gx = sp.x.cpu().numpy()
    assert math.isnan(gx[0, 1]) and gx[0, 2] == 3.5          # left unchanged
    assert abs(gx[0, 0] - (1.5 + 0.4 * 0.1 / math.sqrt(1.01))) < 1e-6   # the good one moved
    sm.sync()                                                  # the flag was cleared
    sm.close()


def test_argument_errors():
    sm = S.Simulation((16, 8, 8), [1, 1, 1], 0.4, np.zeros((3, 3)), np.zeros(3), dims=3, dtype="f64")
    bad = L.fdtd_species((L.C.c_void_p * 3)(0, 0, 0), (L.C.c_void_p * 3)(0, 0, 0), 5, 1.0, 1.0)
    with pytest.raises(L.FdtdError) as e:
        L.fdtd_pic_step(sm.h, 1, [bad])
    assert e.value.status == L.FDTD_EINVAL
    with pytest.raises(L.FdtdError):
        L.fdtd_pic_step(sm.h, -1, [])
    sm.close()
    te = S.Simulation((16, 8, 1), [1, 1, 1], 0.4, np.zeros((3, 3)), np.zeros(3), dims=2, dtype="f64")
    with pytest.raises(L.FdtdError) as e:
        L.fdtd_pic_step(te.h, 1, [])
    assert e.value.status == L.FDTD_EINVAL
    te.close()
