"""Forward stepping on the GPU (libfdtd through the C ABI) against the FP64 oracle."""
import math

import numpy as np
import pytest

from gpu_util import admissible_theta, assert_elementwise, exact_coeffs, rel_l2, rounded_coeffs
from oracle import dispersion as D
from oracle import fdtd as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402
from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300._lib import FdtdError  # noqa: E402

NP = {"f32": np.float32, "f64": np.float64}


def run_gpu(shape, dx, dt, beta, delta, dims, dtype, fields, n, **kw):
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=dims, dtype=dtype, **kw)
    sm.set_state([torch.from_numpy(np.ascontiguousarray(f)) for f in fields])
    sm.step(n)
    out = [t.double().cpu().numpy() for t in sm.get_state()]
    sm.close()
    return out


def run_oracle(coeffs, fields, n, sponge=None, bunch=None):
    s = F.State(fields[:3], fields[3:])
    F.run(s, coeffs, n, bunch=bunch, sponge=sponge)
    return s.E + s.B


# ---------------------------------------------------------------- 2D TE, FP64 (128^2, 200 steps)

@pytest.mark.parametrize("scheme", ["yee", "min3"])
def test_te_2d_fp64_matches_oracle(scheme):
    beta = np.zeros((3, 3))
    delta = np.zeros(3)
    if scheme == "min3":
        beta[0, 1] = beta[1, 0] = -0.065
        delta[:2] = -0.065
    dx, dt, shape = [1.0, 1.0, 1.0], 0.5, (128, 128, 1)
    fields = inputs.te_pulse((128, 128), dx, (64.0, 64.0), 8.0, 16.0, dt, seed=0)
    got = run_gpu(shape, dx, dt, beta, delta, 2, "f64", fields, 200)
    ref = run_oracle(exact_coeffs(beta, delta, dx, dt, 2), fields, 200)
    assert rel_l2(got, ref) <= 1e-12
    assert_elementwise(got, ref, 1e-11, scheme)


# ---------------------------------------------------------------- 3D, several tiles + ragged

# (64, 16, 20), (128, 24, 33), (64, 8, 1) take the fused TMA kernel (nx % 64 == 0, ny % 8 == 0;
# 33 planes leave a ragged last z-chunk); the others take the reference-form kernels.
@pytest.mark.parametrize("shape", [(32, 24, 20), (36, 13, 7), (68, 34, 9), (4, 3, 2), (64, 16, 20),
                                   (128, 24, 33), (64, 8, 1)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_3d_random_fields_match_oracle(shape, dtype):
    beta, delta = admissible_theta(1)
    dx = [1.0, 0.9, 1.1]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=3)
    n = 40
    got = run_gpu(shape, dx, dt, beta, delta, 3, dtype, fields, n)
    if dtype == "f64":
        ref = run_oracle(exact_coeffs(beta, delta, dx, dt, 3), fields, n)
        assert rel_l2(got, ref) <= 1e-12
        assert_elementwise(got, ref, 1e-11, str(shape))
    else:
        fields32 = [f.astype(np.float32).astype(np.float64) for f in fields]
        ref = run_oracle(rounded_coeffs(beta, delta, dx, dt, 3, np.float32), fields32, n)
        assert rel_l2(got, ref) <= 2e-6
        # FP32 round-off after 40 steps, cell by cell
        assert_elementwise(got, ref, 1e-5, str(shape))


def test_1d_yee_courant_one_exact_on_gpu():
    nx = 64
    i = np.arange(nx)
    g = lambda idx: np.exp(-(((idx - 20 + nx / 2) % nx - nx / 2) / 4.0) ** 2)  # noqa: E731
    z = np.zeros((1, 1, nx))
    fields = [z, g(i)[None, None, :], z, z, z, g(i + 1)[None, None, :]]
    got = run_gpu((nx, 1, 1), [1, 1, 1], 1.0, np.zeros((3, 3)), np.zeros(3), 1, "f64", fields, 1000)
    assert np.max(np.abs(got[1] - g(i - 1000)[None, None, :])) < 1e-12


def test_sponge_and_bunch_match_oracle():
    shape = (32, 40, 40)
    dx = [1.0, 1.0, 1.0]
    beta, delta = admissible_theta(2)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=5, scale=0.1)
    bunch = (1.0, 0.999, 8.0, 20.0, 20.0, 2.0, 3.0)
    for dtype in ("f64", "f32"):
        sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, absorb_cells=8,
                          absorb_sigma=0.2)
        sm.set_state([torch.from_numpy(f) for f in fields])
        sm.step(25, source=S.Bunch(*bunch))
        got = [t.double().cpu().numpy() for t in sm.get_state()]
        sm.close()
        sp = F.sponge_factor((40, 40, 32), 8, 0.2)
        if dtype == "f64":
            ref = run_oracle(exact_coeffs(beta, delta, dx, dt, 3), fields, 25, sponge=sp,
                             bunch=F.Bunch(*bunch))
            assert rel_l2(got, ref) <= 1e-12
            assert_elementwise(got, ref, 1e-11, dtype)
        else:
            f32 = [f.astype(np.float32).astype(np.float64) for f in fields]
            ref = run_oracle(rounded_coeffs(beta, delta, dx, dt, 3, np.float32), f32, 25,
                             sponge=sp.astype(np.float32).astype(np.float64), bunch=F.Bunch(*bunch))
            assert rel_l2(got, ref) <= 2e-6
            assert_elementwise(got, ref, 1e-5, dtype)


def test_host_buffers_roundtrip():
    shape = (16, 8, 4)
    beta, delta = admissible_theta(3)
    dt = 0.9 * D.dt_max(beta, delta, [1, 1, 1], 3)
    fields = [torch.from_numpy(f.astype(np.float32)) for f in inputs.random_fields(shape, 1)]
    sm = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32")
    pinned = [f.pin_memory() for f in fields]
    sm.set_state_host(pinned)
    sm.step(3)
    out_h = [torch.empty_like(f).pin_memory() for f in fields]
    sm.get_state_host(out_h)
    out_d = sm.get_state()
    for a, b in zip(out_h, out_d):
        assert torch.equal(a, b.cpu())
    sm.close()


@pytest.mark.parametrize("dtype,shape", [("f32", (64, 16, 12)), ("f64", (64, 16, 12)),
                                          ("f32", (20, 12, 6)), ("f32", (68, 9, 5)),
                                          ("f64", (4, 1, 2))])
def test_host_upload_equals_device_upload(dtype, shape):
    """A state uploaded from pinned host memory (owned cells copied straight into the padded
    arrays, then the periodic images filled) steps bitwise like the same state uploaded from
    device memory, on fused and reference-form grids; the downloads agree bitwise too."""
    beta, delta = admissible_theta(5)
    dt = 0.9 * D.dt_max(beta, delta, [1, 1, 1], 3)
    np_t = np.float32 if dtype == "f32" else np.float64
    fields = [torch.from_numpy(f.astype(np_t)) for f in inputs.random_fields(shape, 9)]
    outs = []
    for host in (True, False):
        sm = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype=dtype)
        if host:
            sm.set_state_host([f.pin_memory() for f in fields])
        else:
            sm.set_state(fields)
        sm.step(4)
        if host:
            out = [torch.empty_like(f).pin_memory() for f in fields]
            sm.get_state_host(out)
        else:
            out = [t.cpu() for t in sm.get_state()]
        outs.append(out)
        sm.close()
    for c, (a, b) in enumerate(zip(*outs)):
        assert torch.equal(a, b), f"component {c}"


def test_checkpoint_restore_is_bitwise():
    shape = (16, 12, 8)
    beta, delta = admissible_theta(4)
    dt = 0.9 * D.dt_max(beta, delta, [1, 1, 1], 3)
    sm = S.Simulation(shape, [1, 1, 1], dt, beta, delta, dims=3, dtype="f32")
    sm.set_state([torch.from_numpy(f) for f in inputs.random_fields(shape, 2)])
    sm.step(5)
    sm.checkpoint_save(0)
    sm.step(7)
    a = sm.get_state()
    sm.checkpoint_restore(0)
    assert sm.step_index == 5
    sm.step(7)
    b = sm.get_state()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    sm.close()


def test_unstable_dt_rejected():
    beta, delta = admissible_theta(5)
    dtm = D.dt_max(beta, delta, [1, 1, 1], 3)
    with pytest.raises(FdtdError) as ei:
        S.Simulation((8, 8, 8), [1, 1, 1], 1.001 * dtm, beta, delta)
    assert "constraints" in str(ei.value)
    with pytest.raises(FdtdError):
        S.Simulation((6, 8, 8), [1, 1, 1], 0.5 * dtm, beta, delta)   # nx % 4 != 0


def test_dt_max_matches_oracle():
    for seed in range(5):
        for dims in (1, 2, 3):
            beta, delta = inputs.random_theta(seed, dims)
            dx = [1.0, 1.3, 0.7]
            got = S.dt_max(beta, delta, dx, dims)
            smin, smax = D.S_extremes(beta, delta, dx, dims)
            assert got[2] == pytest.approx(smax, rel=1e-13)
            assert got[1] == pytest.approx(smin, rel=1e-12, abs=1e-14)


# ---------------------------------------------------------------- full size (256^3, 1000 steps)

def closed_form_plane_wave(shape, dx, dt, coeffs, kvec, pol, n):
    """Exact discrete solution for E^0 = pol cos(k.r) (transverse), B^{-1/2} = 0:
    E^m = a_m E^0 with a_0 = 1, a_1 = 1 - 4 dt^2 S, a_{m+1} = 2 (1 - 2 dt^2 S) a_m - a_{m-1};
    B^{m-1/2} = dt (F E^0) sum_{l<m} a_l."""
    theta = [kvec[a] * dx[a] for a in range(3)]
    kk = [theta[a] / coeffs.dx[a] for a in range(3)]
    Sv = float(D.S_paper(*kk, coeffs.beta, coeffs.delta, coeffs.dx, 3, alpha_override=coeffs.alpha))
    c = 1.0 - 2.0 * dt * dt * Sv
    a_prev, a = 1.0, 1.0 - 4.0 * dt * dt * Sv
    acc = 1.0  # sum_{l<1} a_l
    for m in range(1, n):
        acc += a
        a_prev, a = a, 2 * c * a - a_prev
    E0 = inputs.plane_wave(shape, kvec, pol, dx)[:3]
    FE = F.faraday_rhs(E0, coeffs)
    return [a * e for e in E0] + [dt * acc * f for f in FE], a


# Config 2: 256^3, three seeded coefficient sets, lambda in {4, 8, 16, 32} cells along x,
# (1, 1, 0) and (1, 1, 1), Courant 0.95 of each scheme's limit, 1000 steps.  The bound (1e-5
# relative L2) is against the oracle's closed-form discrete solution on the FP32-rounded
# multipliers the kernels use (pure arithmetic round-off); the error against the exact
# coefficients, which also contains the coefficient quantisation, is printed beside it.
PW_DIRS = {"x": ((1, 0, 0), (0, 0, 1)), "xy": ((1, 1, 0), (0, 0, 1)), "xyz": ((1, 1, 1), (1, -1, 0))}
PW_CASES = ([(s, lam, d) for s in (0, 1, 2) for lam in (4, 8, 16, 32) for d in ("x", "xyz")] +
            [(0, lam, "xy") for lam in (4, 8, 16, 32)])


@pytest.mark.parametrize("seed,lam,dname", PW_CASES)
def test_full_size_plane_wave_fp32_1000_steps(seed, lam, dname):
    n_cells = 256
    shape = (n_cells, n_cells, n_cells)
    dx = [1.0, 1.0, 1.0]
    direction, pol = PW_DIRS[dname]
    beta, delta = admissible_theta(seed)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    dvec = np.array(direction, dtype=np.float64)
    m = max(1, round(n_cells / (lam * np.linalg.norm(dvec))))
    kvec = dvec * 2 * math.pi * m / n_cells
    fields = inputs.plane_wave(shape, kvec, pol, dx)
    got = run_gpu(shape, dx, dt, beta, delta, 3, "f32", [f.astype(np.float32) for f in fields], 1000)
    ref, _ = closed_form_plane_wave(shape, dx, dt, rounded_coeffs(beta, delta, dx, dt, 3, np.float32),
                                    kvec, pol, 1000)
    err = rel_l2(got, ref)
    del ref
    ref_x, _ = closed_form_plane_wave(shape, dx, dt, exact_coeffs(beta, delta, dx, dt, 3), kvec, pol,
                                      1000)
    err_x = rel_l2(got, ref_x)
    lam_real = 2 * math.pi / np.linalg.norm(kvec)
    print(f"\nplane-wave accuracy seed={seed} lambda={lam} (realised {lam_real:.3f}) dir={dname}: "
          f"rel L2 vs rounded-multiplier oracle {err:.2e}, vs exact-coefficient oracle {err_x:.2e}")
    assert err <= 1e-5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(64, 16, 20), (128, 8, 3), (64, 8, 1)])
def test_fused_kernel_bitwise_equals_reference_form(dtype, shape, monkeypatch):
    """The fused TMA step and the reference-form kernels share their arithmetic: equal bits."""
    beta, delta = admissible_theta(7)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=8)
    kw = dict(absorb_cells=2, absorb_sigma=0.2) if shape[2] >= 4 else {}
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("FDTD_FUSED", flag)
        sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, **kw)
        sm.set_state([torch.from_numpy(f) for f in fields])
        sm.step(7, source=S.Bunch(1.0, 0.9, 10.0, 4.0, 1.0, 2.0, 2.0))
        sm.sync()
        outs.append(sm.get_state())
        sm.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


# The FP32 step kernel keeps each thread's own rows in tensor memory in slots that rotate with
# the plane index inside a z-chunk; the chunk length depends on the grid (whole waves of resident
# CTAs).  These shapes give single-plane grids, one- and two-plane chunks, ragged last chunks,
# chunks of 16-64 planes and launches of one to several waves.
@pytest.mark.parametrize("shape", [(64, 8, 2), (64, 8, 3), (192, 24, 5), (128, 40, 17),
                                   (256, 16, 38), (64, 64, 75), (256, 64, 64)])
def test_fused_fp32_tmem_kernel_bitwise_equals_reference_form(shape, monkeypatch):
    beta, delta = admissible_theta(11)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=23)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("FDTD_FUSED", flag)
        sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f32")
        sm.set_state([torch.from_numpy(f) for f in fields])
        sm.step(5)
        sm.sync()
        outs.append(sm.get_state())
        sm.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("dtype,shape", [("f64", (64, 32, 4)), ("f32", (64, 32, 5)), ("f64", (36, 10, 3))])
def test_batched_2d_equals_independent_runs(dtype, shape):
    """batched = 1: the nz planes are independent 2D problems (z multipliers are zero)."""
    nx, ny, nz = shape
    beta = np.zeros((3, 3))
    beta[0, 1], beta[1, 0] = 0.02, 0.03
    delta = np.array([-0.03, -0.05, 0.0])
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 2)
    fields = inputs.random_fields(shape, seed=9)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=2, dtype=dtype, batched=True,
                      absorb_cells=3, absorb_sigma=0.2)
    sm.set_state([torch.from_numpy(f) for f in fields])
    sm.step(30)
    got = [t.double().cpu().numpy() for t in sm.get_state()]
    sm.close()
    np_t = NP[dtype]
    c = exact_coeffs(beta, delta, dx, dt, 2) if dtype == "f64" else \
        rounded_coeffs(beta, delta, dx, dt, 2, np_t)
    # the sponge acts on +-y only: the z axis is the batch axis
    sp = F.sponge_profile(ny, 3, 0.2)[None, :, None] * np.ones((1, ny, nx))
    if dtype == "f32":
        sp = sp.astype(np.float32).astype(np.float64)
    for k in range(nz):
        f_k = [f[k:k + 1].astype(np_t).astype(np.float64) for f in fields]
        ref = run_oracle(c, f_k, 30, sponge=sp)
        err = rel_l2([g[k:k + 1] for g in got], ref)
        assert err <= (1e-12 if dtype == "f64" else 2e-6), (k, err)
        assert_elementwise([g[k:k + 1] for g in got], ref, 1e-11 if dtype == "f64" else 1e-5, f"member {k}")


def test_expired_wait_reports_timeout_and_handle_stays_usable():
    """Failure path without a fault: a bounded mbarrier wait that runs out raises the handle's
    error flag; fdtd_sync reports FDTD_ETIMEOUT once, and the handle keeps stepping correctly."""
    shape = (64, 16, 12)
    beta, delta = admissible_theta(4)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, 7)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    sm.set_state([torch.from_numpy(f) for f in fields])
    with pytest.raises(L.FdtdError):
        L.fdtd_selftest_wait_expiry(sm.h, 0)          # argument checked on the host
    L.fdtd_selftest_wait_expiry(sm.h, 512)
    with pytest.raises(L.FdtdError) as ei:
        sm.sync()
    assert ei.value.status == L.FDTD_ETIMEOUT
    sm.sync()                                         # reported once, then cleared
    sm.step(3)
    got = [t.cpu().numpy() for t in sm.get_state()]
    sm.close()
    st = F.run(F.State(fields[:3], fields[3:]), F.Coeffs(beta, delta, dx, dt), 3)
    for g, r in zip(got, st.E + st.B):
        assert np.max(np.abs(g - r)) <= 1e-12 * max(1.0, np.max(np.abs(r)))


# (64, 16, 12) takes the fused kernels (FP32 and FP64), (36, 13, 7) the reference-form ones
@pytest.mark.parametrize("dtype,shape", [("f32", (64, 16, 12)), ("f64", (64, 16, 12)),
                                         ("f32", (36, 13, 7)), ("f64", (36, 13, 7))])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_field_is_reported(dtype, shape, bad):
    """A non-finite value in the fields (what a blow-up leaves) is detected by the step kernels
    as they write E: the next fdtd_sync returns FDTD_ENONFINITE once and clears the flag; the
    handle then steps a finite state correctly."""
    beta, delta = admissible_theta(4)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, 13)
    broken = [f.copy() for f in fields]
    broken[4][shape[2] // 2, 5, 7] = bad          # one B_y value
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype)
    sm.set_state([torch.from_numpy(f) for f in broken])
    sm.step(2)
    with pytest.raises(FdtdError) as ei:
        sm.sync()
    assert ei.value.status == L.FDTD_ENONFINITE
    assert "non-finite" in str(ei.value)
    sm.sync()                                     # reported once, then cleared
    sm.set_state([torch.from_numpy(f) for f in fields])
    sm.step(3)
    sm.sync()
    got = [t.double().cpu().numpy() for t in sm.get_state()]
    sm.close()
    if dtype == "f64":
        ref = run_oracle(exact_coeffs(beta, delta, dx, dt, 3), fields, 3)
        assert_elementwise(got, ref, 1e-12)
    else:
        f32 = [f.astype(np.float32).astype(np.float64) for f in fields]
        ref = run_oracle(rounded_coeffs(beta, delta, dx, dt, 3, np.float32), f32, 3)
        assert_elementwise(got, ref, 1e-5)


# slab lengths: (64, 8, 20) / 4 -> 5 slabs; (128, 16, 33) / 5 -> 6 slabs of 5-6 planes;
# (64, 16, 9) / 3 -> 3 slabs; (64, 8, 8) / 4 -> 2 slabs; 256^3 / 32 -> the bench's 8 slabs
@pytest.mark.parametrize("shape,slab,sponge", [((64, 8, 20), 4, False), ((128, 16, 33), 5, True),
                                               ((64, 16, 9), 3, False), ((64, 8, 8), 4, True),
                                               ((256, 256, 256), 32, False)])
@pytest.mark.parametrize("n", [4, 5])
def test_temporal_blocking_bitwise_equals_single_steps(shape, slab, sponge, n):
    """Temporally blocked pairs (slab-interleaved through L2, intermediate planes discarded from
    L2) give the same bits as one launch per step; an odd last step runs unblocked."""
    if shape[2] == 256 and n == 5:
        pytest.skip("one full-size case suffices")
    beta, delta = admissible_theta(3)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    fields = [torch.from_numpy(f.astype(np.float32)) for f in inputs.random_fields(shape, 17)]
    kw = dict(absorb_cells=2, absorb_sigma=0.2) if sponge else {}
    outs = []
    for T in (1, 2):
        sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f32", **kw)
        sm.set_temporal_blocking(T, slab)
        sm.set_state(fields)
        sm.step(n)
        sm.step(2)      # a second call continues from the blocked result
        sm.sync()
        assert sm.step_index == n + 2
        outs.append(sm.get_state())
        sm.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_temporal_blocking_arguments():
    sm = S.Simulation((64, 8, 8), [1, 1, 1], 0.3, np.zeros((3, 3)), np.zeros(3), dims=3, dtype="f32")
    for T, slab in ((3, 0), (2, 2), (0, 0), (2, -1)):
        with pytest.raises(FdtdError):
            sm.set_temporal_blocking(T, slab)
    sm.set_temporal_blocking(2, 0)
    sm.close()
