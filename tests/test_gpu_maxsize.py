"""Maximum sizes and the limits of the launch shapes, against the oracle.

Every input here is invariant along y and z (one random or plane-wave row along x, repeated),
so the state stays invariant and the oracle run on the one-row grid (1, 1, nx) gives every
cell's exact expected value; the comparison covers all cells (on the device).

* nz = 70000 (above the 65535 limit of a grid's y / z extent): the reference-form forward,
  adjoint (with the coefficient gradient) and PIC field kernels, FP64.
* FP32, the largest padded arrays the fused TMA step kernel takes (just under 2^31 elements,
  its 32-bit offsets at their largest), and arrays just over 2^31 elements (the reference-form
  kernels with 64-bit offsets).  About 120 GB of device memory each; skipped when the device
  has less free.
"""
import numpy as np
import pytest

from gpu_util import admissible_theta, exact_coeffs, rounded_coeffs
from oracle import dispersion as D
from oracle import fdtd as F

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402


def _rows_to_dev(rows, shape_xyz, tdtype):
    nx, ny, nz = shape_xyz
    return [None if r is None else
            torch.from_numpy(np.ascontiguousarray(r)).to("cuda", tdtype).expand(nz, ny, nx).contiguous()
            for r in rows]


def _max_dev(got, row):
    """max |got[k, j, i] - row[i]| over the whole array, on the device."""
    r = torch.from_numpy(np.ascontiguousarray(row.reshape(-1))).to("cuda", torch.float64)
    return float((got.double() - r).abs().max())


def test_nz_beyond_the_grid_extent_limit_fp64():
    shape = (36, 7, 70000)   # not a multiple of the TMA tiles: reference-form kernels
    beta, delta = admissible_theta(4)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    rows = [0.5 * a for a in inputs.random_fields((36, 1, 1), seed=51)]   # (1, 1, 36) each
    lam_rows = inputs.random_fields((36, 1, 1), seed=52)
    n = 3
    c = exact_coeffs(beta, delta, dx, dt, 3)

    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    sm.set_state(_rows_to_dev(rows, shape, torch.float64))
    sm.step(n, record=True)
    got = sm.get_state()
    states = [F.State(rows[:3], rows[3:])]
    for _ in range(n):
        states.append(F.step(states[-1].copy(), c))
    want = states[-1].E + states[-1].B
    for a in range(6):
        assert _max_dev(got[a], want[a]) <= 1e-12 * max(1.0, float(np.abs(want[a]).max())), a
    del got
    # adjoint over the recorded steps, with the coefficient gradient (a sum over all cells:
    # ny nz times the one-row gradient)
    sm.set_adjoint(_rows_to_dev(lam_rows, shape, torch.float64))
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    sm.step_adjoint(n, grad)
    lam = sm.get_adjoint()
    ls = F.State(lam_rows[:3], lam_rows[3:])
    gd = {}
    for m in range(n - 1, -1, -1):
        F.adjoint_step(ls, states[m].E, c, gd)
    rgb, rgd = F.grad_to_arrays(gd)
    for a, want_a in enumerate(ls.E + ls.B):
        assert _max_dev(lam[a], want_a) <= 1e-11 * max(1.0, float(np.abs(want_a).max())), a
    g = grad.cpu().numpy()
    cells = shape[1] * shape[2]
    ref = np.concatenate([rgb.reshape(-1), rgd]) * cells
    assert np.max(np.abs(g - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    sm.close()
    # the PIC cycle's field halves (no particles) on the same grid
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    sm.set_state(_rows_to_dev(rows, shape, torch.float64))
    sm.pic_step(n, [])
    got = sm.get_state()
    for a in range(6):
        assert _max_dev(got[a], want[a]) <= 1e-12 * max(1.0, float(np.abs(want[a]).max())), a
    sm.close()


def _big_fp32(shape):
    free, _ = torch.cuda.mem_get_info()
    if free < 140 * 2 ** 30:
        pytest.skip(f"needs ~125 GB of free device memory, {free / 2 ** 30:.0f} GB free")
    nx, ny, nz = shape
    beta, delta = admissible_theta(0)
    dx = [1.0, 1.0, 1.0]
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    row = inputs.plane_wave((nx, 1, 1), (2 * np.pi * 64 / nx, 0.0, 0.0), (0.0, 0.0, 1.0), dx)
    n = 2
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f32")
    ez = _rows_to_dev([row[2]], shape, torch.float32)[0]
    sm.set_state([None, None, ez, None, None, None])
    del ez
    sm.step(n)
    out_ez = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    out_by = torch.empty_like(out_ez)
    L.fdtd_get_state(sm.h, [None, None, out_ez.data_ptr(), None, out_by.data_ptr(), None],
                     L.FDTD_MEM_DEVICE)
    sm.sync()
    c = rounded_coeffs(beta, delta, dx, dt, 3, np.float32)
    st = F.State([np.zeros((1, 1, nx)), np.zeros((1, 1, nx)), row[2].astype(np.float32)],
                 [np.zeros((1, 1, nx))] * 3)
    for _ in range(n):
        F.step(st, c)
    err_e = _max_dev(out_ez, st.E[2])
    err_b = _max_dev(out_by, st.B[1])
    sm.close()
    del out_ez, out_by
    torch.cuda.empty_cache()
    return err_e, err_b


def test_fp32_fused_kernel_at_its_largest_offsets():
    # padded arrays (4096 + 8) x (8 + 4) x 43600 = 2,147,212,800 elements < 2^31
    err_e, err_b = _big_fp32((4096, 8, 43600))
    assert err_e <= 2e-6 and err_b <= 2e-6, (err_e, err_b)


def test_fp32_beyond_2_31_elements():
    # padded arrays (4096 + 8) x (8 + 4) x 43700 = 2,152,137,600 elements > 2^31
    err_e, err_b = _big_fp32((4096, 8, 43700))
    assert err_e <= 2e-6 and err_b <= 2e-6, (err_e, err_b)
