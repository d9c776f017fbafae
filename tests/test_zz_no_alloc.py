"""disp_norm_eval_noalloc: the dispersion norm for callers that must not allocate device memory.

Such callers (for example code that runs while another stream of the device is being
captured into a CUDA graph, or a host whose own pool owns all device memory) get the same
result as disp_norm_eval from a scratch area the library declares statically per device.
This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process and after the others.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300 import inputs  # noqa: E402

# (coefficients, dims, N, weight, weight parameter): two different calls in a row, so the
# second one runs on scratch that still holds the first call's contents
CASES = [
    (inputs.isotropic_theta(-0.05, -0.04, 0.02, 0.01), 3, (48, 40, 36), L.FDTD_W_UNIFORM, 0.0),
    (inputs.isotropic_theta(-0.02, -0.06, 0.05, -0.01), 2, (512, 256, 1), L.FDTD_W_CONE_X,
     math.radians(30)),
]


def _dt(beta, delta, dims):
    dtm, _, _ = L.fdtd_dt_max(L.make_coeffs(beta, delta), [1.0, 1.0, 1.0], dims)
    return 0.9 * dtm


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    for (beta, delta), dims, N, w, wp in CASES:
        c = L.make_coeffs(beta, delta)
        dt = _dt(beta, delta, dims)
        got = np.array(L.disp_norm_eval_noalloc(c, dt, [1, 1, 1], dims, N, w, wp))
        ref = np.array(L.disp_norm_eval(c, dt, [1, 1, 1], dims, N, w, wp))
        # tolerance of the other GPU norm tests (FP64 throughout)
        assert got[0] == pytest.approx(ref[0], rel=1e-12)
        assert np.allclose(got[1:], ref[1:], rtol=1e-11, atol=1e-13 * max(1.0, abs(ref[0])))


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    (beta, delta), dims = CASES[0][0], 3
    c = L.make_coeffs(beta, delta)
    with pytest.raises(L.FdtdError) as ei:
        L.disp_norm_eval_noalloc(c, _dt(beta, delta, dims), [1, 1, 1], dims, (4097, 8, 8))
    assert ei.value.status == L.FDTD_EINVAL
    assert "4096" in str(ei.value)


def test_noalloc_calls_leave_device_memory_unchanged():
    """The property the entry point exists for: after one warm-up call (which looks the scratch
    address up), further calls take no device memory, whether from cudaMalloc or a pool (the
    device's free memory, as the driver reports it, does not move)."""
    torch = pytest.importorskip("torch")
    (beta, delta), dims, N, w, wp = CASES[1]
    c = L.make_coeffs(beta, delta)
    dt = _dt(beta, delta, dims)
    torch.cuda.synchronize()
    L.disp_norm_eval_noalloc(c, dt, [1, 1, 1], dims, N, w, wp)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        L.disp_norm_eval_noalloc(c, dt, [1, 1, 1], dims, N, w, wp)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
