"""ctypes binding of libfdtd (include/fdtd.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and raises
``FdtdError`` on a non-zero status.  The shared library is built in-tree by
``paper_1710_06829_gb300.build``; if it is missing, importing the compute
entry points fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdtd.so")

FDTD_OK = 0
FDTD_EINVAL = -1
FDTD_EUNSTABLE = -2
FDTD_ECUDA = -3
FDTD_ENOMEM = -4
FDTD_ENONFINITE = -5
FDTD_ESTATE = -6
FDTD_ETIMEOUT = -7

FDTD_F32 = 0
FDTD_F64 = 1
FDTD_MEM_DEVICE = 0
FDTD_MEM_HOST = 1
FDTD_SRC_NONE = 0
FDTD_SRC_BUNCH = 1
FDTD_SRC_DENSE = 2
FDTD_W_UNIFORM = 0
FDTD_W_CONE_X = 1
FDTD_W_GAUSS_Y = 2
FDTD_DIAG_ENERGY = 0
FDTD_DIAG_PLANEWAVE = 1
FDTD_DIAG_MOMENTS = 2
FDTD_DIV_STAR_B = 0
FDTD_DIV_YEE_B = 1
FDTD_DIV_E = 2

STATUS_NAMES = {0: "FDTD_OK", -1: "FDTD_EINVAL", -2: "FDTD_EUNSTABLE", -3: "FDTD_ECUDA",
                -4: "FDTD_ENOMEM", -5: "FDTD_ENONFINITE", -6: "FDTD_ESTATE",
                -7: "FDTD_ETIMEOUT"}

# every symbol include/fdtd.h declares
EXPORTS = ["fdtd_create", "fdtd_set_coeffs", "fdtd_set_state", "fdtd_get_state", "fdtd_get_step",
           "fdtd_step", "fdtd_checkpoint", "fdtd_set_adjoint", "fdtd_get_adjoint",
           "fdtd_step_adjoint", "fdtd_diagnostic", "fdtd_divergence", "fdtd_pic_step",
           "fdtd_deposit_rho", "fdtd_selftest_wait_expiry", "fdtd_set_temporal_blocking",
           "fdtd_sync", "fdtd_destroy", "disp_norm_eval",
           "disp_norm_eval_noalloc", "disp_group_norm_eval", "disp_omega_eval", "fdtd_coeff_update", "fdtd_dt_max", "fdtd_last_error"]


class FdtdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fdtd_grid(C.Structure):
    _fields_ = [("dims", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dtype", C.c_int32), ("absorb_cells", C.c_int32), ("absorb_sigma", C.c_double),
                ("batched", C.c_int32)]


class fdtd_coeffs(C.Structure):
    _fields_ = [("beta", (C.c_double * 3) * 3), ("delta", C.c_double * 3)]


class fdtd_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("q", C.c_double), ("v", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("z0", C.c_double), ("sigma_par", C.c_double),
                ("sigma_perp", C.c_double), ("J", C.c_void_p * 3)]


class fdtd_probe(C.Structure):
    _fields_ = [("component", C.c_int32), ("x_index", C.c_int32), ("target", C.c_void_p),
                ("target_steps", C.c_int64)]


class fdtd_species(C.Structure):
    _fields_ = [("x", C.c_void_p * 3), ("u", C.c_void_p * 3), ("n", C.c_int64), ("q", C.c_double),
                ("q_over_m", C.c_double)]


_lib = None


def load():
    """Load libfdtd.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    I32 = C.c_int32
    D = C.c_double
    pd = C.POINTER(C.c_double)
    lib.fdtd_create.argtypes = [C.POINTER(fdtd_grid), pd, D, C.POINTER(fdtd_coeffs), P,
                                C.POINTER(P)]
    lib.fdtd_set_coeffs.argtypes = [P, D, C.POINTER(fdtd_coeffs)]
    lib.fdtd_set_state.argtypes = [P, C.POINTER(P), I32, C.c_int64]
    lib.fdtd_get_state.argtypes = [P, C.POINTER(P), I32]
    lib.fdtd_get_step.argtypes = [P, C.POINTER(C.c_int64)]
    lib.fdtd_step.argtypes = [P, I32, C.POINTER(fdtd_source), C.POINTER(fdtd_probe), P, I32]
    lib.fdtd_checkpoint.argtypes = [P, I32, I32]
    lib.fdtd_set_adjoint.argtypes = [P, C.POINTER(P), I32]
    lib.fdtd_get_adjoint.argtypes = [P, C.POINTER(P), I32]
    lib.fdtd_step_adjoint.argtypes = [P, I32, C.POINTER(fdtd_probe), P]
    lib.fdtd_diagnostic.argtypes = [P, I32, pd, P]
    lib.fdtd_divergence.argtypes = [P, I32, P]
    lib.fdtd_sync.argtypes = [P]
    lib.fdtd_selftest_wait_expiry.argtypes = [P, C.c_int32]
    lib.fdtd_set_temporal_blocking.argtypes = [P, C.c_int32, C.c_int32]
    lib.fdtd_destroy.argtypes = [P]
    lib.fdtd_destroy.restype = None
    lib.disp_norm_eval.argtypes = [C.POINTER(fdtd_coeffs), D, pd, I32, C.POINTER(I32), I32, D,
                                   pd, P]
    lib.disp_norm_eval_noalloc.argtypes = lib.disp_norm_eval.argtypes
    lib.disp_group_norm_eval.argtypes = lib.disp_norm_eval.argtypes
    lib.disp_omega_eval.argtypes = [C.POINTER(fdtd_coeffs), D, pd, I32, P, I32, P, P]
    lib.fdtd_coeff_update.argtypes = [I32, pd, pd, pd, pd, D, pd, pd, P, P]
    lib.fdtd_dt_max.argtypes = [C.POINTER(fdtd_coeffs), pd, I32, pd, pd, pd]
    lib.fdtd_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("fdtd_destroy", "fdtd_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(status):
    if status != FDTD_OK:
        raise FdtdError(status, load().fdtd_last_error().decode())


def _ptrs6(fields):
    arr = (C.c_void_p * 6)()
    if fields is not None:
        for i, f in enumerate(fields):
            arr[i] = f
    return arr


def make_coeffs(beta, delta):
    c = fdtd_coeffs()
    for i in range(3):
        for j in range(3):
            c.beta[i][j] = float(beta[i][j])
        c.delta[i] = float(delta[i])
    return c


def _d3(x):
    return (C.c_double * 3)(*[float(v) for v in x])


# ---- entry points (same names as the C ABI) ---------------------------------


def fdtd_create(grid: fdtd_grid, dx, dt, coeffs: fdtd_coeffs, stream=0):
    h = C.c_void_p()
    check(load().fdtd_create(C.byref(grid), _d3(dx), float(dt), C.byref(coeffs),
                             C.c_void_p(stream), C.byref(h)))
    return h


def fdtd_set_coeffs(h, dt, coeffs):
    check(load().fdtd_set_coeffs(h, float(dt), C.byref(coeffs)))


def fdtd_set_state(h, fields, mem, step0=0):
    check(load().fdtd_set_state(h, _ptrs6(fields), mem, int(step0)))


def fdtd_get_state(h, fields, mem):
    check(load().fdtd_get_state(h, _ptrs6(fields), mem))


def fdtd_get_step(h):
    s = C.c_int64()
    check(load().fdtd_get_step(h, C.byref(s)))
    return s.value


def fdtd_step(h, n, src=None, probe=None, loss_dev=None, record=0):
    check(load().fdtd_step(h, int(n), C.byref(src) if src is not None else None,
                           C.byref(probe) if probe is not None else None,
                           C.c_void_p(loss_dev) if loss_dev else None, int(record)))


def fdtd_checkpoint(h, slot, op):
    check(load().fdtd_checkpoint(h, int(slot), int(op)))


def fdtd_set_adjoint(h, fields, mem):
    check(load().fdtd_set_adjoint(h, _ptrs6(fields), mem))


def fdtd_get_adjoint(h, fields, mem):
    check(load().fdtd_get_adjoint(h, _ptrs6(fields), mem))


def fdtd_step_adjoint(h, n, probe=None, grad_dev=None):
    check(load().fdtd_step_adjoint(h, int(n), C.byref(probe) if probe is not None else None,
                                   C.c_void_p(grad_dev)))


def fdtd_diagnostic(h, kind, params, out_dev):
    check(load().fdtd_diagnostic(h, int(kind), (C.c_double * len(params))(*map(float, params)),
                                 C.c_void_p(out_dev)))


def fdtd_divergence(h, which, out_dev):
    check(load().fdtd_divergence(h, int(which), C.c_void_p(out_dev)))


def fdtd_pic_step(h, n, species):
    arr = (fdtd_species * max(1, len(species)))(*species)
    check(load().fdtd_pic_step(h, int(n), arr, len(species)))


def fdtd_deposit_rho(h, species, rho_dev):
    arr = (fdtd_species * max(1, len(species)))(*species)
    check(load().fdtd_deposit_rho(h, arr, len(species), C.c_void_p(rho_dev)))


def fdtd_sync(h):
    check(load().fdtd_sync(h))


def fdtd_selftest_wait_expiry(h, tries):
    check(load().fdtd_selftest_wait_expiry(h, tries))


def fdtd_set_temporal_blocking(h, T, slab_planes=0):
    check(load().fdtd_set_temporal_blocking(h, T, slab_planes))


def fdtd_destroy(h):
    load().fdtd_destroy(h)


def disp_norm_eval(coeffs, dt, dx, dims, N, weight=FDTD_W_UNIFORM, weight_param=0.0, stream=0):
    out = (C.c_double * 14)()
    n3 = (C.c_int32 * 3)(*[int(v) for v in N])
    check(load().disp_norm_eval(C.byref(coeffs), float(dt), _d3(dx), int(dims), n3, int(weight),
                                float(weight_param), out, C.c_void_p(stream)))
    return list(out)


def disp_group_norm_eval(coeffs, dt, dx, dims, N, weight=FDTD_W_UNIFORM, weight_param=0.0, stream=0):
    out = (C.c_double * 14)()
    n3 = (C.c_int32 * 3)(*[int(v) for v in N])
    check(load().disp_group_norm_eval(C.byref(coeffs), float(dt), _d3(dx), int(dims), n3,
                                      int(weight), float(weight_param), out, C.c_void_p(stream)))
    return list(out)


def disp_norm_eval_noalloc(coeffs, dt, dx, dims, N, weight=FDTD_W_UNIFORM, weight_param=0.0,
                           stream=0):
    """disp_norm_eval on the library's static per-device scratch (allocates nothing)."""
    out = (C.c_double * 14)()
    n3 = (C.c_int32 * 3)(*[int(v) for v in N])
    check(load().disp_norm_eval_noalloc(C.byref(coeffs), float(dt), _d3(dx), int(dims), n3,
                                        int(weight), float(weight_param), out, C.c_void_p(stream)))
    return list(out)


def disp_omega_eval(coeffs, dt, dx, dims, k_dev, n, omega_dev, stream=0):
    check(load().disp_omega_eval(C.byref(coeffs), float(dt), _d3(dx), int(dims), C.c_void_p(k_dev),
                                 int(n), C.c_void_p(omega_dev), C.c_void_p(stream)))


def fdtd_coeff_update(theta, grad13, T, c0, eta, lo, hi, out_dev, stream=0):
    """theta' = clip(theta - eta T grad13, lo, hi), c' = c0 + T^T theta' into out_dev (device)."""
    n = len(theta)
    arr = lambda v: (C.c_double * len(v))(*[float(x) for x in v])  # noqa: E731
    Tflat = [float(x) for row in T for x in row]
    check(load().fdtd_coeff_update(n, arr(theta), arr(grad13), arr(Tflat), arr(c0), float(eta),
                                   arr(lo), arr(hi), C.c_void_p(out_dev), C.c_void_p(stream)))


def fdtd_dt_max(coeffs, dx, dims):
    dtm, smin, smax = C.c_double(), C.c_double(), C.c_double()
    check(load().fdtd_dt_max(C.byref(coeffs), _d3(dx), int(dims), C.byref(dtm), C.byref(smin),
                             C.byref(smax)))
    return dtm.value, smin.value, smax.value


def fdtd_last_error():
    return load().fdtd_last_error().decode()
