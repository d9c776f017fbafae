"""Thin Python objects over the C ABI; torch provides device memory and streams only.

All arithmetic of the method runs in libfdtd's CUDA kernels; this module
allocates tensors, passes their pointers and reads results back.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

_DT = {"f32": (L.FDTD_F32, torch.float32), "f64": (L.FDTD_F64, torch.float64)}


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def coeffs_struct(beta, delta):
    return L.make_coeffs(beta, delta)


def dt_max(beta, delta, dx, dims):
    """Exact CFL limit of Eq. (constraints) and the extremes of S (host FP64 in libfdtd)."""
    return L.fdtd_dt_max(coeffs_struct(beta, delta), dx, dims)


class Bunch:
    """Rigid Gaussian bunch source (see fdtd_source in include/fdtd.h)."""

    def __init__(self, q, v, x0, y0, z0, sigma_par, sigma_perp):
        self.s = L.fdtd_source(L.FDTD_SRC_BUNCH, q, v, x0, y0, z0, sigma_par, sigma_perp)


class DenseCurrent:
    """A current J^{n+1/2} on the grid (see fdtd_source in include/fdtd.h): three device tensors
    (nz, ny, nx) of the simulation's dtype (None = 0), applied in every step of a call."""

    def __init__(self, Jx=None, Jy=None, Jz=None):
        self.J = [None if t is None else t.contiguous() for t in (Jx, Jy, Jz)]
        for t in self.J:
            assert t is None or t.is_cuda
        ptrs = (L.C.c_void_p * 3)(*[None if t is None else t.data_ptr() for t in self.J])
        self.s = L.fdtd_source(L.FDTD_SRC_DENSE, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, ptrs)
        self.dtype = next((t.dtype for t in self.J if t is not None), None)


class Probe:
    """Probe-plane misfit of E_component at x = x_index against target[(steps), nz, ny]."""

    def __init__(self, component, x_index, target: torch.Tensor):
        """target must be a contiguous CUDA tensor of the simulation's dtype."""
        assert target.is_cuda and target.is_contiguous() and target.dim() == 3
        self.target = target
        self.s = L.fdtd_probe(int(component), int(x_index), target.data_ptr(), target.shape[0])


class Species:
    """Macro-particles of one species on the device (see fdtd_species in include/fdtd.h):
    x, u are (3, n) tensors (positions, u = gamma v) of the simulation's dtype, updated in
    place by Simulation.pic_step; q is the macro-particle charge, qm the charge-to-mass ratio."""

    def __init__(self, x: torch.Tensor, u: torch.Tensor, q, qm):
        assert x.is_cuda and u.is_cuda and x.shape == u.shape and x.shape[0] == 3
        assert x.dtype == u.dtype
        self.x = x.contiguous()
        self.u = u.contiguous()
        self.q, self.qm = float(q), float(qm)

    def struct(self):
        n = self.x.shape[1]
        return L.fdtd_species((L.C.c_void_p * 3)(*[self.x[a].data_ptr() for a in range(3)]),
                              (L.C.c_void_p * 3)(*[self.u[a].data_ptr() for a in range(3)]),
                              n, self.q, self.qm)


class Simulation:
    """One FDTD state (E, B) on a periodic nx x ny x nz grid, owned by libfdtd."""

    def __init__(self, shape, dx, dt, beta, delta, dims=3, dtype="f32", absorb_cells=0,
                 absorb_sigma=0.0, stream=None, batched=False):
        nx, ny, nz = shape
        self.shape = (nz, ny, nx)
        self.dims = dims
        self.code, self.tdtype = _DT[dtype]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = L.fdtd_grid(dims, nx, ny, nz, self.code, absorb_cells, absorb_sigma, int(batched))
        self.h = L.fdtd_create(g, dx, dt, coeffs_struct(beta, delta), _stream_ptr(self.stream))
        self.dx = tuple(dx)
        self.dt = dt

    def close(self):
        if self.h is not None:
            L.fdtd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ---------------------------------------------------------------
    def _empty6(self):
        return [torch.empty(self.shape, dtype=self.tdtype, device="cuda") for _ in range(6)]

    def set_state(self, fields, step0=0):
        """fields: six tensors (E_x, E_y, E_z, B_x, B_y, B_z) of shape (nz, ny, nx); None = 0."""
        keep, ptrs, mem = [], [], L.FDTD_MEM_DEVICE
        for f in fields:
            if f is None:
                ptrs.append(None)
                continue
            t = torch.as_tensor(f).to(device="cuda", dtype=self.tdtype).contiguous()
            keep.append(t)
            ptrs.append(t.data_ptr())
        L.fdtd_set_state(self.h, ptrs, mem, step0)
        self.stream.synchronize()

    def set_state_host(self, fields, step0=0):
        """Host (CPU tensor) variant: the copy to the device happens inside libfdtd."""
        ptrs = [None if f is None else f.data_ptr() for f in fields]
        L.fdtd_set_state(self.h, ptrs, L.FDTD_MEM_HOST, step0)

    def get_state(self):
        out = self._empty6()
        L.fdtd_get_state(self.h, [t.data_ptr() for t in out], L.FDTD_MEM_DEVICE)
        self.stream.synchronize()
        return out

    def get_state_host(self, out):
        L.fdtd_get_state(self.h, [t.data_ptr() for t in out], L.FDTD_MEM_HOST)
        return out

    @property
    def step_index(self):
        return L.fdtd_get_step(self.h)

    def set_coeffs(self, dt, beta, delta):
        L.fdtd_set_coeffs(self.h, dt, coeffs_struct(beta, delta))
        self.dt = dt

    # -- stepping ------------------------------------------------------------
    def step(self, n, source: Bunch | None = None, probe: Probe | None = None, loss=None,
             record=False):
        if probe is not None and probe.target.dtype != self.tdtype:
            raise TypeError("probe target dtype does not match the simulation dtype")
        if isinstance(source, DenseCurrent) and source.dtype not in (None, self.tdtype):
            raise TypeError("current dtype does not match the simulation dtype")
        L.fdtd_step(self.h, n, source.s if source is not None else None,
                    probe.s if probe is not None else None,
                    loss.data_ptr() if loss is not None else None, 1 if record else 0)

    def checkpoint_save(self, slot):
        L.fdtd_checkpoint(self.h, slot, 0)

    def checkpoint_restore(self, slot):
        L.fdtd_checkpoint(self.h, slot, 1)

    # -- adjoint -------------------------------------------------------------
    def set_adjoint(self, fields=None):
        keep, ptrs = [], []
        for f in (fields if fields is not None else [None] * 6):
            if f is None:
                ptrs.append(None)
                continue
            t = torch.as_tensor(f).to(device="cuda", dtype=self.tdtype).contiguous()
            keep.append(t)
            ptrs.append(t.data_ptr())
        L.fdtd_set_adjoint(self.h, ptrs, L.FDTD_MEM_DEVICE)
        self.stream.synchronize()

    def get_adjoint(self):
        out = self._empty6()
        L.fdtd_get_adjoint(self.h, [t.data_ptr() for t in out], L.FDTD_MEM_DEVICE)
        self.stream.synchronize()
        return out

    def step_adjoint(self, n, grad: torch.Tensor, probe: Probe | None = None):
        """grad: float64 CUDA tensor of 12 entries (beta 3x3 row-major, delta 3), accumulated."""
        assert grad.is_cuda and grad.dtype == torch.float64 and grad.numel() >= 12
        if probe is not None and probe.target.dtype != self.tdtype:
            raise TypeError("probe target dtype does not match the simulation dtype")
        L.fdtd_step_adjoint(self.h, n, probe.s if probe is not None else None, grad.data_ptr())

    # -- macro-particles (PIC cycle) -----------------------------------------
    def _check_species(self, species):
        for sp in species:
            if sp.x.dtype != self.tdtype:
                raise TypeError("species dtype does not match the simulation dtype")

    def pic_step(self, n, species):
        """n PIC cycles: extended Faraday, gather + Boris push + Esirkepov current for every
        species, Yee Ampere with the current (fdtd_pic_step)."""
        self._check_species(species)
        L.fdtd_pic_step(self.h, n, [sp.struct() for sp in species])

    def deposit_rho(self, species, out=None):
        """Charge density at the nodes (first-order shape), dense (nz, ny, nx) of the dtype."""
        self._check_species(species)
        if out is None:
            out = torch.zeros(self.shape, dtype=self.tdtype, device="cuda")
        L.fdtd_deposit_rho(self.h, [sp.struct() for sp in species], out.data_ptr())
        return out

    # -- diagnostics -----------------------------------------------------------
    def energy(self, x_lo, x_len, margin=0, out=None):
        """(1/2) sum (E^2 + B^2) dV over a periodic x-window (FP64, device tensor of 1)."""
        out = out if out is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        L.fdtd_diagnostic(self.h, L.FDTD_DIAG_ENERGY, [x_lo, x_len, margin], out.data_ptr())
        return out

    def plane_wave(self, component, k, out=None):
        """sum F exp(-i k.r) over the grid: device tensor (Re, Im)."""
        out = out if out is not None else torch.empty(2, dtype=torch.float64, device="cuda")
        L.fdtd_diagnostic(self.h, L.FDTD_DIAG_PLANEWAVE, [component, *k], out.data_ptr())
        return out

    def energy_moments(self, axis, out=None):
        """(W, C, S) = sum (1/2) F^2 dV (1, cos th, sin th), th = 2 pi x_axis / L_axis, over the
        six components at their staggered positions (FP64, device tensor of 3).  The periodic
        energy centroid of a packet is atan2(S, C) L_axis / (2 pi)."""
        out = out if out is not None else torch.empty(3, dtype=torch.float64, device="cuda")
        L.fdtd_diagnostic(self.h, L.FDTD_DIAG_MOMENTS, [axis], out.data_ptr())
        return out

    def divergence(self, which):
        """Dense FP64 divergence field (nz, ny, nx): L.FDTD_DIV_STAR_B / _YEE_B / _E."""
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        L.fdtd_divergence(self.h, which, out.data_ptr())
        self.stream.synchronize()
        return out

    def sync(self):
        L.fdtd_sync(self.h)

    def set_temporal_blocking(self, T, slab_planes=0):
        """T = 2: FP32 steps advance in pairs, slab by slab through L2 (fdtd_set_temporal_blocking)."""
        L.fdtd_set_temporal_blocking(self.h, T, slab_planes)


def disp_norm(beta, delta, dt, dx, dims, N, weight=L.FDTD_W_UNIFORM, weight_param=0.0,
              stream=None):
    """Eq. (norm) and its gradient on the GPU.

    Returns (f, g_beta 3x3 (list of lists), g_delta (3), g_dt)."""
    out = L.disp_norm_eval(coeffs_struct(beta, delta), dt, dx, dims, N, weight, weight_param,
                           _stream_ptr(stream))
    gb = [out[1:4], out[4:7], out[7:10]]
    return out[0], gb, out[10:13], out[13]


def group_norm(beta, delta, dt, dx, dims, N, weight=L.FDTD_W_UNIFORM, weight_param=0.0,
               stream=None):
    """Group-velocity norm (|d omega/dk| - c)^2 on the norm's grid, and its gradient, on the GPU.

    Returns (f_g, g_beta 3x3 (list of lists), g_delta (3), g_dt)."""
    out = L.disp_group_norm_eval(coeffs_struct(beta, delta), dt, dx, dims, N, weight, weight_param,
                                 _stream_ptr(stream))
    gb = [out[1:4], out[4:7], out[7:10]]
    return out[0], gb, out[10:13], out[13]


def omega(beta, delta, dt, dx, dims, k, stream=None):
    """omega(k) of the scheme (Eq. dispersion_relation) on the GPU for an (n, 3) array of k."""
    kt = torch.as_tensor(np.asarray(k, dtype=np.float64).reshape(-1, 3)).cuda().contiguous()
    out = torch.empty(kt.shape[0], dtype=torch.float64, device="cuda")
    L.disp_omega_eval(coeffs_struct(beta, delta), dt, dx, dims, kt.data_ptr(), kt.shape[0],
                      out.data_ptr(), _stream_ptr(stream))
    return out.cpu().numpy()
