"""Constrained coefficient minimisation on the GPU (Sec. 4): projected gradient descent in FP64.

The paper minimises the dispersion norm (Eq. norm) under Eq. (constraints) with SLSQP
inside a bounds cuboid; ``slsqp`` does the same with every norm and gradient evaluation on
the GPU.  ``minimise`` is a GPU-resident alternative in which every evaluation and every
update runs in libfdtd:
``disp_norm_eval`` gives the norm and its exact gradient, ``fdtd_coeff_update`` forms
theta' = clip(theta - eta T g, lo, hi) and the scheme parameters c' = c0 + T^T theta', and
a candidate that violates Eq. (constraints) is rejected by the library's exact CFL check.
The step length grows by 1.5 after an accepted step and halves after a rejected one.

Optionally a propagation term mu * L(theta) is added to the objective, with L and its
gradient supplied by a callable (for instance batched FDTD runs and their adjoint).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

# index of each scheme parameter in c = (beta 3x3 row-major, delta 3, dt)
B = lambda i, j: 3 * i + j  # noqa: E731
DELTA = lambda i: 9 + i  # noqa: E731
DT = 12


class Tying:
    """Linear map from free parameters theta to c = c0 + T^T theta."""

    def __init__(self, T, c0, names):
        self.T = np.asarray(T, dtype=np.float64)
        self.c0 = np.asarray(c0, dtype=np.float64)
        self.names = list(names)

    @property
    def n(self):
        return self.T.shape[0]

    @staticmethod
    def split(c):
        c = np.asarray(c, dtype=np.float64)
        return c[:9].reshape(3, 3), c[9:12], float(c[12])

    @classmethod
    def symmetric_2d(cls, dt=None):
        """2D, beta_xy = beta_yx = beta, delta_x = delta_y = delta (Table 1); dt fixed or free."""
        rows = [np.zeros(13), np.zeros(13)]
        rows[0][B(0, 1)] = rows[0][B(1, 0)] = 1.0
        rows[1][DELTA(0)] = rows[1][DELTA(1)] = 1.0
        c0 = np.zeros(13)
        names = ["beta", "delta"]
        if dt is None:
            r = np.zeros(13)
            r[DT] = 1.0
            rows.append(r)
            names.append("dt")
        else:
            c0[DT] = dt
        return cls(np.array(rows), c0, names)

    @classmethod
    def sym_beta_2d(cls, dt):
        """2D, beta_xy = beta_yx = beta, delta_x and delta_y free, fixed dt (Sec. 5: with delta_y
        held at zero by its bounds this family contains Lehe's scheme)."""
        T = np.zeros((3, 13))
        T[0][B(0, 1)] = T[0][B(1, 0)] = 1.0
        T[1][DELTA(0)] = 1.0
        T[2][DELTA(1)] = 1.0
        c0 = np.zeros(13)
        c0[DT] = dt
        return cls(T, c0, ["beta", "delta_x", "delta_y"])

    @classmethod
    def general_2d(cls):
        """2D, theta = (beta_xy, beta_yx, delta_x, delta_y, dt), all free (unequal steps)."""
        T = np.zeros((5, 13))
        T[0][B(0, 1)] = 1.0
        T[1][B(1, 0)] = 1.0
        T[2][DELTA(0)] = 1.0
        T[3][DELTA(1)] = 1.0
        T[4][DT] = 1.0
        return cls(T, np.zeros(13), ["beta_xy", "beta_yx", "delta_x", "delta_y", "dt"])

    @classmethod
    def isotropic_3d(cls, dt):
        """3D theta = (delta_x, delta_perp, beta_x, beta_perp) at fixed dt."""
        T = np.zeros((4, 13))
        T[0][DELTA(0)] = 1.0
        T[1][DELTA(1)] = T[1][DELTA(2)] = 1.0
        for (i, j) in [(0, 1), (0, 2), (1, 0), (2, 0)]:
            T[2][B(i, j)] = 1.0
        for (i, j) in [(1, 2), (2, 1)]:
            T[3][B(i, j)] = 1.0
        c0 = np.zeros(13)
        c0[DT] = dt
        return cls(T, c0, ["delta_x", "delta_perp", "beta_x", "beta_perp"])


class NormObjective:
    """phase * Eq. (norm) + group * (group-velocity norm) on a midpoint k-grid (GPU), plus an
    optional mu * propagation loss."""

    def __init__(self, dx, dims, N, weight=L.FDTD_W_UNIFORM, weight_param=0.0, prop=None, mu=0.0,
                 phase=1.0, group=0.0):
        self.dx, self.dims, self.N = list(dx), dims, tuple(N)
        self.weight, self.wparam = weight, weight_param
        self.prop, self.mu = prop, mu
        self.phase, self.group = phase, group
        self.evals = 0

    def __call__(self, c):
        """Returns (J, grad13) or (None, None) when c violates Eq. (constraints)."""
        beta, delta, dt = Tying.split(c)
        st = torch.cuda.current_stream().cuda_stream
        J, g = 0.0, np.zeros(13)
        try:
            for wgt, fn in ((self.phase, L.disp_norm_eval), (self.group, L.disp_group_norm_eval)):
                if wgt != 0.0:
                    out = fn(L.make_coeffs(beta, delta), dt, self.dx, self.dims, self.N,
                             self.weight, self.wparam, st)
                    J += wgt * out[0]
                    g += wgt * np.array(out[1:14])
        except L.FdtdError as e:
            if e.status == L.FDTD_EUNSTABLE:
                return None, None
            raise
        self.evals += 1
        if self.prop is not None and self.mu != 0.0:
            Lp, gp = self.prop(beta, delta, dt)
            J = J + self.mu * Lp
            g = g + self.mu * np.asarray(gp)
        return J, g


def minimise(objective, tying: Tying, theta0, lo, hi, iters=50, eta0=1e-2, max_halvings=40):
    """Projected gradient descent with step-length adaptation; returns (theta, c, J, history)."""
    stream = torch.cuda.current_stream()
    out = torch.empty(tying.n + 13, dtype=torch.float64, device="cuda")
    theta = np.asarray(theta0, dtype=np.float64)
    zero = np.zeros(13)

    def update(th, g, eta):
        L.fdtd_coeff_update(th, g, tying.T, tying.c0, eta, lo, hi, out.data_ptr(), stream.cuda_stream)
        v = out.cpu().numpy()
        return v[:tying.n], v[tying.n:]

    theta, c = update(theta, zero, 0.0)   # projects theta0 into the cuboid and forms c
    J, g = objective(c)
    if J is None:
        raise ValueError("the start point violates Eq. (constraints)")
    eta = eta0
    hist = [(0, J)]
    for it in range(1, iters + 1):
        for _ in range(max_halvings):
            th_c, c_c = update(theta, g, eta)
            J_c, g_c = objective(c_c)
            if J_c is not None and J_c < J:
                theta, c, J, g = th_c, c_c, J_c, g_c
                eta *= 1.5
                break
            eta *= 0.5
        else:
            break
        hist.append((it, J))
    return theta, c, J, hist


def slsqp(objective, tying: Tying, starts, lo, hi, maxiter=200):
    """The paper's optimiser (Sec. 4: SLSQP under Eq. (constraints) inside a bounds cuboid, from a
    grid of start points), with every norm and gradient evaluation on the GPU
    (``disp_norm_eval``) and the constraints from the library's exact extremes of S
    (``fdtd_dt_max``): 1 - dt^2 max S >= 0 and min S >= 0.  SciPy's SLSQP drives the search on
    the host.  Returns (theta, c, J) of the best feasible result over the starts."""
    from scipy.optimize import minimize

    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)

    def coeffs(theta):
        return tying.c0 + tying.T.T @ np.asarray(theta, dtype=np.float64)

    def extremes(theta):
        beta, delta, dt = Tying.split(coeffs(theta))
        _, smin, smax = L.fdtd_dt_max(L.make_coeffs(beta, delta), objective.dx, objective.dims)
        return smin, smax, dt

    def cfl(theta):
        smin, smax, dt = extremes(theta)
        return 1.0 - dt * dt * smax

    def pos(theta):
        return extremes(theta)[0]

    cache = {}

    def fun(theta):
        key = tuple(np.round(theta, 15))
        if key not in cache:
            if cfl(theta) < -1e-9 or pos(theta) < -1e-9:
                cache[key] = (1e3, np.zeros(tying.n))
            else:
                J, g13 = objective(coeffs(theta))
                cache[key] = (1e3, np.zeros(tying.n)) if J is None else (J, tying.T @ g13)
        return cache[key]

    best = (None, None, np.inf)
    for x0 in starts:
        x0 = np.clip(np.asarray(x0, dtype=np.float64), lo, hi)
        if cfl(x0) < 0 or pos(x0) < 0:
            continue
        res = minimize(lambda t: fun(t)[0], x0, jac=lambda t: fun(t)[1], method="SLSQP",
                       bounds=list(zip(lo, hi)),
                       constraints=[{"type": "ineq", "fun": cfl}, {"type": "ineq", "fun": pos}],
                       options={"maxiter": maxiter, "ftol": 1e-12})
        x = np.clip(res.x, lo, hi)
        if cfl(x) < -1e-9 or pos(x) < -1e-9:
            continue
        J = fun(x)[0]
        if J < best[2]:
            best = (x, coeffs(x), J)
    return best
