"""Helpers shared by the GPU parity tests (oracle side and comparison metrics)."""
import math

import numpy as np

from oracle import dispersion as D
from oracle import fdtd as F


def rounded_coeffs(beta, delta, dx, dt, dims, np_dtype):
    """Oracle coefficients reproducing the update multipliers of a kernel working in
    ``np_dtype``: m = round(dt * coef / dx_a) for the Faraday taps, round(dt / dx_a) for
    Ampere, each computed in FP64 first (the definition of the multipliers)."""
    b, d = D.clean_coeffs(beta, delta, dims)
    alpha = [1.0 - 2.0 * (b[i, 0] + b[i, 1] + b[i, 2]) - 3.0 * d[i] for i in range(3)]
    dx = [float(v) for v in dx]
    cE = [float(np_dtype(dt / dx[a])) for a in range(3)]
    dxe = [dt / cE[a] for a in range(3)]
    be = np.zeros((3, 3))
    de = np.zeros(3)
    ae = np.zeros(3)
    for a in range(3):
        for c in range(3):
            be[a, c] = float(np_dtype(dt * b[a, c] / dx[a])) * dxe[a] / dt
        de[a] = float(np_dtype(dt * d[a] / dx[a])) * dxe[a] / dt
        ae[a] = float(np_dtype(dt * alpha[a] / dx[a])) * dxe[a] / dt
    return F.Coeffs(be, de, dxe, dt, alpha=ae)


def exact_coeffs(beta, delta, dx, dt, dims):
    b, d = D.clean_coeffs(beta, delta, dims)
    return F.Coeffs(b, d, dx, dt)


def rel_l2(a_list, b_list):
    num = sum(float(np.sum((np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) ** 2))
              for a, b in zip(a_list, b_list))
    den = sum(float(np.sum(np.asarray(b, dtype=np.float64) ** 2)) for b in b_list)
    return math.sqrt(num / max(den, 1e-300))


def admissible_theta(seed, dims=3):
    """First admissible draw (min S >= 0) from the seeded generator, starting at `seed`."""
    from paper_1710_06829_gb300 import inputs
    s = seed
    while True:
        beta, delta = inputs.random_theta(s, dims)
        smin, _ = D.S_extremes(beta, delta, [1, 1, 1], dims)
        if smin >= 0:
            return beta, delta
        s += 1000


def max_elem_err(a_list, b_list):
    """Per component c: max_i |a_c[i] - b_c[i]| / max_i |b_c[i]|, and the worst element's index."""
    out = []
    for a, b in zip(a_list, b_list):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        d = np.abs(a - b)
        i = int(np.argmax(d))
        out.append((float(d.flat[i]) / max(float(np.max(np.abs(b))), 1e-300),
                    np.unravel_index(i, d.shape)))
    return out


def assert_elementwise(a_list, b_list, tol, what=""):
    """Element-by-element check of every component: |a - b| <= tol * max|b| at every cell
    (a seam, ghost-image or edge-tile error in one cell cannot hide in a whole-field norm)."""
    for c, (err, idx) in enumerate(max_elem_err(a_list, b_list)):
        assert err <= tol, f"{what} component {c}: max error {err:.3e} x max|ref| at (z, y, x) = {idx}"
