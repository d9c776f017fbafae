"""GPU constrained minimisation (fdtd_coeff_update + disp_norm_eval) against the SLSQP oracle."""
import math

import numpy as np
import pytest

from oracle import dispersion as D

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import _lib as L  # noqa: E402
from paper_1710_06829_gb300 import optimize as O  # noqa: E402


def test_coeff_update_kernel_is_the_projected_step():
    tie = O.Tying.isotropic_3d(0.4)
    theta = np.array([-0.05, -0.02, 0.03, 0.01])
    g = np.linspace(-1.0, 1.0, 13)
    lo, hi = np.full(4, -0.06), np.full(4, 0.06)
    out = torch.empty(17, dtype=torch.float64, device="cuda")
    L.fdtd_coeff_update(theta, g, tie.T, tie.c0, 0.05, lo, hi, out.data_ptr())
    v = out.cpu().numpy()
    th_ref = np.clip(theta - 0.05 * tie.T @ g, lo, hi)
    assert np.allclose(v[:4], th_ref, rtol=0, atol=1e-15)
    assert np.allclose(v[4:], tie.c0 + tie.T.T @ th_ref, rtol=0, atol=1e-15)


def test_2d_minimum_matches_slsqp_oracle():
    """Fixed c dt/dx = 0.5, beta_xy = beta_yx, delta_x = delta_y (Table 1 setting without Eq. beta)."""
    nu, N = 0.5, (256, 256, 1)
    tie = O.Tying.symmetric_2d(dt=nu)
    lo, hi = np.array([-0.125, -0.125]), np.array([0.25, 0.125])
    obj = O.NormObjective([1, 1, 1], 2, N)
    theta, c, J, hist = O.minimise(obj, tie, [0.0, 0.0], lo, hi, iters=50)

    def up(x):
        beta = np.zeros((3, 3))
        beta[0, 1] = beta[1, 0] = x[0]
        return beta, np.array([x[1], x[1], 0.0]), nu
    x, fs = D.minimise(up, [(-0.125, 0.25), (-0.125, 0.125)], [[0.0, 0.0], [0.1, -0.1]],
                       [1, 1, 1], N, 2)
    assert J <= 1.01 * fs
    assert np.allclose(theta, x, atol=2e-3)


def test_3d_isotropic_minimum_matches_slsqp_oracle():
    """3D, theta = (delta_x, delta_perp, beta_x, beta_perp), fixed dt, uniform weight, small k-grid."""
    N = (24, 24, 24)
    beta0, delta0 = np.zeros((3, 3)), np.zeros(3)
    dt = 0.5 * D.dt_max(beta0, delta0, [1, 1, 1], 3)
    tie = O.Tying.isotropic_3d(dt)
    lo, hi = np.full(4, -0.125), np.full(4, 0.125)
    obj = O.NormObjective([1, 1, 1], 3, N)
    theta, c, J, hist = O.minimise(obj, tie, np.zeros(4), lo, hi, iters=100)

    def up(x):
        beta = np.array([[0, x[2], x[2]], [x[2], 0, x[3]], [x[2], x[3], 0]])
        return beta, np.array([x[0], x[1], x[1]]), dt
    x, fs = D.minimise(up, [(-0.125, 0.125)] * 4, [np.zeros(4), np.array([-0.1, -0.1, 0.05, 0.0])],
                       [1, 1, 1], N, 3)
    assert J <= 1.01 * fs, (J, fs, theta, x)


def _table1(golden):
    return {r[0]: r for r in golden("table1_uniform_norms.txt")}


def _printed(value, printed, rel=0.05):
    p = float(printed)
    dec = len(printed.split(".")[1]) if "." in printed else 0
    return abs(value - p) <= 0.5 * 10 ** (-dec) or abs(value - p) <= rel * abs(p)


def test_gpu_slsqp_reproduces_ndfx_and_lehe(golden):
    """Sec. 5, reproducing published stencils, with every norm evaluation on the GPU (256^2
    k-grid): c dt = dx gives NDFX (beta 1/8, delta 0; norm as printed in Table 1); delta_y held at
    zero with c dt / dx = 0.96 gives Lehe's scheme (beta 1/8, delta_x -0.021)."""
    N = (256, 256, 1)
    obj = O.NormObjective([1, 1, 1], 2, N)
    tie = O.Tying.symmetric_2d(dt=None)
    theta, c, J = O.slsqp(obj, tie, [[0.0625, 0.0625, 1.0], [0.2, 0.0, 1.0], [0.15, 0.02, 1.0]],
                          [-0.125, -0.125, 1.0], [0.25, 0.125, 1.0])
    assert abs(theta[0] - 0.125) <= 0.002 and abs(theta[1]) <= 0.002, theta
    assert _printed(J, _table1(golden)["NDFX"][5])
    tie = O.Tying.sym_beta_2d(0.96)
    starts = [[b, d, 0.0] for b in (0.0, 0.1, 0.2) for d in (-0.1, 0.0)]
    theta, c, J = O.slsqp(obj, tie, starts, [-0.125, -0.125, -1e-6], [0.25, 0.125, 1e-6])
    assert abs(theta[0] - 0.125) <= 0.002 and abs(theta[1] + 0.021) <= 0.002, theta
    # the paper states the coefficients; the minimum lies a little below the norm of the printed
    # (rounded) Lehe coefficients
    assert J <= 1.0 * O.NormObjective([1, 1, 1], 2, N)(
        O.Tying.sym_beta_2d(0.96).c0 + O.Tying.sym_beta_2d(0.96).T.T @ np.array([0.125, -0.021, 0.0]))[0]


def test_gpu_slsqp_reproduces_min1(golden):
    """min.1 of Table 1 (beta_xy = beta_yx, delta_x = delta_y, dt free) from the 3 x 2 x 2 start
    grid, every evaluation on the GPU (256^2 k-grid)."""
    row = _table1(golden)["min1"]
    obj = O.NormObjective([1, 1, 1], 2, (256, 256, 1))
    tie = O.Tying.symmetric_2d(dt=None)
    starts = [[b, d, n] for b in (-0.1, 0.05, 0.2) for d in (-0.1, 0.1) for n in (0.3, 0.8)]
    theta, c, J = O.slsqp(obj, tie, starts, [-0.125, -0.125, 0.05], [0.25, 0.125, 1.0])
    assert abs(theta[0] - float(row[2])) <= 0.002
    assert abs(theta[1] - float(row[3])) <= 0.002
    assert abs(theta[2] - float(row[1])) <= 0.002
    assert _printed(J, row[5])


def _table2(golden):
    return {r[0]: r for r in golden("table2_xaxis_weight.txt")}


@pytest.mark.parametrize("name", ["min5", "min6"])
def test_gpu_slsqp_table2_weighted_minima(golden, name):
    """Table 2 (Sec. 5.2, weight exp(-(k_y dy / 0.1)^2)): at the printed c dt / dx of min.5
    (0.96) and min.6 (0.999), with beta_xy = beta_yx and delta_x, delta_y free, SLSQP over the
    GPU norm reaches the oracle minimiser's weighted norm (within 1 %) and the printed delta_x.
    The printed norms of Lehe and min.5 are not used (they differ ~10x under every reading; only
    their ordering is pinned, on the oracle)."""
    row = _table2(golden)[name]
    nu, dx_printed = float(row[1]), float(row[3])
    N = (256, 256, 1)
    objw = O.NormObjective([1, 1, 1], 2, N, L.FDTD_W_GAUSS_Y, 0.1)
    tie = O.Tying.sym_beta_2d(nu)
    starts = [[b, dx_, dy_] for b in (0.1, 0.13) for dx_ in (-0.02, 0.0) for dy_ in (-0.02, 0.0)]
    lo, hi = [-0.125, -0.125, -0.125], [0.25, 0.125, 0.125]
    theta, c, J = O.slsqp(objw, tie, starts, lo, hi)

    def up(x):
        beta = np.zeros((3, 3))
        beta[0, 1] = beta[1, 0] = x[0]
        return beta, np.array([x[1], x[2], 0.0]), nu
    # starts outside Eq. (constraints) at this c dt / dx are skipped by the oracle minimiser
    x, fs = D.minimise(up, list(zip(lo, hi)), [[0.125, 0.0, 0.0], [0.14, -0.01, 0.0],
                                               [0.13, 0.0, -0.02]], [1, 1, 1], N, 2,
                       D.WEIGHT_GAUSS_Y, 0.1)
    assert J <= 1.01 * fs, (J, fs, theta, x)
    assert abs(theta[1] - dx_printed) <= 0.002, (theta, dx_printed)
    # the GPU minimum is a minimum of the oracle's norm too
    assert D.norm(*up(theta), [1, 1, 1], N, 2, D.WEIGHT_GAUSS_Y, 0.1) == pytest.approx(J, rel=1e-10)


def test_gpu_fig3_aspect_ratio(golden):
    """Fig. 3 (Sec. 5.3, dy = 10 dx; norms in units where the larger step is 1): Yee at 0.95 of
    its limit on the GPU is the printed 20.7 within 1 %, and the optimum over all five
    parameters found with the GPU norm matches the oracle minimiser's within 1 %."""
    (dxs, dys, frac, printed), = golden("fig3_aspect_ratio.txt")
    dxa = [float(dxs), float(dys), 1.0]
    N = (128, 128, 1)
    obj = O.NormObjective(dxa, 2, (512, 512, 1))
    yee_dt = float(frac) * L.fdtd_dt_max(L.make_coeffs(np.zeros((3, 3)), np.zeros(3)), dxa, 2)[0]
    J_yee = obj(np.r_[np.zeros(12), yee_dt])[0]
    assert J_yee == pytest.approx(float(printed), rel=0.01)
    obj = O.NormObjective(dxa, 2, N)
    tie = O.Tying.general_2d()
    lo, hi = [-0.125, -0.125, -0.125, -0.125, 0.001], [0.25, 0.25, 0.125, 0.125, 0.2]
    starts = [[0.0, 0.0, -0.1, 0.0, 0.9 * yee_dt], [0.1, 0.0, 0.0, 0.0, 0.5 * yee_dt],
              [0.0, 0.1, -0.1, 0.0, 0.5 * yee_dt]]
    theta, c, J = O.slsqp(obj, tie, starts, lo, hi)

    def up(x):
        beta = np.zeros((3, 3))
        beta[0, 1], beta[1, 0] = x[0], x[1]
        return beta, np.array([x[2], x[3], 0.0]), x[4]
    x, fs = D.minimise(up, list(zip(lo, hi)), starts, dxa, N, 2)
    assert J <= 1.01 * fs, (J, fs, theta, x)
    assert J < 0.01 * J_yee
