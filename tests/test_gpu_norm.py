"""GPU dispersion norm + gradient (disp_norm_eval) against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import dispersion as D

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402
from paper_1710_06829_gb300 import _lib as L  # noqa: E402

WK = {"uniform": (D.WEIGHT_UNIFORM, L.FDTD_W_UNIFORM, 0.0),
      "cone": (D.WEIGHT_CONE_X, L.FDTD_W_CONE_X, math.radians(30)),
      "gauss": (D.WEIGHT_GAUSS_Y, L.FDTD_W_GAUSS_Y, 0.1)}


@pytest.mark.parametrize("dims,N", [(2, (64, 48, 1)), (3, (24, 20, 17)), (1, (100, 1, 1)), (3, (1, 1, 1))])
@pytest.mark.parametrize("w", ["uniform", "cone", "gauss"])
def test_norm_and_gradient_match_oracle(dims, N, w):
    okind, gkind, par = WK[w]
    beta, delta = inputs.random_theta(7, dims)
    smin, _ = D.S_extremes(beta, delta, [1, 1, 1], dims)
    if smin < 0:
        beta, delta = beta * 0.3, delta * 0.3
    dx = [1.0, 1.2, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, dims)
    f, gb, gd, gdt = S.disp_norm(beta, delta, dt, dx, dims, N, gkind, par)
    rf, rgb, rgd, rgdt = D.norm_and_grad(beta, delta, dt, dx, N, dims, okind, par)
    assert f == pytest.approx(rf, rel=1e-12, abs=1e-300)
    assert np.allclose(np.array(gb), rgb, rtol=1e-11, atol=1e-13 * max(1.0, abs(rf)))
    assert np.allclose(gd, rgd, rtol=1e-11, atol=1e-13 * max(1.0, abs(rf)))
    assert gdt == pytest.approx(rgdt, rel=1e-11, abs=1e-13)


def test_table1_on_gpu(golden):
    for name, nu, b, dxx, dyy, printed in golden("table1_uniform_norms.txt"):
        beta = np.zeros((3, 3))
        beta[0, 1] = beta[1, 0] = float(b)
        delta = np.array([float(dxx), float(dyy), 0.0])
        f, *_ = S.disp_norm(beta, delta, float(nu), [1, 1, 1], 2, (512, 512, 1))
        ref = D.norm(beta, delta, float(nu), [1, 1, 1], (512, 512, 1), 2)
        assert f == pytest.approx(ref, rel=1e-12), name


def test_full_size_256_cubed_sampled():
    """256^3 norm: value and gradient agree with the oracle's own evaluation at full size."""
    beta, delta = inputs.isotropic_theta(-0.05, -0.04, 0.02, 0.01)
    dt = 0.9 * D.dt_max(beta, delta, [1, 1, 1], 3)
    f, gb, gd, gdt = S.disp_norm(beta, delta, dt, [1, 1, 1], 3, (256, 256, 256))
    rf, rgb, rgd, rgdt = D.norm_and_grad(beta, delta, dt, [1, 1, 1], (256, 256, 256), 3)
    assert f == pytest.approx(rf, rel=1e-11)
    assert np.allclose(gd, rgd, rtol=1e-10)
    assert np.allclose(np.array(gb), rgb, rtol=1e-10, atol=1e-12)


def test_rejects_unstable():
    beta = np.zeros((3, 3))
    with pytest.raises(L.FdtdError):
        S.disp_norm(beta, np.zeros(3), 0.8, [1, 1, 1], 2, (16, 16, 1))


def test_omega_eval_matches_oracle_and_table3(golden):
    rng = np.random.default_rng(3)
    beta, delta = inputs.random_theta(11, 3)
    dx = [1.0, 1.2, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    k = rng.uniform(0, 1, (500, 3)) * np.pi / np.array(dx)
    got = S.omega(beta, delta, dt, dx, 3, k)
    ref = D.omega(k[:, 0], k[:, 1], k[:, 2], beta, delta, dt, dx, 3)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    # Table 3 extremes of v_ph from GPU omega on a 512^2 grid (2D, dx = dy)
    t1 = {r[0]: r for r in golden("table1_uniform_norms.txt")}
    n = 512
    kk = np.arange(1, n + 1) * np.pi / n
    KY, KX = np.meshgrid(kk, kk, indexing="ij")
    K = np.stack([KX.ravel(), KY.ravel(), np.zeros(KX.size)], axis=1)
    for name, vmin, vmax in golden("table3_phase_velocity.txt"):
        _, nu, b, dxx, dyy, _ = t1[name]
        be = np.zeros((3, 3))
        be[0, 1] = be[1, 0] = float(b)
        de = np.array([float(dxx), float(dyy), 0.0])
        w = S.omega(be, de, float(nu), [1, 1, 1], 2, K)
        v = w / np.linalg.norm(K, axis=1)
        assert abs(v.min() - float(vmin)) <= 0.015 and abs(v.max() - float(vmax)) <= 0.015, name


@pytest.mark.parametrize("dims,N", [(2, (64, 48, 1)), (3, (24, 20, 17)), (1, (100, 1, 1))])
@pytest.mark.parametrize("w", ["uniform", "cone", "gauss"])
def test_group_norm_and_gradient_match_oracle(dims, N, w):
    okind, gkind, par = WK[w]
    beta, delta = inputs.random_theta(9, dims)
    smin, _ = D.S_extremes(beta, delta, [1, 1, 1], dims)
    if smin < 0:
        beta, delta = beta * 0.3, delta * 0.3
    dx = [1.0, 1.2, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, dims)
    f, gb, gd, gdt = S.group_norm(beta, delta, dt, dx, dims, N, gkind, par)
    rf, rgb, rgd, rgdt = D.group_norm_and_grad(beta, delta, dt, dx, N, dims, okind, par)
    assert f == pytest.approx(rf, rel=1e-11, abs=1e-300)
    scale = max(1.0, abs(rf))
    assert np.allclose(np.array(gb), rgb, rtol=1e-10, atol=1e-12 * scale)
    assert np.allclose(gd, rgd, rtol=1e-10, atol=1e-12 * scale)
    assert gdt == pytest.approx(rgdt, rel=1e-10, abs=1e-12 * scale)


def test_group_norm_full_size_256_cubed():
    """256^3 group norm: value and gradient against the oracle's own full-size evaluation."""
    beta, delta = inputs.isotropic_theta(-0.05, -0.04, 0.02, 0.01)
    dt = 0.9 * D.dt_max(beta, delta, [1, 1, 1], 3)
    f, gb, gd, gdt = S.group_norm(beta, delta, dt, [1, 1, 1], 3, (256, 256, 256))
    rf, rgb, rgd, rgdt = D.group_norm_and_grad(beta, delta, dt, [1, 1, 1], (256, 256, 256), 3)
    assert f == pytest.approx(rf, rel=1e-10)
    assert np.allclose(gd, rgd, rtol=1e-9)
    assert np.allclose(np.array(gb), rgb, rtol=1e-9, atol=1e-11)
    assert gdt == pytest.approx(rgdt, rel=1e-9)


def test_group_norm_1d_yee_courant_one_is_zero():
    """1D Yee at c dt = dx: v_g = 1 exactly, so f_g is round-off only (near k dx = pi both the
    numerator and sqrt(1 - dt^2 S) of |v_g| vanish, which amplifies it)."""
    f, *_ = S.group_norm(np.zeros((3, 3)), np.zeros(3), 1.0, [1, 1, 1], 1, (4096, 1, 1))
    assert f < 1e-18
