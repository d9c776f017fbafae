"""GPU adjoint step and coefficient gradient against the oracle adjoint and finite differences."""
import math

import numpy as np
import pytest

from gpu_util import admissible_theta, assert_elementwise, exact_coeffs, rel_l2, rounded_coeffs
from oracle import dispersion as D
from oracle import fdtd as F

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1710_06829_gb300 import inputs  # noqa: E402
from paper_1710_06829_gb300 import sim as S  # noqa: E402
from paper_1710_06829_gb300.autograd import FdtdProbeLoss, ProbeLossProblem, tied_coefficients  # noqa: E402


def oracle_adjoint(coeffs, fields, lam_fields, n, sponge=None, probe=None):
    """Oracle reverse sweep: returns (lambda after n reverse steps, grad beta 3x3, grad delta 3).
    probe = (component, x_index, target[n, nz, ny])."""
    states = [F.State(fields[:3], fields[3:])]
    for _ in range(n):
        states.append(F.step(states[-1].copy(), coeffs, None, sponge))
    lam = F.State(lam_fields[:3], lam_fields[3:])
    g = {}
    for m in range(n - 1, -1, -1):
        if probe is not None:
            comp, xp, tgt = probe
            E = states[m + 1].E[comp]
            lam.E[comp][:, :, xp] += 2.0 * (E[:, :, xp] - tgt[m])
        F.adjoint_step(lam, states[m].E, coeffs, g, sponge)
    gb, gd = F.grad_to_arrays(g)
    return lam.E + lam.B, gb, gd


def gpu_adjoint(shape, dx, dt, beta, delta, dtype, fields, lam_fields, n, probe=None, **kw):
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, **kw)
    sm.set_state([torch.from_numpy(f) for f in fields])
    pr = None
    if probe is not None:
        comp, xp, tgt = probe
        tt = torch.from_numpy(tgt).to("cuda", dtype=sm.tdtype).contiguous()
        pr = S.Probe(comp, xp, tt)
    sm.step(n, record=True)
    sm.set_adjoint([torch.from_numpy(f) for f in lam_fields])
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    sm.step_adjoint(n, grad, probe=pr)
    lam = [t.double().cpu().numpy() for t in sm.get_adjoint()]
    g = grad.cpu().numpy()
    sm.close()
    return lam, g[:9].reshape(3, 3), g[9:]


@pytest.mark.parametrize("shape,sponge", [((16, 12, 10), False), ((20, 24, 24), True), ((4, 3, 2), False)])
def test_adjoint_fp64_matches_oracle(shape, sponge):
    beta, delta = admissible_theta(6)
    dx = [1.0, 1.1, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, 11)
    lam0 = inputs.random_fields(shape, 12)
    n = 6
    kw = dict(absorb_cells=5, absorb_sigma=0.3) if sponge else {}
    nx, ny, nz = shape
    sp = F.sponge_factor((nz, ny, nx), 5, 0.3) if sponge else None
    rng = np.random.default_rng(0)
    probe = (2, 3, rng.standard_normal((n, nz, ny)))
    lam, gb, gd = gpu_adjoint(shape, dx, dt, beta, delta, "f64", fields, lam0, n, probe, **kw)
    rlam, rgb, rgd = oracle_adjoint(exact_coeffs(beta, delta, dx, dt, 3), fields, lam0, n, sp, probe)
    assert rel_l2(lam, rlam) <= 1e-12
    assert_elementwise(lam, rlam, 1e-11, str(shape))
    scale = max(np.abs(rgb).max(), np.abs(rgd).max())
    assert np.max(np.abs(gb - rgb)) <= 1e-11 * scale
    assert np.max(np.abs(gd - rgd)) <= 1e-11 * scale


def test_adjoint_fp32_vs_fp64_finite_differences():
    """FP32 fields, FP64 gradient reduction vs central differences (h = 1e-4) of the FP64 oracle."""
    shape = (24, 16, 16)
    beta, delta = admissible_theta(8)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, 21)
    n = 10
    nx, ny, nz = shape
    tgt = np.zeros((n, nz, ny))
    probe = (2, 5, tgt)
    lam0 = [np.zeros((nz, ny, nx))] * 6
    lam, gb, gd = gpu_adjoint(shape, dx, dt, beta, delta, "f32",
                              [f.astype(np.float32) for f in fields], lam0, n, probe)

    def loss(b, d):
        s = F.State(fields[:3], fields[3:])
        c = exact_coeffs(b, d, dx, dt, 3)
        tot = 0.0
        for m in range(n):
            F.step(s, c)
            tot += float(np.sum((s.E[2][:, :, 5] - tgt[m]) ** 2))
        return tot
    h = 1e-4
    for (i, j) in [(0, 1), (1, 2), (2, 0)]:
        bp, bm = beta.copy(), beta.copy()
        bp[i, j] += h
        bm[i, j] -= h
        fd = (loss(bp, delta) - loss(bm, delta)) / (2 * h)
        assert gb[i, j] == pytest.approx(fd, rel=1e-4)
    for i in range(3):
        dp, dm = delta.copy(), delta.copy()
        dp[i] += h
        dm[i] -= h
        fd = (loss(beta, dp) - loss(beta, dm)) / (2 * h)
        assert gd[i] == pytest.approx(fd, rel=1e-4)


def test_autograd_checkpointed_matches_oracle():
    """Config-4 shape at small size: probe loss, checkpoint every 5 of 20 steps, tied theta."""
    shape = (32, 16, 16)
    nx, ny, nz = shape
    dx = [1.0, 1.0, 1.0]
    theta0 = torch.tensor([-0.05, -0.04, 0.02, 0.01], dtype=torch.float64)
    b0, d0 = inputs.isotropic_theta(*theta0.tolist())
    dt = 0.95 * D.dt_max(b0, d0, dx, 3)
    Ez = inputs.pulse_ez_3d(shape, dx, 10.0, 3.0, 5.0, 8.0)
    z = np.zeros_like(Ez)
    init = [torch.from_numpy(a) for a in (z, z, Ez, z, z, z)]
    n, every, xp = 20, 5, 20
    rng = np.random.default_rng(3)
    tgt = rng.standard_normal((n, nz, ny)) * 0.01
    prob = ProbeLossProblem(shape, dx, dt, init, 2, xp, torch.from_numpy(tgt).cuda(), n, every,
                            dtype="f64")
    theta = theta0.clone().requires_grad_(True)
    beta, delta = tied_coefficients(theta)
    loss = FdtdProbeLoss.apply(beta, delta, prob)
    loss.backward()
    # oracle: loss and gradient of the same problem
    c = exact_coeffs(b0, d0, dx, dt, 3)
    fields = [a.numpy() for a in init]
    _, rgb, rgd = oracle_adjoint(c, fields, [np.zeros_like(Ez)] * 6, n, None, (2, xp, tgt))
    g_ref = np.array([rgd[0], rgd[1] + rgd[2], rgb[0, 1] + rgb[0, 2] + rgb[1, 0] + rgb[2, 0],
                      rgb[1, 2] + rgb[2, 1]])
    s = F.State(fields[:3], fields[3:])
    ref_loss = 0.0
    for m in range(n):
        F.step(s, c)
        ref_loss += float(np.sum((s.E[2][:, :, xp] - tgt[m]) ** 2))
    assert float(loss.detach()) == pytest.approx(ref_loss, rel=1e-12)
    assert np.allclose(theta.grad.numpy(), g_ref, rtol=1e-10, atol=1e-12 * np.abs(g_ref).max())


def test_autograd_checkpointed_fp32_one_kernel_matches_oracle():
    """The checkpointed autograd path in FP32 on a TMA-eligible grid: every reverse segment runs
    the one-kernel step, whose two adjoint state sets alternate across segments of odd length
    (checkpoint every 5 of 25 steps); loss and tied-theta gradient against the oracle on the
    FP32-rounded multipliers."""
    shape = (64, 16, 16)
    nx, ny, nz = shape
    dx = [1.0, 1.0, 1.0]
    theta0 = torch.tensor([-0.05, -0.04, 0.02, 0.01], dtype=torch.float64)
    b0, d0 = inputs.isotropic_theta(*theta0.tolist())
    dt = 0.95 * D.dt_max(b0, d0, dx, 3)
    Ez = inputs.pulse_ez_3d(shape, dx, 20.0, 8.0, 8.0, 8.0).astype(np.float32)
    z = np.zeros_like(Ez)
    init = [torch.from_numpy(a) for a in (z, z, Ez, z, z, z)]
    n, every, xp = 25, 5, 30
    rng = np.random.default_rng(4)
    tgt = (rng.standard_normal((n, nz, ny)) * 0.01).astype(np.float32)
    prob = ProbeLossProblem(shape, dx, dt, init, 2, xp, torch.from_numpy(tgt).cuda(), n, every,
                            dtype="f32")
    theta = theta0.clone().requires_grad_(True)
    beta, delta = tied_coefficients(theta)
    loss = FdtdProbeLoss.apply(beta, delta, prob)
    loss.backward()
    c = rounded_coeffs(b0, d0, dx, dt, 3, np.float32)
    fields = [a.numpy().astype(np.float64) for a in init]
    t64 = tgt.astype(np.float64)
    _, rgb, rgd = oracle_adjoint(c, fields, [np.zeros_like(fields[0])] * 6, n, None, (2, xp, t64))
    g_ref = np.array([rgd[0], rgd[1] + rgd[2], rgb[0, 1] + rgb[0, 2] + rgb[1, 0] + rgb[2, 0],
                      rgb[1, 2] + rgb[2, 1]])
    st = F.State(fields[:3], fields[3:])
    ref_loss = 0.0
    for m in range(n):
        F.step(st, c)
        ref_loss += float(np.sum((st.E[2][:, :, xp] - t64[m]) ** 2))
    assert float(loss.detach()) == pytest.approx(ref_loss, rel=1e-5)
    g = theta.grad.numpy()
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.abs(g_ref).max(), (g, g_ref)


def test_batched_2d_adjoint_gradient_is_the_sum_over_members():
    shape = (64, 16, 3)
    nx, ny, nz = shape
    beta = np.zeros((3, 3))
    beta[0, 1], beta[1, 0] = 0.02, -0.01
    delta = np.array([-0.04, -0.02, 0.0])
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 2)
    fields = inputs.random_fields(shape, 31)
    lam0 = inputs.random_fields(shape, 32)
    n = 5
    rng = np.random.default_rng(1)
    tgt = rng.standard_normal((n, nz, ny))
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=2, dtype="f64", batched=True)
    sm.set_state([torch.from_numpy(f) for f in fields])
    sm.step(n, record=True)
    sm.set_adjoint([torch.from_numpy(f) for f in lam0])
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    probe = S.Probe(1, 7, torch.from_numpy(tgt).cuda())
    sm.step_adjoint(n, grad, probe=probe)
    lam = [t.cpu().numpy() for t in sm.get_adjoint()]
    g = grad.cpu().numpy()
    sm.close()
    c = exact_coeffs(beta, delta, dx, dt, 2)
    gb_sum, gd_sum = np.zeros((3, 3)), np.zeros(3)
    for k in range(nz):
        rl, gb, gd = oracle_adjoint(c, [f[k:k + 1] for f in fields], [f[k:k + 1] for f in lam0], n,
                                    None, (1, 7, tgt[:, k:k + 1, :]))
        assert rel_l2([x[k:k + 1] for x in lam], rl) <= 1e-12
        assert_elementwise([x[k:k + 1] for x in lam], rl, 1e-11, f"member {k}")
        gb_sum += gb
        gd_sum += gd
    scale = max(np.abs(gb_sum).max(), np.abs(gd_sum).max())
    assert np.max(np.abs(g[:9].reshape(3, 3) - gb_sum)) <= 1e-11 * scale
    assert np.max(np.abs(g[9:] - gd_sum)) <= 1e-11 * scale
    # entries of the absent z axis are exactly zero
    assert g[2] == 0 and g[5] == 0 and g[6] == 0 and g[7] == 0 and g[11] == 0


def test_batched_2d_adjoint_fp32_one_kernel_matches_oracle():
    """Batched 2D problems (z indexes independent members) through the FP32 one-kernel reverse
    step (a TMA-eligible grid): each member's lambda against the oracle's 2D adjoint on the
    FP32-rounded multipliers, the gradient against the sum over members, the absent z axis's
    entries exactly zero."""
    shape = (64, 16, 5)
    nx, ny, nz = shape
    beta = np.zeros((3, 3))
    beta[0, 1], beta[1, 0] = 0.02, -0.01
    delta = np.array([-0.04, -0.02, 0.0])
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 2)
    fields = [f.astype(np.float32) for f in inputs.random_fields(shape, 33)]
    lam0 = [f.astype(np.float32) for f in inputs.random_fields(shape, 34)]
    n = 5
    rng = np.random.default_rng(2)
    tgt = rng.standard_normal((n, nz, ny)).astype(np.float32)
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=2, dtype="f32", batched=True)
    sm.set_state([torch.from_numpy(f) for f in fields])
    sm.step(n, record=True)
    sm.set_adjoint([torch.from_numpy(f) for f in lam0])
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    sm.step_adjoint(n, grad, probe=S.Probe(1, 7, torch.from_numpy(tgt).cuda()))
    lam = [t.double().cpu().numpy() for t in sm.get_adjoint()]
    g = grad.cpu().numpy()
    sm.close()
    c = rounded_coeffs(beta, delta, dx, dt, 2, np.float32)
    gb_sum, gd_sum = np.zeros((3, 3)), np.zeros(3)
    for k in range(nz):
        rl, gb, gd = oracle_adjoint(c, [f[k:k + 1].astype(np.float64) for f in fields],
                                    [f[k:k + 1].astype(np.float64) for f in lam0], n, None,
                                    (1, 7, tgt[:, k:k + 1, :].astype(np.float64)))
        assert_elementwise([x[k:k + 1] for x in lam], rl, 2e-5, f"member {k}")
        gb_sum += gb
        gd_sum += gd
    scale = max(np.abs(gb_sum).max(), np.abs(gd_sum).max())
    assert np.max(np.abs(g[:9].reshape(3, 3) - gb_sum)) <= 2e-5 * scale
    assert np.max(np.abs(g[9:] - gd_sum)) <= 2e-5 * scale
    assert g[2] == 0 and g[5] == 0 and g[6] == 0 and g[7] == 0 and g[11] == 0


@pytest.mark.parametrize("shape,sponge", [((64, 16, 12), False), ((128, 24, 40), True), ((64, 8, 1), False)])
def test_adjoint_fp32_staged_kernel_matches_oracle(shape, sponge):
    """FP32 adjoint on TMA-eligible grids (nx % 64 == 0, ny % 8 == 0) vs the oracle adjoint run
    with the FP32-rounded multipliers; 40 planes leave a ragged last z-chunk."""
    beta, delta = admissible_theta(9)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = [f.astype(np.float32) for f in inputs.random_fields(shape, 41)]
    lam0 = [f.astype(np.float32) for f in inputs.random_fields(shape, 42)]
    n = 6
    nx, ny, nz = shape
    kw = dict(absorb_cells=4, absorb_sigma=0.3) if sponge else {}
    sp = F.sponge_factor((nz, ny, nx), 4, 0.3).astype(np.float32).astype(np.float64) if sponge else None
    rng = np.random.default_rng(5)
    probe = (0, 9, rng.standard_normal((n, nz, ny)).astype(np.float32))
    lam, gb, gd = gpu_adjoint(shape, dx, dt, beta, delta, "f32", fields, lam0, n, probe, **kw)
    f64 = [f.astype(np.float64) for f in fields]
    l64 = [f.astype(np.float64) for f in lam0]
    rlam, rgb, rgd = oracle_adjoint(rounded_coeffs(beta, delta, dx, dt, 3, np.float32), f64, l64, n,
                                    sp, (probe[0], probe[1], probe[2].astype(np.float64)))
    assert rel_l2(lam, rlam) <= 5e-6
    # FP32 round-off of 6 reverse steps (with the probe source), cell by cell
    assert_elementwise(lam, rlam, 2e-5, str(shape))
    scale = max(np.abs(rgb).max(), np.abs(rgd).max())
    assert np.max(np.abs(gb - rgb)) <= 2e-5 * scale
    assert np.max(np.abs(gd - rgd)) <= 2e-5 * scale


def test_adjoint_fp32_staged_vs_fp64_finite_differences():
    """FP32 fields + FP64 gradient reduction on a TMA-eligible grid vs FP64 central differences."""
    shape = (64, 16, 16)
    beta, delta = admissible_theta(8)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, 21)
    n = 10
    nx, ny, nz = shape
    tgt = np.zeros((n, nz, ny))
    lam0 = [np.zeros((nz, ny, nx))] * 6
    lam, gb, gd = gpu_adjoint(shape, dx, dt, beta, delta, "f32",
                              [f.astype(np.float32) for f in fields], lam0, n, (2, 5, tgt))

    def loss(b, d):
        s = F.State(fields[:3], fields[3:])
        c = exact_coeffs(b, d, dx, dt, 3)
        tot = 0.0
        for m in range(n):
            F.step(s, c)
            tot += float(np.sum((s.E[2][:, :, 5] - tgt[m]) ** 2))
        return tot
    h = 1e-4
    for (i, j) in [(0, 1), (1, 2), (2, 0)]:
        bp, bm = beta.copy(), beta.copy()
        bp[i, j] += h
        bm[i, j] -= h
        assert gb[i, j] == pytest.approx((loss(bp, delta) - loss(bm, delta)) / (2 * h), rel=1e-4)
    for i in range(3):
        dp, dm = delta.copy(), delta.copy()
        dp[i] += h
        dm[i] -= h
        assert gd[i] == pytest.approx((loss(beta, dp) - loss(beta, dm)) / (2 * h), rel=1e-4)


def test_adjoint_fp32_256_transpose_and_gradient_vs_fp64():
    """Full size (256^3, the bench's grid and launch configuration): the staged FP32 reverse step
    is the transpose of the FP32 forward step, <M u - u, lam> = <u, M^T lam - lam> (a property
    at any size), and its coefficient gradient agrees with the FP64 path's (reference-form
    kernels, themselves matched to the oracle on small grids)."""
    n = 256
    shape = (n, n, n)
    dx = [1.0, 1.0, 1.0]
    beta, delta = admissible_theta(0)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    u = [torch.from_numpy(f.astype(np.float32)) for f in inputs.random_fields(shape, 51)]
    lam = [torch.from_numpy(f.astype(np.float32)) for f in inputs.random_fields(shape, 52)]
    grads = {}
    for dtype in ("f32", "f64"):
        sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype)
        tu = [t.to(sm.tdtype) for t in u]
        tl = [t.to(sm.tdtype) for t in lam]
        sm.set_state(tu)
        sm.step(1, record=True)
        Mu = sm.get_state()
        sm.set_adjoint(tl)
        grad = torch.zeros(12, dtype=torch.float64, device="cuda")
        sm.step_adjoint(1, grad)
        MTl = sm.get_adjoint()
        sm.close()
        if dtype == "f32":
            lhs = sum(float(((Mu[c].double() - u[c].cuda().double()) * lam[c].cuda().double()).sum())
                      for c in range(6))
            rhs = sum(float((u[c].cuda().double() * (MTl[c].double() - lam[c].cuda().double())).sum())
                      for c in range(6))
            assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
        grads[dtype] = grad.cpu().numpy()
        del Mu, MTl
    g32, g64 = grads["f32"], grads["f64"]
    assert np.max(np.abs(g32 - g64)) <= 1e-4 * np.max(np.abs(g64))


def test_adjoint_fp32_256_reverse_step_matches_oracle():
    """Full size (256^3, the bench's grid and launch configuration), one reverse step of the
    staged FP32 kernels against the oracle adjoint run on the FP32-rounded multipliers: lambda
    element by element, and the 12-entry coefficient gradient."""
    n = 256
    shape = (n, n, n)
    dx = [1.0, 1.0, 1.0]
    beta, delta = admissible_theta(0)
    dt = 0.95 * D.dt_max(beta, delta, dx, 3)
    u = [f.astype(np.float32) for f in inputs.random_fields(shape, 61)]
    lam0 = [f.astype(np.float32) for f in inputs.random_fields(shape, 62)]
    lam, gb, gd = gpu_adjoint(shape, dx, dt, beta, delta, "f32", u, lam0, 1)
    rlam, rgb, rgd = oracle_adjoint(rounded_coeffs(beta, delta, dx, dt, 3, np.float32),
                                    [f.astype(np.float64) for f in u],
                                    [f.astype(np.float64) for f in lam0], 1)
    assert_elementwise(lam, rlam, 1e-5, "256^3 reverse step")
    scale = max(np.abs(rgb).max(), np.abs(rgd).max())
    assert np.max(np.abs(gb - rgb)) <= 1e-4 * scale
    assert np.max(np.abs(gd - rgd)) <= 1e-4 * scale


@pytest.mark.parametrize("shape,sponge", [((64, 8, 3), False), ((128, 16, 37), True),
                                          ((192, 24, 75), False), ((64, 16, 1), False),
                                          ((64, 8, 9), True)])
def test_one_kernel_reverse_step_equals_two_kernel_step(shape, sponge, monkeypatch):
    """The one-kernel FP32 reverse step (default: mu on the tile and its halo, lambda_E two planes
    behind, gradient from the transposed brackets) against the two-kernel step
    (FDTD_ADJOINT_SPLIT=1: mu in place, then lambda_E), same inputs and probe, 4 reverse steps:
    lambda bitwise equal (the same arithmetic per value), the gradient equal up to the order of
    the FP32 partial sums (forward brackets on E^n there, transposed brackets on mu here)."""
    beta, delta = admissible_theta(7)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = [f.astype(np.float32) for f in inputs.random_fields(shape, 71)]
    lam0 = [f.astype(np.float32) for f in inputs.random_fields(shape, 72)]
    n = 4
    nx, ny, nz = shape
    kw = dict(absorb_cells=2, absorb_sigma=0.3) if sponge else {}
    rng = np.random.default_rng(7)
    probe = (1, 5, rng.standard_normal((n, nz, ny)).astype(np.float32))
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("FDTD_ADJOINT_SPLIT", flag)
        out[flag] = gpu_adjoint(shape, dx, dt, beta, delta, "f32", fields, lam0, n, probe, **kw)
    (l1, gb1, gd1), (l2, gb2, gd2) = out["0"], out["1"]
    for c in range(6):
        nd = int(np.count_nonzero(l1[c] != l2[c]))
        assert nd == 0, (f"component {c}: {nd} of {l1[c].size} differ, max |diff| "
                         f"{np.max(np.abs(l1[c] - l2[c])):.3e}, at {np.argwhere(l1[c] != l2[c])[:4].tolist()}")
    scale = max(np.abs(gb2).max(), np.abs(gd2).max())
    assert np.max(np.abs(gb1 - gb2)) <= 1e-5 * scale
    assert np.max(np.abs(gd1 - gd2)) <= 1e-5 * scale
