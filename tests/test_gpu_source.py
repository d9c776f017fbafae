"""A current given on the grid (FDTD_SRC_DENSE) against the oracle's step with J.

* Steps with a constant dense J, FP64 and FP32, on a grid the fused TMA kernel takes and on a
  ragged one (reference-form kernels), with and without the absorbing layer, and with a NULL
  component: E^{n+1} = E^n + dt (D x B^{n+1/2} - J) element by element (App. A update
  equations).
* Recording the E history while the current is applied (the fused kernel writes the
  snapshot before the current is added; the library replaces it): the adjoint and its
  coefficient gradient over that history equal the oracle's over the true E^n.
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

TD = {"f64": (torch.float64, np.float64), "f32": (torch.float32, np.float32)}


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", TD[dtype][0])


@pytest.mark.parametrize("dtype,shape,absorb,drop", [
    ("f64", (64, 16, 12), 0, None), ("f32", (64, 16, 12), 0, None),
    ("f64", (20, 13, 11), 3, None), ("f32", (20, 13, 11), 0, 1), ("f64", (64, 16, 12), 2, 2)])
def test_dense_current_matches_oracle(dtype, shape, absorb, drop):
    beta, delta = admissible_theta(7)
    dx = [1.0, 1.1, 0.9]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    npd = TD[dtype][1]
    fields = [f.astype(npd).astype(np.float64) for f in inputs.random_fields(shape, seed=61)]
    J = [f.astype(npd).astype(np.float64) for f in inputs.random_fields(shape, seed=62)[:3]]
    if drop is not None:
        J[drop] = None
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype=dtype, absorb_cells=absorb,
                      absorb_sigma=0.4)
    sm.set_state([_dev(f, dtype) for f in fields])
    cur = S.DenseCurrent(*[None if j is None else _dev(j, dtype) for j in J])
    n = 3
    sm.step(n, source=cur)
    got = [t.cpu().numpy().astype(np.float64) for t in sm.get_state()]
    sm.sync()
    sm.close()
    c = exact_coeffs(beta, delta, dx, dt, 3) if dtype == "f64" else \
        rounded_coeffs(beta, delta, dx, dt, 3, np.float32)
    sponge = F.sponge_factor((shape[2], shape[1], shape[0]), absorb, 0.4) if absorb else None
    st = F.State(fields[:3], fields[3:])
    for _ in range(n):
        F.step(st, c, J, sponge)
    want = st.E + st.B
    scale = max(float(np.abs(w).max()) for w in want)
    tol = 1e-13 if dtype == "f64" else 1e-5
    for a in range(6):
        assert np.max(np.abs(got[a] - want[a])) <= tol * scale, a


def test_recorded_history_includes_the_current():
    shape = (64, 16, 12)   # the fused TMA kernel, which writes the history itself
    beta, delta = admissible_theta(8)
    dx = [1.0, 1.0, 1.0]
    dt = 0.9 * D.dt_max(beta, delta, dx, 3)
    fields = inputs.random_fields(shape, seed=63)
    J = inputs.random_fields(shape, seed=64)[:3]
    lam0 = inputs.random_fields(shape, seed=65)
    n = 4
    sm = S.Simulation(shape, dx, dt, beta, delta, dims=3, dtype="f64")
    sm.set_state([_dev(f, "f64") for f in fields])
    sm.step(n, source=S.DenseCurrent(*[_dev(j, "f64") for j in J]), record=True)
    sm.set_adjoint([_dev(f, "f64") for f in lam0])
    grad = torch.zeros(12, dtype=torch.float64, device="cuda")
    sm.step_adjoint(n, grad)
    lam = [t.cpu().numpy() for t in sm.get_adjoint()]
    g = grad.cpu().numpy()
    sm.close()
    c = exact_coeffs(beta, delta, dx, dt, 3)
    states = [F.State(fields[:3], fields[3:])]
    for _ in range(n):
        states.append(F.step(states[-1].copy(), c, J))
    ls = F.State(lam0[:3], lam0[3:])
    gd = {}
    for m in range(n - 1, -1, -1):
        F.adjoint_step(ls, states[m].E, c, gd)
    rgb, rgd = F.grad_to_arrays(gd)
    for a, w in enumerate(ls.E + ls.B):
        assert np.max(np.abs(lam[a] - w)) <= 1e-11 * max(1.0, float(np.abs(w).max())), a
    ref = np.concatenate([rgb.reshape(-1), rgd])
    assert np.max(np.abs(g - ref)) <= 1e-10 * max(1.0, float(np.abs(ref).max()))


def test_dense_current_dtype_must_match():
    sm = S.Simulation((64, 16, 12), [1, 1, 1], 0.3, np.zeros((3, 3)), np.zeros(3), dims=3,
                      dtype="f64")
    jx = torch.zeros((12, 16, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        sm.step(1, source=S.DenseCurrent(jx))
    sm.close()
