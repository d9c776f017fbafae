"""Differentiable FDTD: a torch.autograd.Function over libfdtd's forward and adjoint.

The loss is the probe-plane misfit L = sum_s sum_{j,k} (E_c^s[x_p, j, k] - T^s[j, k])^2
over all steps s = 1..n (accumulated in FP64 by the forward kernels).  The
backward pass recomputes each segment of ``ckpt_every`` steps from its
checkpoint (recording E^s), then runs the adjoint kernels over it, newest
segment first; the coefficient gradient is reduced in FP64 on the GPU.
"""
from __future__ import annotations

import torch

from . import sim as S


class ProbeLossProblem:
    """Fixed data of one differentiable run: grid, dt, initial state, probe target."""

    def __init__(self, shape, dx, dt, init_fields, component, x_index, target, nsteps,
                 ckpt_every, dims=3, dtype="f32", absorb_cells=0, absorb_sigma=0.0):
        self.shape, self.dx, self.dt = shape, dx, dt
        self.init = init_fields
        self.component, self.x_index = component, x_index
        self.target = target
        self.nsteps, self.ckpt_every = nsteps, ckpt_every
        self.dims, self.dtype = dims, dtype
        self.absorb = (absorb_cells, absorb_sigma)
        self.sim = None

    def simulation(self, beta, delta):
        if self.sim is None:
            self.sim = S.Simulation(self.shape, self.dx, self.dt, beta, delta, dims=self.dims,
                                    dtype=self.dtype, absorb_cells=self.absorb[0],
                                    absorb_sigma=self.absorb[1])
            self.probe = S.Probe(self.component, self.x_index,
                                 self.target.to(device="cuda", dtype=self.sim.tdtype).contiguous())
        else:
            self.sim.set_coeffs(self.dt, beta, delta)
        return self.sim

    def segments(self):
        s, out = 0, []
        while s < self.nsteps:
            n = min(self.ckpt_every, self.nsteps - s)
            out.append((s, n))
            s += n
        return out


class FdtdProbeLoss(torch.autograd.Function):
    """loss = FdtdProbeLoss.apply(beta (3x3 fp64), delta (3 fp64), problem)."""

    @staticmethod
    def forward(ctx, beta, delta, problem: ProbeLossProblem):
        b = beta.detach().cpu().double().numpy()
        d = delta.detach().cpu().double().numpy()
        sm = problem.simulation(b, d)
        sm.set_state(problem.init)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        for slot, (_, n) in enumerate(problem.segments()):
            sm.checkpoint_save(slot)
            sm.step(n, probe=problem.probe, loss=loss)
        ctx.problem = problem
        ctx.coeffs = (b, d)
        ctx.devices = (beta.device, delta.device)
        return loss[0].to(beta.device)

    @staticmethod
    def backward(ctx, gout):
        problem = ctx.problem
        sm = problem.simulation(*ctx.coeffs)
        sm.set_adjoint(None)
        grad = torch.zeros(12, dtype=torch.float64, device="cuda")
        segs = problem.segments()
        for slot in range(len(segs) - 1, -1, -1):
            _, n = segs[slot]
            sm.checkpoint_restore(slot)
            sm.step(n, record=True)
            sm.step_adjoint(n, grad, probe=problem.probe)
        g = grad.to(ctx.devices[0]) * gout.to(ctx.devices[0])
        return g[:9].reshape(3, 3), g[9:12].to(ctx.devices[1]), None


def tied_coefficients(theta: torch.Tensor):
    """theta = (delta_x, delta_perp, beta_x, beta_perp) -> (beta 3x3, delta 3) with
    delta = (delta_x, delta_perp, delta_perp), beta_xy = beta_yx = beta_xz = beta_zx = beta_x,
    beta_yz = beta_zy = beta_perp (differentiable)."""
    dx_, dp, bx, bp = theta[0], theta[1], theta[2], theta[3]
    z = torch.zeros((), dtype=theta.dtype, device=theta.device)
    beta = torch.stack([torch.stack([z, bx, bx]), torch.stack([bx, z, bp]),
                        torch.stack([bx, bp, z])])
    delta = torch.stack([dx_, dp, dp])
    return beta, delta
