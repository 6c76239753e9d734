"""Gradient of time-averaged wall drag by the discrete adjoint, with
sqrt(T) checkpointed recomputation, behind a ``torch.autograd.Function``.

    J(theta) = (1/T) sum_{t=0}^{T-1} d . F_wall(t),  theta = (g[0..2], u_w[0..2])

F_wall(t) is the uncorrected momentum exchange of Eq. (25) (arXiv
2512.12213, Sec. 5) on one wall during step t -> t+1, the run starting from
rest, f(0) = f^eq(rho0, 0).  Every arithmetic step runs in the library's
kernels (lbm_step / lbm_step_from, lbm_wall_force with FP64 accumulation,
lbm_adjoint_step); this module only schedules them.

Memory: ceil(T/k) checkpoints of the stored state plus k - 1 recomputed
states of one segment, k = ceil(sqrt(T)), plus two adjoint buffers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import lbm


class DragProblem:
    def __init__(self, sim: "lbm.Sim", T: int, wall: int, direction=(1.0, 0.0, 0.0), stride: int | None = None):
        if T < 1:
            raise ValueError("T must be >= 1")
        self.sim, self.T, self.wall = sim, int(T), int(wall)
        self.d = tuple(float(v) for v in direction)
        self.k = int(stride or math.ceil(math.sqrt(T)))
        self.nseg = (self.T + self.k - 1) // self.k
        dev = sim.device
        pb = sim.sizes[lbm.BUF_POP_A]
        self.ckpt = torch.empty((self.nseg, pb), dtype=torch.uint8, device=dev)
        self.seg = None        # recomputed states and adjoint buffers: allocated by backward()
        self.phi = None
        self.Facc = torch.zeros(3, dtype=torch.float64, device=dev)
        self.theta = None

    def set_theta(self, theta):
        th = [float(v) for v in np.asarray(theta, dtype=np.float64).reshape(6)]
        lbm.lbm_set_body_force(self.sim.ctx, th[0:3])
        lbm.lbm_set_wall_velocity(self.sim.ctx, self.wall, th[3:6])
        self.theta = th

    def forward(self, theta) -> float:
        """Run T steps from rest, keep checkpoints, return J."""
        s = self.sim
        st = s.stream
        self.set_theta(theta)
        s.rest()
        self.Facc.zero_()
        for t in range(self.T):
            if t % self.k == 0:
                lbm.lbm_save_state(s.ctx, self.ckpt[t // self.k], st)
            lbm.lbm_step(s.ctx, 1, st)
            lbm.lbm_wall_force(s.ctx, self.wall, lbm.ACCUMULATE, 1.0 / self.T, self.Facc, 0, st)
        F = self.Facc.cpu().numpy()
        return float(np.dot(self.d, F))

    def backward(self) -> np.ndarray:
        """dJ/dtheta (6,) for the theta of the last forward()."""
        s = self.sim
        st = s.stream
        ctx = s.ctx
        if self.seg is None:
            pb = s.sizes[lbm.BUF_POP_A]
            self.seg = torch.empty((max(self.k - 1, 1), pb), dtype=torch.uint8, device=s.device)
            ab = lbm.lbm_adjoint_buffer_bytes(ctx)
            self.phi = [torch.empty(ab, dtype=torch.uint8, device=s.device) for _ in range(2)]
        lbm.lbm_adjoint_reset(ctx, st)
        phi_next, cur = None, 0
        for sg in reversed(range(self.nseg)):
            t0, t1 = sg * self.k, min(self.T, (sg + 1) * self.k)
            states = [self.ckpt[sg]] + [self.seg[i] for i in range(t1 - t0 - 1)]
            for i in range(1, t1 - t0):          # recompute P_{t0}, ..., P_{t1-2}
                lbm.lbm_step_from(ctx, states[i - 1], states[i], t0 + i - 1, st)
            for t in reversed(range(t0, t1)):
                out = self.phi[cur]
                lbm.lbm_adjoint_step(ctx, states[t - t0], phi_next, out, self.wall, self.d, 1.0 / self.T, st)
                phi_next, cur = out, 1 - cur
        g = np.zeros(6)
        lbm.lbm_adjoint_gradient(ctx, g, 1, st)
        return g


class DragFn(torch.autograd.Function):
    """J = DragFn.apply(theta, problem): theta a 6-vector (g, u_w)."""

    @staticmethod
    def forward(ctx, theta, problem):
        J = problem.forward(theta.detach().cpu().numpy())
        ctx.problem = problem
        ctx.tdtype, ctx.tdev = theta.dtype, theta.device
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        g = ctx.problem.backward()
        grad = torch.as_tensor(g, dtype=ctx.tdtype, device=ctx.tdev) * gJ.to(ctx.tdtype)
        return grad, None
