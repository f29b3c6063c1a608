"""Gradient of the basilar-membrane response with respect to the per-segment
bending stiffness, through the reverse time step (``ib_adjoint_step``).

The response is the history of the membrane's normal displacement
eta_l^n = D_l^n . n0_l (n0 the membrane's rest normal) over the last
``window`` of ``n_steps`` forward steps, as a function of the stiffness b
[n_seg].  ``MembraneResponse`` is the torch.autograd.Function: its forward
runs the steps on the context and keeps a state snapshot every
``ckpt_every`` steps in device memory; its backward walks the segments in
reverse, replays each one from its snapshot (keeping every state of the
segment), and applies ``ib_adjoint_step`` step by step, adding the loss's
sensitivity to eta at the observed states and accumulating dJ/db in FP64 on
the device.  All of the time stepping runs in the library's kernels; this
module only orders the calls and holds the buffers.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Context


class MembraneRun:
    """One structure on one context with its initial state (the problem's
    velocity and time, displacement D0 or zero) and checkpoint store."""

    def __init__(self, problem, prec: str = "fp32", n_steps: int = 800, window: int = 200, ckpt_every: int = 40,
                 D0=None):
        if not (0 < window <= n_steps) or ckpt_every < 1:
            raise ValueError("need 0 < window <= n_steps and ckpt_every >= 1")
        st = problem.structure
        if st.normal0 is None or st.n_membrane <= 0:
            raise ValueError("the structure has no membrane normals")
        self.n_steps, self.window, self.ckpt_every = int(n_steps), int(window), int(ckpt_every)
        self.ctx = Context(problem.grid, prec=prec)
        self.ctx.set_structure(st)
        self.m = self.ctx.m
        self.M = int(st.n_membrane)
        self.nseg = len(st.bend_b)
        self.n0 = torch.from_numpy(np.ascontiguousarray(st.normal0[:, :self.M], dtype=np.float64)).cuda()
        self.ctx.set_state(problem.u, None, problem.t0)
        self.ctx.set_displacement(np.zeros((3, self.m)) if D0 is None else D0)
        self.init = self.ctx.new_snapshot()
        self.ctx.snapshot_save(self.init)
        nck = (self.n_steps + self.ckpt_every - 1) // self.ckpt_every
        self.ckpts = [self.ctx.new_snapshot() for _ in range(nck)]
        self.traj = [self.ctx.new_snapshot() for _ in range(self.ckpt_every + 1)]
        self.first_obs = self.n_steps - self.window + 1        # first observed state index

    def _observe(self) -> torch.Tensor:
        D = self.ctx.get_displacement()
        return (D[:, :self.M] * self.n0).sum(0)

    def forward(self, bend_b) -> torch.Tensor:
        """eta [window, M] (float64) of states first_obs .. n_steps."""
        ctx = self.ctx
        ctx.set_bend_stiffness(bend_b)
        ctx.snapshot_load(self.init)
        eta = torch.empty((self.window, self.M), dtype=torch.float64, device="cuda")
        for n in range(self.n_steps):
            if n % self.ckpt_every == 0:
                ctx.snapshot_save(self.ckpts[n // self.ckpt_every])
            ctx.step(1)
            k = n + 1 - self.first_obs
            if k >= 0:
                eta[k] = self._observe()
        return eta

    def backward(self, g_eta: torch.Tensor) -> torch.Tensor:
        """dJ/db [n_seg] (float64, device) given dJ/deta [window, M], for the
        stiffness of the last forward()."""
        ctx = self.ctx
        g_eta = g_eta.to(device="cuda", dtype=torch.float64)
        lam_u = torch.zeros((3,) + ctx.n[::-1], dtype=ctx.dtype_t, device="cuda")
        lam_D = torch.zeros((3, self.m), dtype=torch.float64, device="cuda")
        grad = torch.zeros(self.nseg, dtype=torch.float64, device="cuda")
        nck = len(self.ckpts)
        for k in range(nck - 1, -1, -1):
            start = k * self.ckpt_every
            end = min(start + self.ckpt_every, self.n_steps)
            ctx.snapshot_load(self.ckpts[k])
            for n in range(start, end):
                ctx.snapshot_save(self.traj[n - start])
                ctx.step(1)
            ctx.snapshot_save(self.traj[end - start])
            for n in range(end - 1, start - 1, -1):
                j = n + 1 - self.first_obs                      # sensitivity of the observed state n+1
                if j >= 0:
                    lam_D[:, :self.M] += g_eta[j] * self.n0
                ctx.snapshot_load(self.traj[n - start])
                ctx.adjoint_step(lam_u, lam_D, u_np1=ctx.snapshot_velocity(self.traj[n + 1 - start]),
                                 grad_b=grad, out=(lam_u, lam_D))
        return grad

    def close(self):
        self.ctx.close()


class MembraneResponse(torch.autograd.Function):
    """eta = MembraneResponse.apply(bend_b, run): the membrane's normal
    displacement history [window, M] as a differentiable function of the
    per-segment bending stiffness bend_b [n_seg] (float64)."""

    @staticmethod
    def forward(fctx, bend_b, run: MembraneRun):
        fctx.run = run
        fctx.b_device, fctx.b_dtype = bend_b.device, bend_b.dtype
        return run.forward(bend_b.detach())

    @staticmethod
    def backward(fctx, g_eta):
        grad = fctx.run.backward(g_eta)
        return grad.to(device=fctx.b_device, dtype=fctx.b_dtype), None


def membrane_response(bend_b: torch.Tensor, run: MembraneRun) -> torch.Tensor:
    return MembraneResponse.apply(bend_b, run)


def misfit(eta: torch.Tensor, eta_target: torch.Tensor) -> torch.Tensor:
    """L2 misfit of the normal displacement, averaged over the window and the
    membrane markers."""
    return ((eta - eta_target) ** 2).sum() / eta.numel()
