"""torch.autograd binding of the hand-written adjoint (argument marshalling only).

``advect(q0, scale, forest, t0, dt, nsteps)`` returns q_N after ``nsteps``
time steps of ``forest`` starting from the field ``q0`` with every edge speed
multiplied by ``scale``: global steps of ``dt``, or with ``multirate=True``
coarse multirate steps of ``dt`` (each 2^(lmax-lmin) finest-level substeps,
Sec. 4).  Its backward runs the library's adjoint step
(``fc_adjoint_step_global`` / ``fc_adjoint_step_multirate``) in reverse, with
sqrt(N) checkpointing: the forward keeps the field every ``segment`` steps;
the backward recomputes the states inside one segment at a time from its
checkpoint.  The velocity-scale derivative is accumulated in FP64 on the
device.
"""
from __future__ import annotations

import math

import torch


class _Advect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, scale, forest, t0, dt, nsteps, segment, multirate):
        seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
        step = forest.step_multirate if multirate else forest.step_global
        forest.set_velocity_scale(float(scale))
        forest.set_q(q0.detach().contiguous())
        ckpts = {}
        for k in range(nsteps):
            if k % seg == 0:
                c = torch.empty_like(q0)
                forest.get_q(out=c)
                ckpts[k] = c
            step(t0 + k * dt, dt)
        out = torch.empty_like(q0)
        forest.get_q(out=out)
        ctx.forest, ctx.t0, ctx.dt, ctx.nsteps, ctx.seg = forest, t0, dt, nsteps, seg
        ctx.multirate = multirate
        ctx.ckpts = ckpts
        ctx.scale_shape, ctx.scale_dtype = scale.shape, scale.dtype
        return out

    @staticmethod
    def backward(ctx, grad_out):
        F, t0, dt, n, seg = ctx.forest, ctx.t0, ctx.dt, ctx.nsteps, ctx.seg
        step = F.step_multirate if ctx.multirate else F.step_global
        adjoint = F.adjoint_step_multirate if ctx.multirate else F.adjoint_step_global
        lam = grad_out.contiguous().clone()
        dscale = torch.zeros(1, dtype=torch.float64, device=lam.device)
        for start in sorted(ctx.ckpts, reverse=True):
            end = min(start + seg, n)
            F.set_q(ctx.ckpts[start])
            states = []
            for k in range(start, end):
                s = torch.empty_like(lam)
                F.get_q(out=s)
                states.append(s)
                if k < end - 1:
                    step(t0 + k * dt, dt)
            for k in range(end - 1, start - 1, -1):
                F.set_q(states[k - start])
                adjoint(t0 + k * dt, dt, lam, dscale)
        ctx.ckpts = None
        gscale = dscale.to(ctx.scale_dtype).reshape(ctx.scale_shape)
        return lam, gscale, None, None, None, None, None, None


def advect(q0: torch.Tensor, scale: torch.Tensor, forest, t0: float, dt: float, nsteps: int,
           segment: int = 0, multirate: bool = False) -> torch.Tensor:
    """Differentiable N-step advance of ``forest`` (see module docstring)."""
    return _Advect.apply(q0, scale, forest, t0, dt, nsteps, segment, multirate)
