"""torch.autograd binding of the hand-written adjoint (argument marshalling only).

``advect(q0, scale, forest, t0, dt, nsteps)`` returns q_N after ``nsteps``
time steps of ``forest`` starting from the field ``q0`` with every edge speed
multiplied by ``scale``: global steps of ``dt``, or with ``multirate=True``
coarse multirate steps of ``dt`` (each 2^(lmax-lmin) finest-level substeps,
Sec. 4).  Its backward runs the library's adjoint step in reverse, with
sqrt(N) checkpointing: the forward keeps the field every ``segment`` steps;
the backward recomputes one segment at a time from its checkpoint.  Global
steps: each state of the segment is kept and ``fc_adjoint_step_global``
reversed from it.  Multirate steps: the recompute records every step on a
tape (``fc_step_multirate_record``, one slot per step of the segment) and
``fc_adjoint_step_multirate_taped`` reverses them from their tapes, so no
step is replayed a third time.  With ``tape="forward"`` (the default for
multirate runs of at most FC_MAX_TAPE_SLOTS steps when no segment length is
given) the forward pass itself records every step when a gradient is
needed and the backward only reverses them: no recompute, at the cost of
one tape per step in device memory (the kept tiles of every substep).  The
velocity-scale derivative is accumulated in FP64 on the device.  A forest
holds the tapes of one taped run at a time.
"""
from __future__ import annotations

import math

import torch


MAX_TAPE_SLOTS = 64  # FC_MAX_TAPE_SLOTS


class _Advect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, scale, forest, t0, dt, nsteps, segment, multirate, tape):
        seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
        step = forest.step_multirate if multirate else forest.step_global
        forest.set_velocity_scale(float(scale))
        forest.set_q(q0.detach().contiguous())
        taped = tape == "forward" and any(ctx.needs_input_grad[:2])
        if taped:  # the forest's tapes belong to this run until its backward
            forest._tape_run = getattr(forest, "_tape_run", 0) + 1
            ctx.tape_run = forest._tape_run
        ckpts = {}
        for k in range(nsteps):
            if taped:
                forest.step_multirate_record(t0 + k * dt, dt, k)
                continue
            if k % seg == 0:
                c = torch.empty_like(q0)
                forest.get_q(out=c)
                ckpts[k] = c
            step(t0 + k * dt, dt)
        out = torch.empty_like(q0)
        forest.get_q(out=out)
        ctx.forest, ctx.t0, ctx.dt, ctx.nsteps, ctx.seg = forest, t0, dt, nsteps, seg
        ctx.multirate = multirate
        ctx.taped = taped
        ctx.ckpts = ckpts
        ctx.scale_shape, ctx.scale_dtype = scale.shape, scale.dtype
        return out

    @staticmethod
    def backward(ctx, grad_out):
        F, t0, dt, n, seg = ctx.forest, ctx.t0, ctx.dt, ctx.nsteps, ctx.seg
        lam = grad_out.contiguous().clone()
        dscale = torch.zeros(1, dtype=torch.float64, device=lam.device)
        if ctx.taped:  # every step was recorded by the forward pass
            if getattr(F, "_tape_run", None) != ctx.tape_run:
                raise RuntimeError("the forest's tapes were recorded again by a later taped "
                                   "advect; run this backward first or use tape='recompute'")
            for k in range(n - 1, -1, -1):
                F.adjoint_step_multirate_taped(t0 + k * dt, dt, k, lam, dscale)
            gscale = dscale.to(ctx.scale_dtype).reshape(ctx.scale_shape)
            return lam, gscale, None, None, None, None, None, None, None
        if ctx.multirate:
            for start in sorted(ctx.ckpts, reverse=True):
                end = min(start + seg, n)
                F.set_q(ctx.ckpts[start])
                for k in range(start, end):
                    F.step_multirate_record(t0 + k * dt, dt, k - start)
                for k in range(end - 1, start - 1, -1):
                    F.adjoint_step_multirate_taped(t0 + k * dt, dt, k - start, lam, dscale)
            ctx.ckpts = None
            gscale = dscale.to(ctx.scale_dtype).reshape(ctx.scale_shape)
            return lam, gscale, None, None, None, None, None, None, None
        for start in sorted(ctx.ckpts, reverse=True):
            end = min(start + seg, n)
            F.set_q(ctx.ckpts[start])
            states = []
            for k in range(start, end):
                s = torch.empty_like(lam)
                F.get_q(out=s)
                states.append(s)
                if k < end - 1:
                    F.step_global(t0 + k * dt, dt)
            for k in range(end - 1, start - 1, -1):
                F.set_q(states[k - start])
                F.adjoint_step_global(t0 + k * dt, dt, lam, dscale)
        ctx.ckpts = None
        gscale = dscale.to(ctx.scale_dtype).reshape(ctx.scale_shape)
        return lam, gscale, None, None, None, None, None, None, None


def advect(q0: torch.Tensor, scale: torch.Tensor, forest, t0: float, dt: float, nsteps: int,
           segment: int = 0, multirate: bool = False, tape: str = "auto") -> torch.Tensor:
    """Differentiable N-step advance of ``forest`` (see module docstring).
    tape: "forward" (record every step in the forward pass; multirate, at
    most MAX_TAPE_SLOTS steps), "recompute" (sqrt(N) checkpoints), or
    "auto" (forward when allowed and no segment length is given)."""
    if tape == "auto":
        tape = ("forward" if multirate and nsteps <= MAX_TAPE_SLOTS and not segment
                else "recompute")
    if tape == "forward" and not (multirate and nsteps <= MAX_TAPE_SLOTS):
        raise ValueError("tape='forward' needs multirate steps, at most %d" % MAX_TAPE_SLOTS)
    return _Advect.apply(q0, scale, forest, t0, dt, nsteps, segment, multirate, tape)
