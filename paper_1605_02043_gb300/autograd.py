"""torch.autograd.Function over T explicit flux steps on one schedule.

Forward keeps the state in the schedule's layout, stores a checkpoint every
`every` steps and returns x_T in the caller's layout.  Backward walks the
checkpoints in reverse: it recomputes the states of one segment with the
forward kernel, then runs the hand-written adjoint kernel (same schedule, same
access pattern) step by step back to the checkpoint.  Gradients flow to x0 and
to the task weights w.
"""
from __future__ import annotations

import torch

from . import Schedule


class FluxSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, w, sched: Schedule, steps: int, tau: float, every: int):
        D = int(x0.shape[0])
        x0 = x0.contiguous()
        w = w.contiguous()
        xl = torch.empty(sched.layout_floats(D), device=x0.device, dtype=torch.float32)
        wl = torch.empty(sched.weights_floats(), device=x0.device, dtype=torch.float32)
        sched.layout_in(x0, xl)
        sched.weights_in(w, wl)
        ckpts = []
        for t in range(steps):
            if t % every == 0:
                ckpts.append(xl.clone())
            sched.step(D, xl, xl, wl, None, tau)
        xT = torch.empty_like(x0)
        sched.layout_out(xl, xT)
        ctx.sched, ctx.steps, ctx.tau, ctx.every, ctx.D = sched, steps, tau, every, D
        ctx.save_for_backward(wl, *ckpts)
        return xT

    @staticmethod
    def backward(ctx, g):
        sched, steps, tau, every, D = ctx.sched, ctx.steps, ctx.tau, ctx.every, ctx.D
        wl, *ckpts = ctx.saved_tensors
        g = g.contiguous()
        lam = torch.empty_like(ckpts[0])
        sched.layout_in(g, lam)
        gwl = torch.zeros_like(wl)
        hist = [torch.empty_like(ckpts[0]) for _ in range(max(every - 1, 0))]
        for seg in range(len(ckpts) - 1, -1, -1):
            t0 = seg * every
            T = min(every, steps - t0)
            states = [ckpts[seg]] + hist[: T - 1]
            for t in range(T - 1):
                sched.step(D, states[t], states[t + 1], wl, None, tau)
            for t in range(T - 1, -1, -1):
                sched.adjoint_step(D, states[t], wl, lam, gwl, tau)
        dx0 = torch.empty_like(g)
        sched.layout_out(lam, dx0)
        dw = torch.zeros(sched.m, device=g.device, dtype=torch.float32)
        sched.weights_out_add(gwl, dw)
        return dx0, dw, None, None, None, None


def flux_steps(x0, w, sched: Schedule, steps: int, tau: float = 1e-3, every: int = 5):
    """x_T after `steps` explicit flux steps, differentiable in x0 and w."""
    return FluxSteps.apply(x0, w, sched, steps, tau, every)
