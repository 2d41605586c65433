"""torch.autograd.Function over T explicit flux steps on one schedule.

Forward keeps the state in the schedule's layout, stores a checkpoint every
`every` steps and returns x_T in the caller's layout.  Backward walks the
checkpoints in reverse: it recomputes the states of one segment with the
forward kernel, then runs the hand-written adjoint kernel (same schedule, same
access pattern) step by step back to the checkpoint.  Gradients flow to x0 and
to the task weights w.  Steps leave the copies of shared vertices pending
(one launch per step); a state is finished where it is stored or read whole
(checkpoints, recomputed states, the results).
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
                if t:
                    sched.finish(D, xl, tau)
                ckpts.append(xl.clone())
            sched.step(D, xl, xl, wl, None, tau, pending=True)
        sched.finish(D, xl, tau)
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
                sched.adjoint_step(D, states[t], wl, lam, gwl, tau, pending=True)
        sched.adjoint_finish(D, lam, tau)
        dx0 = torch.empty_like(g)
        sched.layout_out(lam, dx0)
        dw = torch.zeros(sched.m, device=g.device, dtype=torch.float32)
        sched.weights_out_add(gwl, dw)
        return dx0, dw, None, None, None, None


def flux_steps(x0, w, sched: Schedule, steps: int, tau: float = 1e-3, every: int = 5):
    """x_T after `steps` explicit flux steps, differentiable in x0 and w."""
    return FluxSteps.apply(x0, w, sched, steps, tau, every)


class FluxRunner:
    """Forward and backward over `steps` flux steps with preallocated buffers.

    Everything lives in the schedule's layout, so one call of run() only
    enqueues kernels (and device copies) on the current stream and can be
    captured in a CUDA graph after one warm-up run: forward steps with a
    checkpoint every `every` steps, then for every segment in reverse a
    recompute of its states and the adjoint steps.  load() sets x0, w and the
    loss cotangent g; results() returns dL/dx0 and dL/dw.
    """

    def __init__(self, sched: Schedule, D: int, steps: int, tau: float = 1e-3, every: int = 5,
                 device="cuda"):
        self.s, self.D, self.steps, self.tau, self.every = sched, D, steps, tau, every
        nl, nw = sched.layout_floats(D), sched.weights_floats()
        f32 = dict(device=device, dtype=torch.float32)
        self.x0l = torch.zeros(nl, **f32)
        self.gl = torch.zeros(nl, **f32)
        self.xl = torch.zeros(nl, **f32)
        self.lam = torch.zeros(nl, **f32)
        self.wl = torch.zeros(nw, **f32)
        self.gwl = torch.zeros(nw, **f32)
        nseg = (steps + every - 1) // every
        self.ckpt = [torch.zeros(nl, **f32) for _ in range(nseg)]
        self.hist = [torch.zeros(nl, **f32) for _ in range(max(every - 1, 0))]

    def load(self, x0, w, g):
        self.s.layout_in(x0.contiguous(), self.x0l)
        self.s.weights_in(w.contiguous(), self.wl)
        self.s.layout_in(g.contiguous(), self.gl)

    def forward(self):
        s, D, tau = self.s, self.D, self.tau
        self.xl.copy_(self.x0l)
        for t in range(self.steps):
            if t % self.every == 0:
                if t:
                    s.finish(D, self.xl, tau)
                self.ckpt[t // self.every].copy_(self.xl)
            s.step(D, self.xl, self.xl, self.wl, None, tau, pending=True)
        s.finish(D, self.xl, tau)

    def backward(self):
        s, D, tau = self.s, self.D, self.tau
        self.lam.copy_(self.gl)
        self.gwl.zero_()
        for seg in range(len(self.ckpt) - 1, -1, -1):
            T = min(self.every, self.steps - seg * self.every)
            states = [self.ckpt[seg]] + self.hist[: T - 1]
            for t in range(T - 1):
                s.step(D, states[t], states[t + 1], self.wl, None, tau)
            for t in range(T - 1, -1, -1):
                s.adjoint_step(D, states[t], self.wl, self.lam, self.gwl, tau, pending=True)
        s.adjoint_finish(D, self.lam, tau)

    def run(self):
        self.forward()
        self.backward()

    def results(self, x_like, m: int):
        xT = torch.empty_like(x_like)
        self.s.layout_out(self.xl, xT)
        dx0 = torch.empty_like(x_like)
        self.s.layout_out(self.lam, dx0)
        dw = torch.zeros(m, device=x_like.device, dtype=torch.float32)
        self.s.weights_out_add(self.gwl, dw)
        return xT, dx0, dw
