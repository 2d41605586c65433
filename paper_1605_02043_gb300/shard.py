"""Splitting one schedule over G GPUs, and its halo exchange (host logic).

The recursive bisection that builds a schedule numbers its blocks in leaf
order, so the top log2(G) levels of that recursion are G contiguous ranges
of blocks: shard g takes blocks [lo_g, hi_g).  Those levels are the ones the
partitioner cut with the fewest auxiliary edges, and by the argument of
Theorem 1 the number of replicated data vertices between shards, the
exchange volume, is at most that cut.

A vertex touched by blocks of more than one shard is a halo vertex.  One
explicit step on G GPUs is then: every shard accumulates the interactions
of its own tasks (`out` partial sums); the partial sums of the halo vertices
are summed over shards (one all-reduce of a D x |halo| buffer, which is the
reduce and the broadcast of the halo values in one collective); every shard
applies x += tau * out to the vertices it touches.  Vertices outside the
shard are never read by it, so their copies may go stale.

Shard g runs its tasks as an ordinary schedule: its slice of the task order
(edge_perm[block_ptr[lo_g] : block_ptr[hi_g]]) in default order with the
same C reproduces its blocks exactly, because every block but the last holds
exactly C tasks.  This module holds the split, the halo lists and the
exchange; one process per GPU is the launch model, and the tests run the
exchange with CPU ranks over gloo.
"""
from __future__ import annotations

import numpy as np


def shard_blocks(k: int, G: int) -> list[tuple[int, int]]:
    """Block ranges of G shards: the top log2(G) levels of the bisection
    (left part ceil(k'/2) blocks, as in the partitioner).  G is a power of two, <= k."""
    if G < 1 or G & (G - 1):
        raise ValueError(f"G = {G} must be a power of two")
    if G > k:
        raise ValueError(f"G = {G} exceeds the {k} blocks")
    ranges = [(0, k)]
    while len(ranges) < G:
        nxt = []
        for lo, hi in ranges:
            mid = lo + (hi - lo + 1) // 2
            nxt += [(lo, mid), (mid, hi)]
        ranges = nxt
    return ranges


class Halo:
    """Shards of schedule arrays `a` (Schedule.arrays()) over G GPUs."""

    def __init__(self, a: dict, G: int):
        self.G = G
        self.k = int(a["k"])
        self.ranges = shard_blocks(self.k, G)
        bp, ep = a["block_ptr"], a["edge_perm"]
        vp, vl = a["vert_ptr"], a["vert_list"]
        nd = a["relabel"].size
        self.tasks = [ep[bp[lo]:bp[hi]] for lo, hi in self.ranges]
        self.verts = [np.unique(vl[vp[lo]:vp[hi]]) for lo, hi in self.ranges]
        count = np.zeros(nd, np.int64)
        for v in self.verts:
            count[v] += 1
        self.ids = np.flatnonzero(count > 1).astype(np.int64)  # halo vertices, ascending
        self.volume = int((count[self.ids] - 1).sum())  # replicated partial sums
        self.shard_halo = [np.intersect1d(v, self.ids) for v in self.verts]

    def edges(self, g: int, src, dst):
        """Task list of shard g in schedule order (default order with the same C
        gives back its blocks)."""
        t = self.tasks[g]
        return np.asarray(src)[t], np.asarray(dst)[t], t

    def exchange(self, out, group=None):
        """Sum the halo columns of a (D, n) partial-sum tensor over all ranks, in place."""
        import torch
        import torch.distributed as dist

        if self.ids.size == 0:
            return out
        idx = torch.as_tensor(self.ids, device=out.device)
        buf = out.index_select(1, idx).contiguous()
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        out.index_copy_(1, idx, buf)
        return out

    def bytes_per_step(self, D: int) -> int:
        """Halo values one all-reduce moves per rank (4 D bytes per halo vertex)."""
        return 4 * D * int(self.ids.size)


class ShardedFlux:
    """Explicit flux steps of one schedule split over shards, on GPUs.

    Shard g is the default-order schedule of its slice of the task order (it
    reproduces blocks [lo_g, hi_g) exactly) with the halo declared
    (`Schedule.set_halo`), so the sums of halo vertices stay in accumulator
    records.  One step: every shard runs its edge kernel (one launch, shared
    copies pending), packs its halo sums into a D x |halo| buffer, the buffers
    are summed over shards by `reduce`, and every shard unpacks the global
    sums, which its next step (or `finish`) applies to its copies.

    `shards` lists the shard ids this process runs (all of them on one device,
    or one per process); `reduce(bufs)` sums the listed shards' buffers over
    every shard in place: the default sums them on the device (one process
    holds every shard), across processes it is an all-reduce of the local sum.
    """

    def __init__(self, sched, src, dst, n: int, D: int, G: int, shards=None, reduce=None):
        import torch
        from . import Schedule

        self.D, self.n, self.G = D, n, G
        self.halo = Halo(sched.arrays(), G)
        self.mine = list(range(G)) if shards is None else list(shards)
        self.reduce = reduce or _sum_on_device
        self.S, self.tasks = [], []
        for g in self.mine:
            s_, d_, t = self.halo.edges(g, src, dst)
            S = Schedule.partition(s_, d_, n, sched.C, default_order=True)
            S.set_halo(self.halo.ids)
            self.S.append(S)
            self.tasks.append(torch.as_tensor(t, dtype=torch.int64, device="cuda"))
        f32 = dict(device="cuda", dtype=torch.float32)
        self.xl = [torch.zeros(S.layout_floats(D), **f32) for S in self.S]
        self.wl = [torch.zeros(S.weights_floats(), **f32) for S in self.S]
        self.buf = [torch.zeros(self.halo.ids.size, D, **f32) for _ in self.S]

    def load(self, x, w):
        """Global state x (D x n) and task weights w (m), device tensors."""
        for S, xl, wl, t in zip(self.S, self.xl, self.wl, self.tasks):
            S.layout_in(x.contiguous(), xl)
            S.weights_in(w.index_select(0, t).contiguous(), wl)

    def step(self, tau: float = 1e-3):
        for S, xl, wl, buf in zip(self.S, self.xl, self.wl, self.buf):
            S.step(self.D, xl, xl, wl, None, tau, pending=True)
            S.halo_pack(self.D, buf)
        self.reduce(self.buf)
        for S, buf in zip(self.S, self.buf):
            S.halo_unpack(self.D, buf)

    def finish(self, tau: float = 1e-3):
        for S, xl in zip(self.S, self.xl):
            S.finish(self.D, xl, tau)

    def gather(self, x):
        """Writes the vertices of this process's shards into x (D x n, device)."""
        import torch

        tmp = torch.empty_like(x)
        for g, S, xl in zip(self.mine, self.S, self.xl):
            S.layout_out(xl, tmp)
            v = torch.as_tensor(self.halo.verts[g], dtype=torch.int64, device=x.device)
            x.index_copy_(1, v, tmp.index_select(1, v))
        return x


def allreduce_sum(group=None):
    """`reduce` for one process per GPU (or several shards per process): the
    local buffers are summed, one all-reduce sums over processes, and every
    local buffer takes the result."""
    import torch.distributed as dist

    def reduce(bufs):
        total = bufs[0].clone()
        for b in bufs[1:]:
            total += b
        dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
        for b in bufs:
            b.copy_(total)

    return reduce


def _sum_on_device(bufs):
    """Every shard on this device: each buffer becomes the sum of all of them."""
    total = bufs[0].clone()
    for b in bufs[1:]:
        total += b
    for b in bufs:
        b.copy_(total)

