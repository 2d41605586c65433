"""Multi-GPU split of one schedule (shard.py): block ranges from the top
levels of the bisection, halo lists, and the halo exchange run with CPU
ranks over gloo (world sizes 2 and 4).  Each rank computes its partial sums
with the oracle's edge kernel (the GPU kernel is the single-GPU one); what
is tested is the split and the exchange.  No GPU needed."""
import os
import socket

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1605_02043_gb300 as E
from paper_1605_02043_gb300.shard import Halo, shard_blocks

torch = pytest.importorskip("torch")


def test_shard_blocks_follow_the_bisection():
    assert shard_blocks(7, 1) == [(0, 7)]
    assert shard_blocks(7, 2) == [(0, 4), (4, 7)]
    assert shard_blocks(7, 4) == [(0, 2), (2, 4), (4, 6), (6, 7)]
    assert shard_blocks(8, 8) == [(i, i + 1) for i in range(8)]
    for bad in ((7, 3), (3, 4), (5, 0)):
        with pytest.raises(ValueError):
            shard_blocks(*bad)


def test_recursion_tree_matches_partition_sizes():
    # the partitioner's left subtree holds ceil(k/2) * C tasks exactly
    src, dst = W.knn_mesh(2000, 4, 3)
    S = E.Schedule.partition(src, dst, 2000, 100)
    a = S.arrays()
    for lo, hi in shard_blocks(S.k, 4):
        assert a["block_ptr"][hi] - a["block_ptr"][lo] == min(hi * 100, src.size) - lo * 100


@pytest.fixture(scope="module")
def case():
    n = 3000
    src, dst = W.knn_mesh(n, 4, 5)
    C = -(-src.size // 8)  # k = 8
    S = E.Schedule.partition(src, dst, n, C)
    assert S.k == 8
    return n, src, dst, C, S.arrays(), S


def brute_volume(src, dst, shards):
    """Sum over data vertices of (number of shards whose tasks touch it - 1)."""
    touched = [set(np.concatenate([src[t], dst[t]]).tolist()) for t in shards]
    allv = set().union(*touched)
    return sum(sum(v in T for T in touched) - 1 for v in allv)


def aux_cut_between(src, dst, n, shard_of_task):
    """Auxiliary edges of the clone-and-connect graph (Def. 3) joining tasks of
    different shards: per vertex, consecutive incident tasks in index order."""
    cut = 0
    inc = [[] for _ in range(n)]
    for e, (u, v) in enumerate(zip(src.tolist(), dst.tolist())):
        inc[u].append(e)
        if v != u:
            inc[v].append(e)
    for lst in inc:
        cut += sum(shard_of_task[a] != shard_of_task[b] for a, b in zip(lst, lst[1:]))
    return cut


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_halo_volume(case, G):
    n, src, dst, C, a, S = case
    Hl = Halo(a, G)
    assert Hl.volume == brute_volume(src, dst, Hl.tasks)
    owner = np.empty(src.size, np.int64)
    for g, t in enumerate(Hl.tasks):
        owner[t] = g
    assert Hl.volume <= aux_cut_between(src, dst, n, owner)  # Theorem 1's argument
    if G == 1:
        assert Hl.ids.size == 0
    if G == 8:  # one block per shard: the schedule's own vertex cut (Eq. 1)
        assert Hl.volume == S.cost_host()[1]
    for g in range(G):
        assert np.array_equal(np.sort(Hl.shard_halo[g]), Hl.shard_halo[g])
        assert np.isin(Hl.shard_halo[g], Hl.verts[g]).all()


def test_partitioned_split_exchanges_less_than_default(case):
    n, src, dst, C, a, S = case
    d = E.Schedule.partition(src, dst, n, C, default_order=True).arrays()
    assert Halo(a, 2).volume < Halo(d, 2).volume


def test_shard_default_order_reproduces_its_blocks(case):
    n, src, dst, C, a, S = case
    Hl = Halo(a, 4)
    for g, (lo, hi) in enumerate(Hl.ranges):
        s, d, t = Hl.edges(g, src, dst)
        b = E.Schedule.partition(s, d, n, C, default_order=True).arrays()
        vp, vl = a["vert_ptr"], a["vert_list"]
        assert np.array_equal(b["block_ptr"], a["block_ptr"][lo:hi + 1] - a["block_ptr"][lo])
        assert np.array_equal(b["vert_list"], vl[vp[lo]:vp[hi]])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, src, dst, x0, w, C, steps, tau, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S = E.Schedule.partition(src, dst, n, C)
        Hl = Halo(S.arrays(), world)
        s, d, t = Hl.edges(rank, src, dst)
        mine = Hl.verts[rank]
        x = torch.from_numpy(np.array(x0, np.float64))
        for _ in range(steps):
            out = torch.from_numpy(O.flux(s, d, x.numpy(), w[t]))  # partial sums of my tasks
            Hl.exchange(out)
            x[:, mine] += tau * out[:, mine]
        xT, _ = O.flux_steps(src, dst, x0, w, steps, tau)
        err = np.abs(x.numpy()[:, mine] - xT[:, mine]).max()
        q.put((rank, float(err), int(mine.size)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_halo_exchange_with_gloo_ranks(world):
    import torch.multiprocessing as mp

    n = 1500
    src, dst = W.knn_mesh(n, 4, 9)
    x0 = W.flux_state(n, 5, 0).astype(np.float64)
    w = W.flux_weights(src.size, 0).astype(np.float64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main,
                         args=(r, world, port, n, src, dst, x0, w, 128, 3, 1e-3, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert sorted(r for r, _, _ in res) == list(range(world))
    assert sum(c for _, _, c in res) >= n  # the shards cover every vertex
    for _, err, _ in res:
        assert err <= 1e-12


def _reduce_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_1605_02043_gb300.shard import allreduce_sum

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # two shards per rank: buffers rank * 10 + j
        bufs = [torch.full((3, 5), float(rank * 10 + j)) for j in range(2)]
        allreduce_sum()(bufs)
        q.put((rank, [float(b[0, 0]) for b in bufs], [float(b.sum()) for b in bufs]))
    finally:
        dist.destroy_process_group()


def test_allreduce_sum_of_shard_buffers():
    """The multi-process exchange: every local buffer ends as the sum over all shards."""
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    want = float(sum(r * 10 + j for r in range(world) for j in range(2)))  # 0 + 1 + 10 + 11
    for _, firsts, sums in res:
        assert firsts == [want, want] and sums == [15 * want, 15 * want]


def test_set_halo_keeps_the_schedule():
    """ep_set_halo rebuilds only the flux layout: schedule arrays and cost stay."""
    import paper_1605_02043_gb300 as E

    src, dst = W.knn_mesh(4096, 4, 0)
    S = E.Schedule.partition(src, dst, 4096, 256)
    before = S.arrays()
    cost = S.cost_host()
    S.set_halo(np.array([0, 17, 17, 4095], np.int32))
    after = S.arrays()
    for key in ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel"):
        assert np.array_equal(before[key], after[key]), key
    assert S.cost_host() == cost
    S.set_halo(np.array([], np.int32))
    for bad in ([-1], [4096]):
        with pytest.raises(E.EpError) as ei:
            S.set_halo(np.array(bad, np.int32))
        assert ei.value.code == -1
    r, c = W.rmat(scale=10, m_draws=1 << 12, seed=1)
    B = E.Schedule.partition(r, c, 1 << 10, 64, bipartite=True)
    with pytest.raises(E.EpError):
        B.set_halo(np.array([0], np.int32))

