"""bench.py's multi-rank logic (replicas, max over ranks) with CPU ranks over
gloo: every rank sees the maximum time, and the whole-job value counts every
rank's tasks.  No GPU needed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_info()
        bench.barrier(torch)
        t = bench.max_over_ranks(torch, 10.0 + rank)  # rank r took 10 + r ms
        m = 1000  # tasks per replica
        q.put((r, ws, local, t, ws * m / (1e-3 * t)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_with_gloo(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    slowest = 10.0 + world - 1
    for r, (rank, ws, local, t, value) in enumerate(res):
        assert (rank, ws, local) == (r, world, r)
        assert t == slowest
        assert value == pytest.approx(world * 1000 / (1e-3 * slowest))
