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


def test_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The bench takes ncu traffic from profiles/traffic.json only while the
    kernel sources hash to the recorded value."""
    import json
    import shutil

    import bench

    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1605_02043_gb300", "csrc"),
                    root / "paper_1605_02043_gb300" / "csrc")
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.kernel_sources_sha()
    rec = {"k": {"kernel_sources_sha": sha, "dram_bytes_per_launch": 123},
           "old": {"kernel_sources_sha": "0" * 16, "dram_bytes_per_launch": 456}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.traffic("k") == 123
    assert bench.traffic("old") is None and bench.traffic("missing") is None
    with open(root / "paper_1605_02043_gb300" / "csrc" / "kernels.cu", "a") as fh:
        fh.write("\n// changed\n")
    assert bench.kernel_sources_sha() != sha and bench.traffic("k") is None
