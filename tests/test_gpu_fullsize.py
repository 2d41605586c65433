"""Parity at the benchmark sizes, in the launch configuration bench.py times (GPU only).

* 1M-node mesh, C = 512, pipelined kernel with the bench's defaults: schedule,
  vertex lists, relabel and cost bit-exact with the oracle; 10 explicit steps
  and the 10-step adjoint within 1e-5 relative L2 of the FP64 oracle.
* R-MAT scale 20, C = 512, bipartite: full SpMV against the FP64 oracle; the
  schedule is checked through properties that hold at any size (exact block
  sizes, each task once, GPU cost = host cost = loads recomputed from the
  vertex lists); the oracle partition itself is too slow for this size.
* 512 uneven meshes (batched, one launch): every 64th mesh checked one by one
  against the oracle after 3 steps.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_02043_gb300 as E  # noqa: E402

RTOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.fixture(scope="module")
def mesh1m():
    n = 1 << 20
    src, dst = W.knn_mesh(n, 4, 0)
    S = E.Schedule.partition(src, dst, n, 512)
    return n, src, dst, S


def test_mesh1m_schedule_bit_exact(mesh1m):
    n, src, dst, S = mesh1m
    ref = O.ep_schedule(src, dst, n, 512)
    a = S.arrays()
    for key in ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel"):
        assert np.array_equal(a[key], ref[key]), key
    assert S.cost() == (ref["loads"], ref["cut"])
    d = O.ep_schedule(src, dst, n, 512, default_order=True)
    assert ref["loads"] < 0.5 * d["loads"]


def test_mesh1m_forward_and_adjoint(mesh1m):
    n, src, dst, S = mesh1m
    S.set_pipeline(3)
    S.set_threads(256)
    x0 = W.flux_state(n, 5, 0)
    w = W.flux_weights(src.size, 0)
    T, tau = 10, 1e-3
    x = cuda(x0)
    out = torch.zeros_like(x)
    S.run(x, cuda(w), out, steps=T, tau=tau)
    xT, fT = O.flux_steps(src, dst, x0, w, T, tau)
    assert rel_l2(x.cpu().numpy(), xT) <= RTOL
    assert rel_l2(out.cpu().numpy(), fT) <= RTOL
    g = W.loss_weights(n, 5, 1)
    lam = cuda(g)
    gw = torch.zeros(src.size, device="cuda")
    S.run_adjoint(cuda(x0), cuda(w), lam, gw, steps=T, tau=tau)
    dx, dw = O.flux_adjoint(src, dst, x0, w, T, tau, g)
    assert rel_l2(lam.cpu().numpy(), dx) <= RTOL
    assert rel_l2(gw.cpu().numpy(), dw) <= RTOL
    assert S.check_errors() == 0


def test_rmat20_spmv_and_schedule_properties():
    rows, cols = W.rmat()
    n, m = 1 << 20, rows.size
    S = E.Schedule.partition(rows, cols, n, 512, bipartite=True)
    a = S.arrays()
    sizes = np.diff(a["block_ptr"])
    assert np.all(sizes[:-1] == 512) and 0 < sizes[-1] <= 512
    assert np.array_equal(np.sort(a["edge_perm"]), np.arange(m))
    loads, cut = S.cost()
    assert (loads, cut) == S.cost_host() == (a["loads"], a["cut"])
    # loads recomputed from the task lists of every block
    u = (n + rows.astype(np.int64))[a["edge_perm"]]
    v = cols.astype(np.int64)[a["edge_perm"]]
    blk = np.repeat(np.arange(S.k, dtype=np.int64), sizes)
    keys = np.unique(np.concatenate([blk * (2 * n) + u, blk * (2 * n) + v]))
    assert keys.size == loads
    x0, w = W.spmv_inputs(n, m, 0)
    y = torch.empty(n, device="cuda")
    S.run(cuda(x0), cuda(w), y, kernel=E.SPMV)
    assert rel_l2(y.cpu().numpy(), O.spmv(rows, cols, x0, w, n)) <= RTOL


def test_batch512_sampled_meshes():
    from paper_1605_02043_gb300 import autotune

    graphs = W.batch_meshes(512)
    parts = autotune.partition_many(graphs, 256)
    B = E.Schedule.batch(parts)
    N = sum(g[0] for g in graphs)
    x0 = W.flux_state(N, 5, 0)
    w = W.flux_weights(B.m, 0)
    x = cuda(x0)
    B.run(x, cuda(w), None, steps=3, tau=1e-3)
    xg = x.cpu().numpy()
    offs_n = np.cumsum([0] + [g[0] for g in graphs])
    offs_m = np.cumsum([0] + [p.m for p in parts])
    for i in range(0, 512, 64):
        n_i, s_i, d_i = graphs[i]
        lo, hi = offs_n[i], offs_n[i + 1]
        xT, _ = O.flux_steps(s_i, d_i, x0[:, lo:hi], w[offs_m[i]:offs_m[i + 1]], 3, 1e-3)
        assert rel_l2(xg[:, lo:hi], xT) <= RTOL, i
