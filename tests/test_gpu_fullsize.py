"""Parity at the benchmark sizes, in the launch configuration bench.py times (GPU only).

* 1M-node mesh, C = 512, pipelined kernel with the bench's defaults: schedule,
  vertex lists, relabel and cost bit-exact with the oracle; 10 explicit steps
  and the 10-step adjoint, both through ep_run_adjoint and through the
  checkpointed autograd function (every 5 steps), against the FP64 oracle.
* R-MAT scale 20, C = 512, bipartite: full SpMV (staged x and read-only
  cache) against the FP64 oracle; the
  schedule is checked through properties that hold at any size (exact block
  sizes, each task once, GPU cost = host cost = loads recomputed from the
  vertex lists); the oracle partition itself is too slow for this size.
* 512 uneven meshes (batched, one launch per kernel) with the autotuner's C
  and kernel: 20 steps forward and backward (checkpoint every 10) captured in
  one CUDA graph and replayed; x_T, dL/dx0 and dL/dw of 8 sampled meshes
  (the smallest, the largest and 6 more) against the oracle mesh by mesh.
FP32 results: parity.py (relative L2 <= 1e-5 and element-wise bounds).
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
from parity import check_field, check_state  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.fixture(scope="module")
def mesh1m():
    n = 1 << 20
    src, dst = W.knn_mesh(n, 4, 0)
    S = E.Schedule.partition(src, dst, n, 512)
    return n, src, dst, S


@pytest.fixture(scope="module")
def mesh1m_oracle(mesh1m):
    n, src, dst, S = mesh1m
    x0 = W.flux_state(n, 5, 0)
    w = W.flux_weights(src.size, 0)
    g = W.loss_weights(n, 5, 1)
    T, tau = 10, 1e-3
    xT, fT = O.flux_steps(src, dst, x0, w, T, tau)
    dx, dw = O.flux_adjoint(src, dst, x0, w, T, tau, g)
    return dict(x0=x0, w=w, g=g, T=T, tau=tau, xT=xT, fT=fT, dx=dx, dw=dw)


def test_mesh1m_schedule_bit_exact(mesh1m):
    n, src, dst, S = mesh1m
    ref = O.ep_schedule(src, dst, n, 512)
    a = S.arrays()
    for key in ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel"):
        assert np.array_equal(a[key], ref[key]), key
    assert S.cost() == (ref["loads"], ref["cut"])
    d = O.ep_schedule(src, dst, n, 512, default_order=True)
    assert ref["loads"] < 0.5 * d["loads"]


def test_mesh1m_forward_and_adjoint(mesh1m, mesh1m_oracle):
    n, src, dst, S = mesh1m
    r = mesh1m_oracle
    S.set_pipeline(3)
    S.set_threads(256)
    x = cuda(r["x0"])
    out = torch.zeros_like(x)
    S.run(x, cuda(r["w"]), out, steps=r["T"], tau=r["tau"])
    check_state(x, r["xT"], r["x0"], r["T"], "x")
    check_field(out, r["fT"], "out")
    lam = cuda(r["g"])
    gw = torch.zeros(src.size, device="cuda")
    S.run_adjoint(cuda(r["x0"]), cuda(r["w"]), lam, gw, steps=r["T"], tau=r["tau"])
    check_state(lam, r["dx"], r["g"], r["T"], "dx0")
    check_field(gw, r["dw"], "dw")
    assert S.check_errors() == 0


def test_mesh1m_autograd_checkpointed(mesh1m, mesh1m_oracle):
    from paper_1605_02043_gb300.autograd import flux_steps

    n, src, dst, S = mesh1m
    r = mesh1m_oracle
    S.set_pipeline(3)
    S.set_threads(256)
    x = cuda(r["x0"]).requires_grad_(True)
    w = cuda(r["w"]).requires_grad_(True)
    xT = flux_steps(x, w, S, r["T"], r["tau"], 5)
    xT.backward(cuda(r["g"]))
    check_state(xT, r["xT"], r["x0"], r["T"], "xT")
    check_state(x.grad, r["dx"], r["g"], r["T"], "dx0")
    check_field(w.grad, r["dw"], "dw")
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
    ref = O.spmv(rows, cols, x0, w, n)
    for dflt in (False, True):
        Sx = S if not dflt else E.Schedule.partition(rows, cols, n, 512, bipartite=True, default_order=True)
        Sx.set_threads(192)
        for cache in (E.CACHE_SMEM, E.CACHE_L1):
            Sx.set_cache(cache)
            y = torch.empty(n, device="cuda")
            Sx.run(cuda(x0), cuda(w), y, kernel=E.SPMV)
            check_field(y, ref, f"y default_order={dflt} cache={cache}")


def test_batch512_cuda_graph_fwd_bwd_autotuned():
    from paper_1605_02043_gb300 import autotune
    from paper_1605_02043_gb300.autograd import FluxRunner

    graphs = W.batch_meshes(512)
    parts_by_C = {}
    tuned = autotune.tune(graphs, D=5, partitions=parts_by_C)
    parts = parts_by_C.get(tuned["C"]) or autotune.partition_many(graphs, tuned["C"])
    B = E.Schedule.batch(parts)
    B.set_pipeline(tuned["stages"])
    B.set_threads(tuned["threads"])
    N, M = B.n, B.m
    T, tau, every = 20, 1e-3, 10
    x0 = W.flux_state(N, 5, 0)
    w = W.flux_weights(M, 0)
    g = W.loss_weights(N, 5, 1)
    R = FluxRunner(B, 5, T, tau, every)
    R.load(cuda(x0), cuda(w), cuda(g))
    R.run()  # warm-up outside the capture (allocates the library workspace)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        R.run()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert B.check_errors() == 0
    xT, dx, dw = (t.cpu().numpy() for t in R.results(cuda(x0), M))
    offs_n = np.cumsum([0] + [gr[0] for gr in graphs])
    offs_m = np.cumsum([0] + [p.m for p in parts])
    sizes = np.array([gr[0] for gr in graphs])
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    pick |= {int(i) for i in np.random.default_rng(3).choice(512, 6, replace=False)}
    for i in sorted(pick):
        n_i, s_i, d_i = graphs[i]
        lo, hi, mlo, mhi = offs_n[i], offs_n[i + 1], offs_m[i], offs_m[i + 1]
        xr, _ = O.flux_steps(s_i, d_i, x0[:, lo:hi], w[mlo:mhi], T, tau)
        dxr, dwr = O.flux_adjoint(s_i, d_i, x0[:, lo:hi], w[mlo:mhi], T, tau, g[:, lo:hi])
        check_state(xT[:, lo:hi], xr, x0[:, lo:hi], T, f"mesh {i} xT")
        check_state(dx[:, lo:hi], dxr, g[:, lo:hi], T, f"mesh {i} dx0")
        check_field(dw[mlo:mhi], dwr, f"mesh {i} dw")
