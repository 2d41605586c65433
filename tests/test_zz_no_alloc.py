"""ep_cost_noalloc: the load count for callers that cannot allocate (GPU only).

Some callers cannot let a library call cudaMalloc: code that runs while a
stream is captured into a CUDA graph, applications that own all device memory
through their own pool, and loops that cannot take an allocation's implicit
synchronisation.  ep_cost_noalloc() serves them: the caller passes every input
and output as device memory and the only scratch is a fixed device array in
the library.  This test checks it against ep_cost(), which allocates its own
workspace, on two calls in a row (the shared scratch keeps the previous
call's flags, so the second call shows that they are cleared).  It sits in a
file of its own, named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_02043_gb300 as E  # noqa: E402
from paper_1605_02043_gb300 import _lib  # noqa: E402


def device_inputs(S, src, dst, bipartite):
    """Caller-owned device arrays of a schedule: block_ptr, endpoints in schedule order."""
    a = S.arrays()
    ep = a["edge_perm"]
    eu = (src[ep].astype(np.int64) + (S.n if bipartite else 0)).astype(np.int32)
    ev = dst[ep].astype(np.int32)
    sizes = np.diff(a["block_ptr"])
    return (torch.from_numpy(a["block_ptr"]).cuda(), torch.from_numpy(eu).cuda(),
            torch.from_numpy(ev).cuda(), int(sizes.max()))


def call_noalloc(bp, eu, ev, k, nd, max_ne, counts):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.lib().ep_cost_noalloc(ctypes.c_void_p(bp.data_ptr()), ctypes.c_void_p(eu.data_ptr()),
                                      ctypes.c_void_p(ev.data_ptr()), k, nd, max_ne,
                                      ctypes.c_void_p(counts.data_ptr()), stream)


def test_noalloc_cost_matches_allocating_entry_point_twice():
    cases = []
    src, dst = W.knn_mesh(4096, 4, 0)
    cases.append((src, dst, 4096, 256, False, False))
    cases.append((src, dst, 4096, 256, False, True))
    r, c = W.rmat(scale=12, m_draws=1 << 15, seed=1)
    cases.append((r, c, 1 << 12, 512, True, False))
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    for src_, dst_, n, C, bip, dflt in cases:
        S = E.Schedule.partition(src_, dst_, n, C, bipartite=bip, default_order=dflt)
        want = S.cost()  # allocating entry point: (loads, vertex cut)
        bp, eu, ev, max_ne = device_inputs(S, src_, dst_, bip)
        for _ in range(2):  # two calls in a row share the scratch flags
            rc = call_noalloc(bp, eu, ev, S.k, S.nd, max_ne, counts)
            assert rc == 0, _lib.lib().ep_noalloc_last_error()
            torch.cuda.synchronize()
            loads, touched = (int(v) for v in counts.cpu())
            assert (loads, loads - touched) == want


def test_noalloc_rejects_oversized_vertex_count():
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    bp = torch.zeros(2, dtype=torch.int64, device="cuda")
    ids = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = call_noalloc(bp, ids, ids, 1, (1 << 24) + 1, 1, counts)
    assert rc == -1
    assert b"EP_NOALLOC_MAX_VERTICES" in _lib.lib().ep_noalloc_last_error()
