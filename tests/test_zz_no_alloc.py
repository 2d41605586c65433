"""ep_cost_noalloc: the load count for callers that cannot allocate (GPU only).

Some callers cannot let a library call cudaMalloc: applications that hand all
device memory to their own pool or framework allocator and forbid allocations
behind its back, and latency-bound loops that cannot take the device
synchronisation an allocation may cause.  ep_cost_noalloc() serves them: the
caller passes every input and output as device memory and the only scratch is
a fixed device array in the library.  These tests check it against the oracle
and against ep_cost(), which allocates its own workspace, on two calls in a
row (the shared scratch keeps the previous call's flags, so the second call
shows that they are cleared), and check that misuse the host cannot see (a
block longer than max_ne, an id outside [0, nd)) is reported in the counts.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_02043_gb300 as E  # noqa: E402
from paper_1605_02043_gb300 import _lib  # noqa: E402

INVALID = (1 << 64) - 1  # EP_NOALLOC_INVALID
BAD_BLOCK, BAD_ID = 1, 2  # EP_NOALLOC_BAD_BLOCK, EP_NOALLOC_BAD_ID


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


def read_counts(counts):
    torch.cuda.synchronize()
    return tuple(int(v) & ((1 << 64) - 1) for v in counts.cpu())


def cases():
    src, dst = W.knn_mesh(4096, 4, 0)
    r, c = W.rmat(scale=12, m_draws=1 << 15, seed=1)
    return [(src, dst, 4096, 256, False, False), (src, dst, 4096, 256, False, True),
            (r, c, 1 << 12, 512, True, False)]


def test_noalloc_cost_matches_oracle_and_allocating_entry_point_twice():
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    for src_, dst_, n, C, bip, dflt in cases():
        S = E.Schedule.partition(src_, dst_, n, C, bipartite=bip, default_order=dflt)
        ref = O.ep_schedule(src_, dst_, n, C, bipartite=bip, default_order=dflt)
        assert S.cost() == (ref["loads"], ref["cut"])  # allocating entry point
        bp, eu, ev, max_ne = device_inputs(S, src_, dst_, bip)
        for _ in range(2):  # two calls in a row share the scratch flags
            rc = call_noalloc(bp, eu, ev, S.k, S.nd, max_ne, counts)
            assert rc == 0, _lib.lib().ep_noalloc_last_error()
            loads, touched = read_counts(counts)
            assert (loads, loads - touched) == (ref["loads"], ref["cut"])


def test_noalloc_reports_blocks_longer_than_max_ne():
    src, dst, n, C, bip, dflt = cases()[0]
    S = E.Schedule.partition(src, dst, n, C)
    ref = O.ep_schedule(src, dst, n, C)
    bp, eu, ev, max_ne = device_inputs(S, src, dst, bip)
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert call_noalloc(bp, eu, ev, S.k, S.nd, max_ne // 2, counts) == 0
    assert read_counts(counts) == (INVALID, BAD_BLOCK)
    # the next well-formed call is clean again (the status word is cleared)
    assert call_noalloc(bp, eu, ev, S.k, S.nd, max_ne, counts) == 0
    loads, touched = read_counts(counts)
    assert (loads, loads - touched) == (ref["loads"], ref["cut"])


@pytest.mark.parametrize("bad", [4096, 1 << 24, -1])
def test_noalloc_reports_ids_outside_range(bad):
    src, dst, n, C, bip, dflt = cases()[0]
    S = E.Schedule.partition(src, dst, n, C)
    bp, eu, ev, max_ne = device_inputs(S, src, dst, bip)
    ev = ev.clone()
    ev[17] = bad
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert call_noalloc(bp, eu, ev, S.k, S.nd, max_ne, counts) == 0
    assert read_counts(counts) == (INVALID, BAD_ID)
    # both misuses at once
    assert call_noalloc(bp, eu, ev, S.k, S.nd, max_ne // 2, counts) == 0
    loads, reasons = read_counts(counts)
    assert loads == INVALID and reasons & BAD_BLOCK


def test_noalloc_rejects_oversized_vertex_count():
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    bp = torch.zeros(2, dtype=torch.int64, device="cuda")
    ids = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = call_noalloc(bp, ids, ids, 1, (1 << 24) + 1, 1, counts)
    assert rc == -1
    assert b"EP_NOALLOC_MAX_VERTICES" in _lib.lib().ep_noalloc_last_error()
    # a rejected call leaves no CUDA error behind: the next call succeeds
    ids1 = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    bp1 = torch.tensor([0, 2], dtype=torch.int64, device="cuda")
    assert call_noalloc(bp1, ids1, ids1.flip(0).contiguous(), 1, 2, 2, counts) == 0
    assert read_counts(counts) == (2, 2)
