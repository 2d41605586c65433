"""Host-side tests of libepcache (CPU only, no kernel launches).

* the library loads and exports every function include/epcache.h declares;
* its partitioner, vertex lists, cpack and host cost are bit-exact with the
  oracle (the same partition rules implemented twice, sharing no code);
* results do not depend on the number of host threads;
* bad arguments give EP_EINVAL and kernel calls without a GPU give EP_ENODEV.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1605_02043_gb300 as E
from paper_1605_02043_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel")


def declared_functions():
    text = open(os.path.join(ROOT, "include", "epcache.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ep_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported():
    lib = _lib.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.SIGNATURES)


def same_as_oracle(src, dst, n, C, bipartite=False, default_order=False, threads=0):
    S = E.Schedule.partition(src, dst, n, C, bipartite=bipartite, default_order=default_order,
                             threads=threads)
    ref = O.ep_schedule(src, dst, n, C, bipartite=bipartite, default_order=default_order)
    a = S.arrays()
    for key in KEYS:
        assert np.array_equal(a[key], ref[key]), key
    assert (a["loads"], a["cut"]) == (ref["loads"], ref["cut"])
    return S, ref


def test_worked_example():
    src, dst = W.worked_example()
    S, ref = same_as_oracle(src, dst, 6, 3)
    assert S.cost_host() == (7, 1)
    S, ref = same_as_oracle(src, dst, 6, 3, default_order=True)
    assert S.cost_host() == (9, 3)


@pytest.mark.parametrize("C", [1, 2, 17, 64, 256, 1024, 20000])
def test_small_mesh_parity(C):
    src, dst = W.knn_mesh(4096, 4, 0)
    same_as_oracle(src, dst, 4096, min(C, E_MAX_C()))


def E_MAX_C():
    return 16384


@pytest.mark.parametrize("seed", range(6))
def test_random_multigraph_parity(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 400))
    m = int(rng.integers(1, 3000))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    C = int(rng.integers(1, 300))
    same_as_oracle(src, dst, n, C)
    same_as_oracle(src, dst, n, C, default_order=True)


@pytest.mark.parametrize("C", [32, 512])
def test_bipartite_parity(C):
    r, c = W.rmat(scale=11, m_draws=30000, seed=5)
    same_as_oracle(r, c, 1 << 11, C, bipartite=True)
    same_as_oracle(r, c, 1 << 11, C, bipartite=True, default_order=True)


def test_mid_mesh_parity_and_thread_independence():
    src, dst = W.knn_mesh(60000, 4, 3)
    S1, ref = same_as_oracle(src, dst, 60000, 256, threads=1)
    S8 = E.Schedule.partition(src, dst, 60000, 256, threads=8)
    for key in KEYS:
        assert np.array_equal(S1.arrays()[key], S8.arrays()[key])


def test_batch_host_arrays():
    meshes = [W.knn_mesh(nn, 4, 10 + i) for i, nn in enumerate((500, 900))]
    parts = [E.Schedule.partition(s, d, nn, 64) for (s, d), nn in zip(meshes, (500, 900))]
    B = E.Schedule.batch(parts)
    assert (B.m, B.n, B.k) == (sum(p.m for p in parts), 1400, sum(p.k for p in parts))
    # the merged schedule equals the oracle schedule of the union graph with the
    # per-part block ids offset
    src = np.concatenate([meshes[0][0], meshes[1][0] + 500]).astype(np.int32)
    dst = np.concatenate([meshes[0][1], meshes[1][1] + 500]).astype(np.int32)
    part = np.concatenate([parts[0].part(), parts[1].part() + parts[0].k])
    ref = O.schedule(src, dst, 1400, part)
    a = B.arrays()
    for key in KEYS:
        assert np.array_equal(a[key], ref[key]), key
    assert B.cost_host() == (ref["loads"], ref["cut"])


def test_invalid_arguments():
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 3], np.int32)
    for args in ((src, dst, 3, 2), (src, dst, 4, 0), (src, dst, 4, 100000), (src[:0], dst[:0], 4, 2)):
        with pytest.raises(E.EpError) as ei:
            E.Schedule.partition(*args)
        assert ei.value.code == -1
    h = ctypes.c_void_p()
    assert _lib.lib().ep_partition(src.ctypes.data, dst.ctypes.data, 3, 4, 2, 8, 0,
                                   ctypes.byref(h)) == -1  # unknown flag
    S = E.Schedule.partition(src, dst, 4, 2)
    for bad in (-2, 256):
        with pytest.raises(E.EpError) as ei:
            S.debug_stall(bad)
        assert ei.value.code == -1
    S.debug_stall(0)
    S.debug_stall(-1)
    for bad in (-1, 2):
        with pytest.raises(E.EpError):
            S.set_cache(bad)
    S.set_cache(E.CACHE_L1)
    S.set_cache(E.CACHE_SMEM)
    for setter in (S.set_threads, S.set_adjoint_threads):
        for bad in (0, 16, 48 + 1, 1056):
            with pytest.raises(E.EpError) as ei:
                setter(bad)
            assert ei.value.code == -1
        setter(32)
        setter(1024)
    # blocks of more than 4096 vertex positions are too large for the L1 variant
    s2, d2 = W.knn_mesh(20000, 4, 0)
    big = E.Schedule.partition(s2, d2, 20000, 4000, default_order=True)
    with pytest.raises(E.EpError) as ei:
        big.set_cache(E.CACHE_L1)
    assert ei.value.code == -1 and "4096" in str(ei.value)


def test_kernel_calls_need_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    src, dst = W.worked_example()
    S = E.Schedule.partition(src, dst, 6, 3)
    loads, cut = ctypes.c_int64(), ctypes.c_int64()
    rc = _lib.lib().ep_cost(S._h, ctypes.byref(loads), ctypes.byref(cut), None)
    assert rc == -5  # EP_ENODEV: no CPU fallback
    rc = _lib.lib().ep_run(S._h, 0, None, None, None, 5, 1, 1e-3, None)
    assert rc == -1  # null pointers are rejected before anything else
