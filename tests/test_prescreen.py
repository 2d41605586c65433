"""Pre-screen before partitioning (Section 4, the optimisation workflow): the
oracle's outcomes and presets pinned to closed forms and brute force, and the
library's pre-screen bit-exact with the oracle.  No GPU needed."""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_1605_02043_gb300 as E
from test_oracle_partition import cost_sets, equal_blocks

KEYS = ("block_ptr", "edge_perm", "vert_ptr", "vert_list", "relabel")


def path_graph(m, seed, bipartite=False):
    """A simple path of m tasks over shuffled vertex ids, tasks shuffled and
    randomly oriented."""
    rng = np.random.default_rng(seed)
    if bipartite:  # alternate rows and columns: y_r0 - x_c0 - y_r1 - x_c1 ...
        rows = rng.permutation(m)[: (m + 2) // 2]
        cols = rng.permutation(m)[: (m + 1) // 2]
        seq = []
        for i in range(m + 1):
            seq.append(("y", rows[i // 2]) if i % 2 == 0 else ("x", cols[i // 2]))
        src, dst = [], []
        for a, b in zip(seq, seq[1:]):
            r = a[1] if a[0] == "y" else b[1]
            c = a[1] if a[0] == "x" else b[1]
            src.append(r)
            dst.append(c)
        src, dst = np.array(src, np.int32), np.array(dst, np.int32)
        order = rng.permutation(m)
        return src[order], dst[order], m
    n = m + 1 + 5  # a few isolated vertices
    vid = rng.permutation(n)[: m + 1]
    src = vid[:-1].astype(np.int32)
    dst = vid[1:].astype(np.int32)
    flip = rng.random(m) < 0.5
    src, dst = np.where(flip, dst, src), np.where(flip, src, dst)
    order = rng.permutation(m)
    return src[order].astype(np.int32), dst[order].astype(np.int32), n


def star_graph(d, seed):
    rng = np.random.default_rng(seed)
    n = d + 3
    ids = rng.permutation(n)
    c = ids[0]
    leaves = ids[1 : d + 1]
    flip = rng.random(d) < 0.5
    src = np.where(flip, leaves, c).astype(np.int32)
    dst = np.where(flip, c, leaves).astype(np.int32)
    return src, dst, n


@pytest.mark.parametrize("m,C", [(1, 1), (2, 2), (9, 3), (100, 7), (1000, 64), (4097, 256)])
@pytest.mark.parametrize("seed", [0, 1])
def test_path_preset_reaches_m_plus_k(m, C, seed):
    src, dst, n = path_graph(m, seed)
    p = O.prescreen(src, dst, n)
    assert p["origin"] == "path" and p["touched"] == m + 1 and p["degree_sum"] == 2 * m
    # the walk is a path: consecutive tasks share a vertex, each task once
    o = p["order"]
    assert np.array_equal(np.sort(o), np.arange(m))
    for a, b in zip(o, o[1:]):
        assert {src[a], dst[a]} & {src[b], dst[b]}
    # it starts at the smaller-id end
    deg = np.bincount(np.concatenate([src, dst]), minlength=n)
    assert np.flatnonzero(deg == 1).min() in (src[o[0]], dst[o[0]])
    s = O.ep_schedule(src, dst, n, C, prescreen=True)
    k = -(-m // C)
    assert s["loads"] == m + k  # C path edges touch at least C + 1 vertices
    assert cost_sets(src, dst, s["part"])[0] == m + k


@pytest.mark.parametrize("m,C", [(6, 2), (6, 3), (8, 4)])
def test_path_preset_is_brute_force_optimal(m, C):
    src, dst, n = path_graph(m, 3)
    best = min(cost_sets(src, dst, part)[0] for part in equal_blocks(m, C))
    assert O.ep_schedule(src, dst, n, C, prescreen=True)["loads"] == best


def test_bipartite_path():
    src, dst, n = path_graph(40, 5, bipartite=True)
    p = O.prescreen(src, dst, n, bipartite=True)
    assert p["origin"] == "path"
    s = O.ep_schedule(src, dst, n, 8, bipartite=True, prescreen=True)
    assert s["loads"] == 40 + 5


@pytest.mark.parametrize("d,C", [(2, 1), (10, 3), (300, 16)])
def test_star_keeps_default_order(d, C):
    src, dst, n = star_graph(d, d)
    p = O.prescreen(src, dst, n)
    assert p["origin"] == ("path" if d == 2 else "star") and p["max_degree"] == d
    s = O.ep_schedule(src, dst, n, C, prescreen=True)
    k = -(-d // C)
    assert s["loads"] == d + k  # every schedule of a star loads d + k
    if d > 2:
        assert np.array_equal(s["part"], np.arange(d) // C)


def test_low_reuse_keeps_default_order():
    # points each used once, a few centres used by many (streamcluster-like):
    # mean degree of touched vertices is below 2
    rng = np.random.default_rng(1)
    pts = 500
    src = np.arange(pts, dtype=np.int32)
    dst = (pts + rng.integers(0, 4, pts)).astype(np.int32)
    dst[:4] = pts + np.arange(4)
    p = O.prescreen(src, dst, pts + 4)
    assert p["origin"] == "low_reuse" and p["degree_sum"] <= 2 * p["touched"]
    s = O.ep_schedule(src, dst, pts + 4, 64, prescreen=True)
    assert np.array_equal(s["part"], np.arange(pts) // 64)


def test_mesh_is_partitioned_as_without_prescreen():
    src, dst = W.knn_mesh(2000, 4, 0)
    p = O.prescreen(src, dst, 2000)
    assert p["origin"] == "partition" and p["degree_sum"] > 2 * p["touched"]
    a = O.ep_schedule(src, dst, 2000, 128, prescreen=True)
    b = O.ep_schedule(src, dst, 2000, 128)
    assert np.array_equal(a["part"], b["part"])


def test_not_a_path():
    # a cycle, a path plus a duplicate task, two disjoint paths, a self loop
    cyc_s = np.arange(6, dtype=np.int32)
    cyc_d = ((np.arange(6) + 1) % 6).astype(np.int32)
    dup_s = np.array([0, 1, 2, 1], np.int32)
    dup_d = np.array([1, 2, 3, 2], np.int32)
    two_s = np.array([0, 1, 4, 5], np.int32)
    two_d = np.array([1, 2, 5, 6], np.int32)
    loop_s = np.array([0, 1, 2, 2], np.int32)
    loop_d = np.array([1, 2, 3, 2], np.int32)
    for s, d in ((cyc_s, cyc_d), (dup_s, dup_d), (two_s, two_d), (loop_s, loop_d)):
        assert O.prescreen(s, d, 8)["origin"] != "path"
    assert O.prescreen(cyc_s, cyc_d, 8)["origin"] == "low_reuse"  # mean degree 2


CASES = [
    ("path", lambda: path_graph(1000, 2)),
    ("path_small", lambda: path_graph(7, 4)),
    ("star", lambda: star_graph(200, 0)),
    ("mesh", lambda: (*W.knn_mesh(1500, 4, 2), 1500)),
    ("cycle", lambda: (np.arange(50, dtype=np.int32), ((np.arange(50) + 1) % 50).astype(np.int32), 50)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("C", [16, 100])
def test_library_matches_oracle(name, make, C):
    src, dst, n = make()
    p = O.prescreen(src, dst, n)
    q = E.prescreen(src, dst, n)
    for key in ("touched", "degree_sum", "max_degree", "origin"):
        assert p[key] == q[key], key
    S = E.Schedule.partition(src, dst, n, C, prescreen=True)
    ref = O.ep_schedule(src, dst, n, C, prescreen=True)
    a = S.arrays()
    for key in KEYS:
        assert np.array_equal(a[key], ref[key]), key
    assert S.origin == p["origin"]
    assert E.Schedule.partition(src, dst, n, C).origin == "partition"
    assert E.Schedule.partition(src, dst, n, C, default_order=True, prescreen=True).origin == "default"


def test_library_bipartite_matches_oracle():
    src, dst, n = path_graph(60, 8, bipartite=True)
    assert E.prescreen(src, dst, n, bipartite=True)["origin"] == "path"
    S = E.Schedule.partition(src, dst, n, 8, bipartite=True, prescreen=True)
    ref = O.ep_schedule(src, dst, n, 8, bipartite=True, prescreen=True)
    for key in KEYS:
        assert np.array_equal(S.arrays()[key], ref[key]), key


def test_job_takes_the_prescreen_flag():
    src, dst, n = path_graph(500, 9)
    j = E.PartitionJob(src, dst, n, 32, prescreen=True)
    assert j.wait(30)
    S = j.take()
    assert S.origin == "path" and S.cost_host()[0] == 500 + 16
    j.close()
