"""Pins for the oracle's partition, schedule and cost (CPU only).

What the paper fixes and these tests check:
* Section 1 / Fig. 1: the six-particle example needs 9 loads under the default
  schedule and 7 under the partitioned one (tests/golden/worked_example.txt).
* Section 3.1, Eq. 1: C = sum_v (p_v - 1); Section 3.1 example: optimum 1.
* Section 3.2, Definition 3: clone-and-connect in index order
  (tests/golden/worked_example_h.txt, hand-derived).
* Theorem 1: the auxiliary-edge cut of H is >= the vertex cut of the
  reconstructed edge partition, for every partition.
* Theorem 2: OPT_vp <= (d_max - 1) OPT_ep, and the path order grouped by an
  optimal edge partition gives OPT_vp = OPT_ep (brute force, <= 12 tasks).
* Closed forms for the cost: a star and a path.
"""
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import read_golden


# ----------------------------------------------------------------- helpers

def blocks_of(part):
    k = int(part.max()) + 1
    return [np.flatnonzero(part == b) for b in range(k)]


def cost_sets(src, dst, part):
    """loads and vertex cut by set counting (Definition 2)."""
    loads = 0
    touched = set()
    for blk in blocks_of(part):
        vs = set(src[blk].tolist()) | set(dst[blk].tolist())
        loads += len(vs)
        touched |= vs
    return loads, loads - len(touched)


def aux_cut(xadj, adj, ew, part):
    cut = 0
    for a in range(xadj.size - 1):
        for j in range(xadj[a], xadj[a + 1]):
            b = adj[j]
            if a < b and part[a] != part[b]:
                cut += int(ew[j])
    return cut


def equal_blocks(m, C):
    """Every partition of range(m) into m/C unordered blocks of size C."""
    assert m % C == 0

    def rec(rest):
        if not rest:
            yield []
            return
        first, others = rest[0], rest[1:]
        for comb in itertools.combinations(others, C - 1):
            blk = (first,) + comb
            left = [x for x in others if x not in comb]
            for tail in rec(left):
                yield [blk] + tail

    for blocks in rec(list(range(m))):
        part = np.zeros(m, np.int32)
        for b, blk in enumerate(blocks):
            part[list(blk)] = b
        yield part


# ------------------------------------------------------------- worked example

def golden_example():
    g = read_golden("worked_example.txt")
    e = np.array(g["edge"], np.int32)
    return e[:, 1].copy(), e[:, 2].copy(), {k: v[0][0] for k, v in g.items() if k != "edge"}


def test_worked_example_golden_matches_generator():
    src, dst, _ = golden_example()
    s2, d2 = W.worked_example()
    assert np.array_equal(src, s2) and np.array_equal(dst, d2)


def test_worked_example_loads_9_vs_7():
    src, dst, want = golden_example()
    dflt = O.ep_schedule(src, dst, 6, 3, default_order=True)
    assert dflt["loads"] == want["loads_default"]
    assert dflt["cut"] == want["duplicated_default"]
    ep = O.ep_schedule(src, dst, 6, 3)
    assert ep["loads"] == want["loads_partitioned"]
    assert ep["cut"] == want["duplicated_partitioned"] == want["opt_cut"]
    # e1, e2, e4 (tasks 0, 1, 3) share particle a and land in one block
    assert len({int(ep["part"][t]) for t in (0, 1, 3)}) == 1
    # brute force: 7 is the optimum over all 10 balanced bipartitions
    best = min(cost_sets(src, dst, p)[0] for p in equal_blocks(6, 3))
    assert best == 7


def test_worked_example_h_graph():
    src, dst, _ = golden_example()
    g = read_golden("worked_example_h.txt")
    xadj, adj, ew = O.h_graph(src, dst, 6)
    for row in g.values():
        pass
    want = {}
    for key, rows in g.items():
        want[int(key)] = rows[0]
    for a in range(6):
        assert adj[xadj[a]:xadj[a + 1]].tolist() == want[a]
        assert set(ew[xadj[a]:xadj[a + 1]].tolist()) == {1}


# ------------------------------------------------------------------- H graph

@pytest.mark.parametrize("seed", range(5))
def test_h_graph_structure(seed):
    n, m = 7, 12
    src, dst = W.random_graph(n, m, seed)
    xadj, adj, ew = O.h_graph(src, dst, n)
    deg = np.bincount(np.concatenate([src, dst]), minlength=n)
    # total auxiliary weight = sum_v (d_v - 1) over touched vertices (path per vertex)
    assert ew.sum() // 2 == int(np.sum(np.maximum(deg - 1, 0)))
    # every auxiliary edge joins two tasks that share a data vertex
    for a in range(m):
        for j in range(xadj[a], xadj[a + 1]):
            b = adj[j]
            assert a != b
            assert {src[a], dst[a]} & {src[b], dst[b]}
        row = adj[xadj[a]:xadj[a + 1]]
        assert np.all(np.diff(row) > 0)


def test_h_graph_parallel_aux_edges_merge():
    # two tasks on the same pair (u, v): both u's and v's paths join them
    src = np.array([0, 0], np.int32)
    dst = np.array([1, 1], np.int32)
    xadj, adj, ew = O.h_graph(src, dst, 2)
    assert adj.tolist() == [1, 0] and ew.tolist() == [2, 2]


def test_h_graph_self_loop_single_endpoint():
    src = np.array([0, 0, 1], np.int32)
    dst = np.array([0, 1, 1], np.int32)
    xadj, adj, ew = O.h_graph(src, dst, 2)
    # vertex 0: tasks 0,1 -> (0,1); vertex 1: tasks 1,2 -> (1,2)
    assert xadj.tolist() == [0, 1, 3, 4]
    assert adj.tolist() == [1, 0, 2, 1]


# ------------------------------------------------------------ theorems 1, 2

CASES = [(6, 12, 3), (7, 12, 4), (5, 12, 6), (6, 10, 5), (5, 9, 3), (8, 12, 3), (4, 8, 4)]


@pytest.mark.parametrize("n,m,C", CASES)
@pytest.mark.parametrize("seed", range(3))
def test_theorems_brute_force(n, m, C, seed):
    src, dst = W.random_graph(n, m, 100 * seed + n + m + C)
    xadj, adj, ew = O.h_graph(src, dst, n)
    deg = np.bincount(np.concatenate([src, dst]), minlength=n)
    dmax = int(deg.max())
    opt_ep = None
    opt_vp = None
    best_part = None
    for part in equal_blocks(m, C):
        _, cut = cost_sets(src, dst, part)
        ac = aux_cut(xadj, adj, ew, part)
        assert ac >= cut  # Theorem 1, for every partition
        if opt_ep is None or cut < opt_ep:
            opt_ep, best_part = cut, part.copy()
        opt_vp = ac if opt_vp is None else min(opt_vp, ac)
    assert opt_ep <= opt_vp <= max(dmax - 1, 1) * opt_ep or (opt_ep == 0 and opt_vp == 0)
    # the heuristic: feasible, never below the optimum, Theorem 1 holds
    ep = O.ep_schedule(src, dst, n, C)
    assert np.all(np.bincount(ep["part"]) == C)
    assert ep["cut"] >= opt_ep
    assert aux_cut(xadj, adj, ew, ep["part"]) >= ep["cut"]
    # Theorem 2's construction: number tasks block by block of an optimal
    # edge partition, so every vertex's clone path is grouped by block.
    order = np.argsort(best_part, kind="stable")
    s2, d2 = src[order], dst[order]
    p2 = best_part[order]
    x2, a2, w2 = O.h_graph(s2, d2, n)
    assert aux_cut(x2, a2, w2, p2) == opt_ep
    assert min(aux_cut(x2, a2, w2, p) for p in equal_blocks(m, C)) == opt_ep


# -------------------------------------------------------------- cost closed forms

@pytest.mark.parametrize("d,C", [(10, 3), (12, 4), (7, 7), (9, 2)])
def test_cost_star(d, C):
    # star: hub 0 with d leaves; every block holds the hub once plus its leaves
    src = np.zeros(d, np.int32)
    dst = np.arange(1, d + 1, dtype=np.int32)
    k = -(-d // C)
    for dflt in (True, False):
        s = O.ep_schedule(src, dst, d + 1, C, default_order=dflt)
        assert s["loads"] == d + k
        assert s["cut"] == k - 1


@pytest.mark.parametrize("m,C", [(10, 3), (16, 4), (100, 7)])
def test_cost_path(m, C):
    # path 0-1-...-m in path order: a block of c consecutive tasks covers c+1 vertices
    src = np.arange(m, dtype=np.int32)
    dst = src + 1
    k = -(-m // C)
    s = O.ep_schedule(src, dst, m + 1, C, default_order=True)
    assert s["loads"] == m + k and s["cut"] == k - 1
    # the partitioner must find the same optimum (contiguous runs)
    p = O.ep_schedule(src, dst, m + 1, C)
    assert p["loads"] == m + k


# ---------------------------------------------------------- schedule invariants

def check_schedule(src, dst, n, C, s, bipartite=False):
    m = src.size
    k = -(-m // C)
    part = s["part"]
    assert s["k"] == k
    sizes = np.bincount(part, minlength=k)
    assert np.all(sizes[:-1] == C) and sizes[-1] == m - (k - 1) * C
    # edge_perm: grouped by block, ascending id inside a block
    ep, bp = s["edge_perm"], s["block_ptr"]
    assert np.array_equal(np.sort(ep), np.arange(m))
    for b in range(k):
        seg = ep[bp[b]:bp[b + 1]]
        assert np.all(part[seg] == b) and np.all(np.diff(seg) > 0)
    # vertex lists: distinct vertices in first-touch order
    u = (n + src.astype(np.int64)) if bipartite else src.astype(np.int64)
    v = dst.astype(np.int64)
    vp, vl = s["vert_ptr"], s["vert_list"]
    seen_all = set()
    for b in range(k):
        want = []
        seen = set()
        for e in ep[bp[b]:bp[b + 1]]:
            for x in (u[e], v[e]):
                if x not in seen:
                    seen.add(x)
                    want.append(x)
        assert vl[vp[b]:vp[b + 1]].tolist() == want
        seen_all |= seen
    assert s["loads"] == vp[-1] and s["touched"] == len(seen_all)
    assert s["cut"] == s["loads"] - len(seen_all)
    # cpack: a permutation; vertices first touched by block b are consecutive
    nd = 2 * n if bipartite else n
    rl = s["relabel"]
    assert np.array_equal(np.sort(rl), np.arange(nd))
    nxt = 0
    first = set()
    for b in range(k):
        for x in vl[vp[b]:vp[b + 1]]:
            if x not in first:
                first.add(x)
                assert rl[x] == nxt
                nxt += 1


def test_schedule_invariants_small_mesh():
    src, dst = W.knn_mesh(4096, 4, 0)
    for dflt in (False, True):
        s = O.ep_schedule(src, dst, 4096, 256, default_order=dflt)
        check_schedule(src, dst, 4096, 256, s)


def test_partition_beats_default_small_mesh():
    src, dst = W.knn_mesh(4096, 4, 0)
    ep = O.ep_schedule(src, dst, 4096, 256)
    df = O.ep_schedule(src, dst, 4096, 256, default_order=True)
    assert ep["loads"] < 0.5 * df["loads"]
    xadj, adj, ew = O.h_graph(src, dst, 4096)
    # Theorem 1 on the produced partition (vectorised aux cut)
    a = np.repeat(np.arange(src.size), np.diff(xadj))
    cut_aux = int(ew[(a < adj) & (ep["part"][a] != ep["part"][adj])].sum())
    assert cut_aux >= ep["cut"]


def test_schedule_bipartite_invariants():
    r, c = W.rmat(scale=9, m_draws=4000, seed=3)
    n = 1 << 9
    for dflt in (False, True):
        s = O.ep_schedule(r, c, n, 64, bipartite=True, default_order=dflt)
        check_schedule(r, c, n, 64, s, bipartite=True)


def test_ragged_last_block_and_single_block():
    src, dst = W.random_graph(30, 101, 9)
    s = O.ep_schedule(src, dst, 30, 16)
    check_schedule(src, dst, 30, 16, s)
    s1 = O.ep_schedule(src, dst, 30, 1000)
    assert s1["k"] == 1 and s1["loads"] == len(set(src) | set(dst))


def test_invalid_inputs_rejected():
    src = np.array([0, 5], np.int32)
    dst = np.array([1, 2], np.int32)
    with pytest.raises(ValueError):
        O.partition(src, dst, 3, 2)  # vertex id >= n
    with pytest.raises(ValueError):
        O.partition(src[:1], dst[:1], 3, 0)  # C <= 0
    with pytest.raises(ValueError):
        O.partition(src[:0], dst[:0], 3, 2)  # m = 0


# ------------------------------------------------------------------- bisection

def csr(n, pairs):
    nb = [[] for _ in range(n)]
    for a, b in pairs:
        nb[a].append(b)
        nb[b].append(a)
    xadj = np.zeros(n + 1, np.int64)
    adj, ew = [], []
    for a in range(n):
        row = sorted(nb[a])
        adj += row
        ew += [1] * len(row)
        xadj[a + 1] = len(adj)
    return xadj, np.array(adj, np.int32), np.array(ew, np.int32)


def test_bisect_two_cliques():
    s = 40
    pairs = [(a, b) for a in range(s) for b in range(a + 1, s)]
    pairs += [(s + a, s + b) for a in range(s) for b in range(a + 1, s)]
    pairs += [(0, s)]  # one bridge
    xadj, adj, ew = csr(2 * s, pairs)
    side = O.bisect(xadj, adj, ew, s)
    assert side.sum() == s
    assert len({int(x) for x in side[:s]}) == 1 and len({int(x) for x in side[s:]}) == 1


def test_bisect_path_and_grid():
    n = 500
    xadj, adj, ew = csr(n, [(i, i + 1) for i in range(n - 1)])
    side = O.bisect(xadj, adj, ew, 200)
    assert int((side == 0).sum()) == 200
    assert int(np.sum(side[1:] != side[:-1])) == 1  # one contiguous split
    g = 30
    pairs = [(r * g + c, r * g + c + 1) for r in range(g) for c in range(g - 1)]
    pairs += [(r * g + c, (r + 1) * g + c) for r in range(g - 1) for c in range(g)]
    xadj, adj, ew = csr(g * g, pairs)
    side = O.bisect(xadj, adj, ew, g * g // 2)
    a = np.repeat(np.arange(g * g), np.diff(xadj))
    cut = int(np.sum(side[a] != side[adj])) // 2
    assert int((side == 0).sum()) == g * g // 2
    assert cut <= 2 * g  # a straight cut has g edges; allow a ragged one
