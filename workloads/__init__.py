"""Seeded synthetic workloads shared by the oracle, the tests and the bench.

This module only draws inputs: point clouds, k-nearest-neighbour meshes, R-MAT
edge lists, node states and edge weights.  It contains none of the method's
arithmetic (no partitioning, no cost, no edge kernel), so both the CPU oracle
and the CUDA path can take their inputs from it without sharing any code.

Recipes (all NumPy PCG64 streams, float64 draws cast to float32 at the end):

* ``knn_mesh(n, k, seed)``: ``n`` points uniform in the unit cube from
  ``default_rng(seed)``; for every point its ``k`` nearest other points
  (Euclidean, float64, ties to the smaller index); the pairs are symmetrised to
  unique ``(min, max)`` edges, sorted, then shuffled by a permutation drawn from
  ``default_rng([seed, 7])``.  The shuffled order is the "default" task order.
  These meshes stand in for the unstructured CFD meshes the paper evaluates on
  (Section 5: nodes with two to four neighbours, like mc2depi).
* ``rmat(scale, m_draws, abcd, seed)``: R-MAT recursive quadrant draws,
  one ``random()`` vector per level from ``default_rng(seed)``; self loops and
  duplicates dropped; edges sorted by (row, col) (CSR order).  Stands in for the
  power-law matrices of Section 5 (in-2004, scircuit).
* ``flux_state(n, D, seed)``: x ~ N(0, 1) as a ``[D][n]`` float32 array.
* ``flux_weights(m, seed)``: w ~ U(0.5, 1.5) float32.
* ``spmv_inputs(n, m, seed)``: x ~ U(-1, 1), w ~ U(0, 1) float32.
* ``batch_meshes(count, lo, hi, seed)``: node counts ``exp(U(ln lo, ln hi))``
  from ``default_rng(seed)``, mesh ``i`` drawn by ``knn_mesh(n_i, 4, 1000+i)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "knn_mesh",
    "rmat",
    "flux_state",
    "flux_weights",
    "spmv_inputs",
    "batch_sizes",
    "batch_meshes",
    "random_graph",
    "worked_example",
    "MESH_SMALL",
    "MESH_LARGE",
]

# named workloads: (points, neighbours, seed)
MESH_SMALL = (4096, 4, 0)
MESH_LARGE = (1 << 20, 4, 0)


def knn_mesh(n: int, k: int = 4, seed: int = 0):
    """Symmetrised k-NN mesh on ``n`` uniform points; returns (src, dst) int32.

    The edge order is a seeded random permutation (the default task order)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    kk = min(k + 1, n)
    dist, idx = cKDTree(pts).query(pts, k=kk, workers=-1)
    idx = np.asarray(idx, dtype=np.int64).reshape(n, kk)
    dist = np.asarray(dist).reshape(n, kk)
    # stable order by (distance, index) so equal distances go to the smaller index
    order = np.lexsort((idx, dist), axis=1)
    idx = np.take_along_axis(idx, order, axis=1)
    rows = np.repeat(np.arange(n, dtype=np.int64), kk)
    cols = idx.reshape(-1)
    keep = cols != rows
    rows, cols = rows[keep], cols[keep]
    # first k non-self neighbours of every point
    rank = np.zeros_like(rows)
    # position among kept entries of the same row
    starts = np.searchsorted(rows, np.arange(n))
    rank = np.arange(rows.size) - starts[rows]
    sel = rank < k
    rows, cols = rows[sel], cols[sel]
    a = np.minimum(rows, cols)
    b = np.maximum(rows, cols)
    key = np.unique(a * n + b)
    src = (key // n).astype(np.int32)
    dst = (key % n).astype(np.int32)
    perm = np.random.default_rng([seed, 7]).permutation(src.size)
    return src[perm].copy(), dst[perm].copy()


def rmat(scale: int = 20, m_draws: int = 1 << 24, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0):
    """R-MAT edge list (rows, cols) int32 in CSR order; self loops and duplicates removed."""
    a, b, c, _ = abcd
    rng = np.random.default_rng(seed)
    row = np.zeros(m_draws, dtype=np.int64)
    col = np.zeros(m_draws, dtype=np.int64)
    for level in range(scale):
        r = rng.random(m_draws)
        bit = np.int64(1) << np.int64(scale - 1 - level)
        # quadrants: [0,a) -> (0,0); [a,a+b) -> (0,1); [a+b,a+b+c) -> (1,0); rest -> (1,1)
        rbit = r >= a + b
        cbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        row += rbit * bit
        col += cbit * bit
    keep = row != col
    nv = np.int64(1) << np.int64(scale)
    key = np.unique(row[keep] * nv + col[keep])
    return (key // nv).astype(np.int32), (key % nv).astype(np.int32)


def flux_state(n: int, D: int = 5, seed: int = 0) -> np.ndarray:
    """Node states x ~ N(0,1), shape [D][n], float32."""
    return np.random.default_rng([seed, 1]).standard_normal((D, n)).astype(np.float32)


def flux_weights(m: int, seed: int = 0) -> np.ndarray:
    """Edge weights w ~ U(0.5, 1.5), float32."""
    return np.random.default_rng([seed, 2]).uniform(0.5, 1.5, m).astype(np.float32)


def spmv_inputs(n: int, m: int, seed: int = 0):
    """SpMV-style inputs: x ~ U(-1,1) [n] and w ~ U(0,1) [m], float32."""
    x = np.random.default_rng([seed, 3]).uniform(-1.0, 1.0, n).astype(np.float32)
    w = np.random.default_rng([seed, 4]).uniform(0.0, 1.0, m).astype(np.float32)
    return x, w


def loss_weights(n: int, D: int = 5, seed: int = 1) -> np.ndarray:
    """Fixed cotangent g ~ N(0,1), shape [D][n], for the linear loss <g, x_T>."""
    return np.random.default_rng(seed).standard_normal((D, n))


def batch_sizes(count: int = 512, lo: int = 1024, hi: int = 65536, seed: int = 0) -> np.ndarray:
    """Node counts log-uniform in [lo, hi] (rounded to int)."""
    u = np.random.default_rng(seed).uniform(np.log(lo), np.log(hi), count)
    return np.rint(np.exp(u)).astype(np.int64)


def batch_meshes(count: int = 512, lo: int = 1024, hi: int = 65536, seed: int = 0):
    """List of (n_i, src_i, dst_i) k=4 meshes with log-uniform node counts."""
    out = []
    for i, n_i in enumerate(batch_sizes(count, lo, hi, seed)):
        s, d = knn_mesh(int(n_i), 4, 1000 + i)
        out.append((int(n_i), s, d))
    return out


def random_graph(n: int, m: int, seed: int):
    """Small random multigraph without self loops (for brute-force tests)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n - 1, m)
    dst = np.where(dst >= src, dst + 1, dst)
    return src.astype(np.int32), dst.astype(np.int32)


def worked_example():
    """Six particles a..f and six interactions e1..e6 (Fig. 1 / Fig. 3 graph).

    The paper's figure is not in the text; this graph satisfies every stated
    constraint: schedule {e1,e2,e3}|{e4,e5,e6} needs 9 loads with three particles
    fetched twice, schedule {e1,e2,e4}|{e3,e5,e6} needs 7 loads with one particle
    fetched twice, and e1, e2, e4 share one particle (a)."""
    a, b, c, d, e, f = range(6)
    src = np.array([a, a, b, a, b, e], dtype=np.int32)
    dst = np.array([b, c, e, d, f, f], dtype=np.int32)
    return src, dst
