"""CPU oracle for the edge-partitioned gather-interact-scatter path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports it and shares no code with it.

* Partition, schedule, cpack and cost: ``ep_oracle.c`` (plain serial C, built
  with gcc on first use).  See that file's header for the rules it follows
  (Section 3.2 transform, Definition 4 reconstruction, Section 4.1 cpack,
  Eq. 1 cost).
* Edge kernels, time stepping and the adjoint: NumPy float64 below.
* ``cpu_fair.c``: the same explicit steps in FP64 on all host cores (OpenMP),
  only for the bench's CPU context line; checked against the NumPy oracle.

Parity status: the partition heuristic's tie-break output is a rule of this
project (the paper delegates to METIS); beyond the worked example and the
brute-force/theorem checks its exact output is "parity unpinned" against the
paper and is pinned only as a specification shared by two implementations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ep_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libeporacle.so")
_lock = threading.Lock()
_lib = None

BIPARTITE = 1
DEFAULT_ORDER = 2


def build() -> str:
    """Compile the C oracle (idempotent); returns the shared-object path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_FAIR_SRC = os.path.join(_HERE, "cpu_fair.c")
_FAIR_SO = os.path.join(_BUILD, "libcpufair.so")


def build_fair() -> str | None:
    """Compile the OpenMP CPU baseline (cpu_fair.c); None if the compiler
    cannot (it is optional: only the bench's CPU context line uses it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(_FAIR_SO) or os.path.getmtime(_FAIR_SO) < os.path.getmtime(_FAIR_SRC):
        tmp = _FAIR_SO + f".{os.getpid()}.tmp"
        try:
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c99", "-shared", "-fPIC", "-o",
                                   tmp, _FAIR_SRC], stderr=subprocess.DEVNULL)
        except (OSError, subprocess.CalledProcessError):
            return None
        os.replace(tmp, _FAIR_SO)
    return _FAIR_SO


class FairCpu:
    """Multi-threaded FP64 explicit flux steps on all host cores (cpu_fair.c)."""

    def __init__(self, src, dst, n: int, D: int):
        so = build_fair()
        if so is None:
            raise RuntimeError("cpu_fair.c could not be built (no OpenMP)")
        lib = ctypes.CDLL(so)
        P = ctypes.c_void_p
        lib.fair_build.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
        lib.fair_build.restype = P
        lib.fair_free.argtypes = [P]
        lib.fair_steps.argtypes = [P, P, P, P, P, P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32]
        lib.fair_steps.restype = ctypes.c_int
        self._lib = lib
        self.src, self.dst = _edges(src, dst)
        self.n, self.D = n, D
        self._h = lib.fair_build(_p(self.src), _p(self.dst), self.src.size, n, D)
        if not self._h:
            raise ValueError("fair_build failed")

    def steps(self, x, w, steps: int, tau: float, threads: int = 0):
        """x float64 [D][n] updated in place; returns (flux of the last step, threads used)."""
        assert x.dtype == np.float64 and x.flags.c_contiguous and x.shape == (self.D, self.n)
        w = np.ascontiguousarray(w, np.float64)
        out = np.zeros_like(x)
        used = self._lib.fair_steps(self._h, _p(self.src), _p(self.dst), _p(w), _p(x), _p(out),
                                    steps, tau, threads)
        return out, used

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.fair_free(self._h)
            self._h = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
            lib.orc_h_nnz.argtypes = [P, P, i64, i64, i32]
            lib.orc_h_nnz.restype = i64
            lib.orc_h_graph.argtypes = [P, P, i64, i64, i32, P, P, P]
            lib.orc_h_graph.restype = i32
            lib.orc_bisect.argtypes = [P, P, P, i32, i64, P]
            lib.orc_bisect.restype = i32
            lib.orc_prescreen.argtypes = [P, P, i64, i64, u32, P, P]
            lib.orc_prescreen.restype = i32
            lib.orc_partition.argtypes = [P, P, i64, i64, i32, u32, P]
            lib.orc_partition.restype = i32
            lib.orc_schedule.argtypes = [P, P, i64, i64, u32, P, i32, P, P, P, P, P, P]
            lib.orc_schedule.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _edges(src, dst):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape or src.ndim != 1:
        raise ValueError("src and dst must be equal-length 1-D arrays")
    return src, dst


def h_graph(src, dst, n: int, bipartite: bool = False):
    """Contracted clone-and-connect graph H as CSR (xadj, adj, ew)."""
    src, dst = _edges(src, dst)
    lib = _load()
    m = src.size
    nnz = lib.orc_h_nnz(_p(src), _p(dst), m, n, int(bipartite))
    if nnz < 0:
        raise ValueError("invalid edge list")
    xadj = np.zeros(m + 1, np.int64)
    adj = np.zeros(max(nnz, 1), np.int32)
    ew = np.zeros(max(nnz, 1), np.int32)
    if lib.orc_h_graph(_p(src), _p(dst), m, n, int(bipartite), _p(xadj), _p(adj), _p(ew)):
        raise ValueError("invalid edge list")
    return xadj, adj[:nnz], ew[:nnz]


def bisect(xadj, adj, ew, s_left: int) -> np.ndarray:
    """One multilevel bisection of a unit-weight graph; side[u] in {0, 1}."""
    xadj = np.ascontiguousarray(xadj, np.int64)
    adj = np.ascontiguousarray(adj, np.int32)
    ew = np.ascontiguousarray(ew, np.int32)
    n = xadj.size - 1
    side = np.zeros(n, np.uint8)
    if _load().orc_bisect(_p(xadj), _p(adj), _p(ew), n, s_left, _p(side)):
        raise ValueError("invalid bisection request")
    return side


PRESCREEN_OUTCOMES = {0: "partition", 2: "path", 3: "star", 4: "low_reuse"}


def prescreen(src, dst, n: int, bipartite: bool = False) -> dict:
    """Pre-screen of Section 4's workflow (see orc_prescreen): degree summary,
    outcome, and for a path the walk order of its tasks."""
    src, dst = _edges(src, dst)
    out = np.zeros(4, np.int64)
    order = np.full(src.size, -1, np.int32)
    if _load().orc_prescreen(_p(src), _p(dst), src.size, n, BIPARTITE if bipartite else 0,
                             _p(out), _p(order)):
        raise ValueError("orc_prescreen failed")
    outcome = PRESCREEN_OUTCOMES[int(out[3])]
    return dict(touched=int(out[0]), degree_sum=int(out[1]), max_degree=int(out[2]),
                origin=outcome, order=order if outcome == "path" else None)


def partition(src, dst, n: int, C: int, bipartite: bool = False, default_order: bool = False,
              prescreen: bool = False):
    """Block id of every task (edge); k = ceil(m / C) blocks."""
    src, dst = _edges(src, dst)
    part = np.zeros(src.size, np.int32)
    flags = ((BIPARTITE if bipartite else 0) | (DEFAULT_ORDER if default_order else 0)
             | (4 if prescreen else 0))
    rc = _load().orc_partition(_p(src), _p(dst), src.size, n, C, flags, _p(part))
    if rc:
        raise ValueError(f"orc_partition failed ({rc})")
    return part


def schedule(src, dst, n: int, part, bipartite: bool = False) -> dict:
    """Schedule arrays and cost from a partition (see ep_oracle.c)."""
    src, dst = _edges(src, dst)
    part = np.ascontiguousarray(part, np.int32)
    m = src.size
    k = int(part.max()) + 1
    nd = 2 * n if bipartite else n
    block_ptr = np.zeros(k + 1, np.int64)
    edge_perm = np.zeros(m, np.int32)
    vert_ptr = np.zeros(k + 1, np.int64)
    vert_list = np.zeros(2 * m, np.int32)
    relabel = np.zeros(nd, np.int32)
    stats = np.zeros(3, np.int64)
    rc = _load().orc_schedule(_p(src), _p(dst), m, n, BIPARTITE if bipartite else 0, _p(part), k,
                              _p(block_ptr), _p(edge_perm), _p(vert_ptr), _p(vert_list),
                              _p(relabel), _p(stats))
    if rc:
        raise ValueError("orc_schedule failed")
    return dict(k=k, block_ptr=block_ptr, edge_perm=edge_perm, vert_ptr=vert_ptr,
                vert_list=vert_list[: int(stats[0])].copy(), relabel=relabel,
                loads=int(stats[0]), cut=int(stats[1]), touched=int(stats[2]))


def ep_schedule(src, dst, n: int, C: int, bipartite: bool = False, default_order: bool = False,
                prescreen: bool = False):
    """partition() followed by schedule(); adds 'part'."""
    part = partition(src, dst, n, C, bipartite, default_order, prescreen)
    s = schedule(src, dst, n, part, bipartite)
    s["part"] = part
    return s


# ------------------------------------------------------------ edge kernels (FP64)

def flux(src, dst, x, w):
    """Edge interaction of Section 1's cfd example as a flux kernel.

    For every task e = (u, v): d = x_v - x_u, s = |d|^2, f = w_e d / (1 + s);
    out_u += f and out_v -= f.  x is [D][n]; returns out [D][n] in float64."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    u = np.asarray(src, np.int64)
    v = np.asarray(dst, np.int64)
    d = x[:, v] - x[:, u]
    s = np.sum(d * d, axis=0)
    f = w * d / (1.0 + s)
    out = np.zeros_like(x)
    for c in range(x.shape[0]):
        np.add.at(out[c], u, f[c])
        np.add.at(out[c], v, -f[c])
    return out


def flux_steps(src, dst, x0, w, steps: int, tau: float = 1e-3):
    """Explicit steps x_{t+1} = x_t + tau * flux(x_t); returns (x_T, flux(x_{T-1}))."""
    x = np.array(x0, np.float64)
    out = None
    for _ in range(steps):
        out = flux(src, dst, x, w)
        x = x + tau * out
    return x, out


def spmv(rows, cols, x, w, n_rows: int):
    """y_i = sum over tasks (i, j) of w_e x_j (the SpMV data-affinity kernel)."""
    x = np.asarray(x, np.float64)
    y = np.zeros(n_rows, np.float64)
    np.add.at(y, np.asarray(rows, np.int64), np.asarray(w, np.float64) * x[np.asarray(cols, np.int64)])
    return y


def flux_adjoint(src, dst, x0, w, steps: int, tau: float, g):
    """Reverse-mode gradient of L = <g, x_T> for the explicit flux steps.

    Returns (dL/dx0 [D][n], dL/dw [m]) in float64.  For each step, with
    gbar_e = lam_u - lam_v, d = x_v - x_u, s = |d|^2:
      dw_e   += tau <gbar_e, d> / (1 + s)
      h_e     = w_e (gbar_e / (1 + s) - 2 d (d . gbar_e) / (1 + s)^2)
      lam_t   = lam_{t+1} + tau * (scatter +h_e to v, -h_e to u)."""
    u = np.asarray(src, np.int64)
    v = np.asarray(dst, np.int64)
    w = np.asarray(w, np.float64)
    xs = [np.array(x0, np.float64)]
    for _ in range(steps):
        xs.append(xs[-1] + tau * flux(src, dst, xs[-1], w))
    lam = np.array(g, np.float64)
    dw = np.zeros_like(w)
    for t in range(steps - 1, -1, -1):
        x = xs[t]
        d = x[:, v] - x[:, u]
        s = np.sum(d * d, axis=0)
        gb = lam[:, u] - lam[:, v]
        dg = np.sum(d * gb, axis=0)
        dw += tau * dg / (1.0 + s)
        h = w * (gb / (1.0 + s) - 2.0 * d * dg / (1.0 + s) ** 2)
        new = lam.copy()
        for c in range(lam.shape[0]):
            np.add.at(new[c], v, tau * h[c])
            np.add.at(new[c], u, -tau * h[c])
        lam = new
    return lam, dw
