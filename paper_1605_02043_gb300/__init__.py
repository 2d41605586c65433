"""Edge-partitioned gather/interact/scatter kernels on GB300.

Python face of libepcache (include/epcache.h).  Every call is argument
marshalling into the C ABI: the partition runs in the library's C++ host code,
every per-task and per-vertex computation runs in its CUDA kernels.  There is
no CPU fallback; kernel calls raise when no CUDA device or library is there.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import EpError, check, lib

__all__ = ["Schedule", "PartitionJob", "EpError", "prescreen", "FLUX", "SPMV", "BIPARTITE", "DEFAULT_ORDER", "record_floats",
           "T_EDGE_FWD", "T_BND", "T_EDGE_ADJ", "T_SPMV", "T_LAYOUT", "T_COST"]

FLUX = 0
SPMV = 1
BIPARTITE = 1
DEFAULT_ORDER = 2
PRESCREEN = 4
ORIGINS = ("partition", "default", "path", "star", "low_reuse")  # EP_ORIGIN_*
CACHE_SMEM = 0  # ep_set_cache modes
CACHE_L1 = 1
JOB_TEST_FAIL = 0x100  # test hooks of ep_partition_start (host-side fault injection)
JOB_TEST_HOLD = 0x200
# kernel classes of Schedule.timing_read (EP_T_* in epcache.h)
T_EDGE_FWD, T_BND, T_EDGE_ADJ, T_SPMV, T_LAYOUT, T_COST = range(6)


def _vp(t):
    """Device pointer of a tensor (or None)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need_cuda_f32(t, name, numel=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")


def _edges(src, dst):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    if src.shape != dst.shape or src.ndim != 1:
        raise ValueError("src and dst must be equal-length 1-D arrays")
    return src, dst


class _PrescreenInfo(ctypes.Structure):
    _fields_ = [("touched", ctypes.c_int64), ("degree_sum", ctypes.c_int64),
                ("max_degree", ctypes.c_int64), ("origin", ctypes.c_int32), ("pad", ctypes.c_int32)]


def prescreen(src, dst, n: int, bipartite: bool = False) -> dict:
    """Outcome of the pre-screen (ep_prescreen): degree summary and origin name."""
    src, dst = _edges(src, dst)
    info = _PrescreenInfo()
    check(lib().ep_prescreen(src.ctypes.data, dst.ctypes.data, src.size, n,
                             BIPARTITE if bipartite else 0, ctypes.byref(info)))
    return dict(touched=info.touched, degree_sum=info.degree_sum, max_degree=info.max_degree,
                origin=ORIGINS[info.origin])


def record_floats(D: int) -> int:
    return int(lib().ep_record_floats(D))


class Schedule:
    """A partitioned task schedule (owns host arrays, device copy, workspace)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        m, n, nd, k = (ctypes.c_int64() for _ in range(4))
        C = ctypes.c_int32()
        fl = ctypes.c_uint32()
        check(lib().ep_schedule_info(self._h, *(ctypes.byref(v) for v in (m, n, nd, k, C, fl))))
        self.m, self.n, self.nd, self.k = m.value, n.value, nd.value, k.value
        self.C, self.flags = C.value, fl.value

    # ---------------------------------------------------------------- build
    @classmethod
    def partition(cls, src, dst, n: int, C: int, bipartite: bool = False,
                  default_order: bool = False, threads: int = 0,
                  prescreen: bool = False) -> "Schedule":
        src, dst = _edges(src, dst)
        flags = ((BIPARTITE if bipartite else 0) | (DEFAULT_ORDER if default_order else 0)
                 | (PRESCREEN if prescreen else 0))
        h = ctypes.c_void_p()
        check(lib().ep_partition(src.ctypes.data, dst.ctypes.data, src.size, n, C, flags, threads,
                                 ctypes.byref(h)))
        return cls(h)

    @classmethod
    def batch(cls, parts) -> "Schedule":
        arr = (ctypes.c_void_p * len(parts))(*[p._h for p in parts])
        h = ctypes.c_void_p()
        check(lib().ep_batch(arr, len(parts), ctypes.byref(h)))
        return cls(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().ep_schedule_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bipartite(self) -> bool:
        return bool(self.flags & BIPARTITE)

    @property
    def origin(self) -> str:
        """How the task order was chosen (ORIGINS)."""
        o = ctypes.c_int32()
        check(lib().ep_schedule_origin(self._h, ctypes.byref(o)))
        return ORIGINS[o.value]

    # ---------------------------------------------------------------- views
    def arrays(self) -> dict:
        """Copies of the schedule's host arrays (see ep_schedule_arrays)."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        check(lib().ep_schedule_arrays(self._h, *(ctypes.byref(p) for p in ptrs)))
        loads, cut = self.cost_host()

        def view(p, ctype, count, dtype):
            if count == 0:
                return np.zeros(0, dtype)
            buf = (ctype * count).from_address(p.value)
            return np.frombuffer(buf, dtype=dtype).copy()

        return dict(
            k=self.k,
            block_ptr=view(ptrs[0], ctypes.c_int64, self.k + 1, np.int64),
            edge_perm=view(ptrs[1], ctypes.c_int32, self.m, np.int32),
            vert_ptr=view(ptrs[2], ctypes.c_int64, self.k + 1, np.int64),
            vert_list=view(ptrs[3], ctypes.c_int32, loads, np.int32),
            relabel=view(ptrs[4], ctypes.c_int32, self.nd, np.int32),
            loads=loads, cut=cut,
        )

    def part(self) -> np.ndarray:
        """Block id of every task."""
        a = self.arrays()
        p = np.empty(self.m, np.int32)
        for b in range(self.k):
            p[a["edge_perm"][a["block_ptr"][b]:a["block_ptr"][b + 1]]] = b
        return p

    def cost_host(self):
        loads, cut = ctypes.c_int64(), ctypes.c_int64()
        check(lib().ep_cost_host(self._h, ctypes.byref(loads), ctypes.byref(cut)))
        return loads.value, cut.value

    def cost(self, stream=None):
        """(loads, vertex cut) computed by the GPU sort/unique kernel."""
        loads, cut = ctypes.c_int64(), ctypes.c_int64()
        check(lib().ep_cost(self._h, ctypes.byref(loads), ctypes.byref(cut), _stream(stream)))
        return loads.value, cut.value

    # ------------------------------------------------------------- kernels
    def run(self, x, w, out=None, steps: int = 1, tau: float = 1e-3, kernel: int = FLUX,
            stream=None):
        """Forward run in the caller's layout (see ep_run); x is updated in place."""
        D = 1 if kernel == SPMV else int(x.shape[0])
        nx = self.n if kernel == SPMV else D * self.n
        _need_cuda_f32(x, "x", nx)
        _need_cuda_f32(w, "w", self.m)
        if out is not None:
            _need_cuda_f32(out, "out", nx)
        check(lib().ep_run(self._h, kernel, _vp(x), _vp(w), _vp(out), D, steps, tau, _stream(stream)))
        return x if kernel == FLUX else out

    def run_host(self, x, w, out=None, steps: int = 1, tau: float = 1e-3, kernel: int = FLUX,
                 D: int = 1, stream=None):
        """ep_run_host on host tensors/arrays (pinned memory recommended)."""
        def ptr(a):
            if a is None:
                return None
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        check(lib().ep_run_host(self._h, kernel, ptr(x), ptr(w), ptr(out), D, steps, tau,
                                _stream(stream)))

    def run_adjoint(self, x0, w, lam, grad_w, steps: int, tau: float = 1e-3, stream=None):
        D = int(x0.shape[0])
        for t, nm, k in ((x0, "x0", D * self.n), (lam, "lam", D * self.n), (w, "w", self.m),
                         (grad_w, "grad_w", self.m)):
            _need_cuda_f32(t, nm, k)
        check(lib().ep_run_adjoint(self._h, _vp(x0), _vp(w), _vp(lam), _vp(grad_w), D, steps, tau,
                                   _stream(stream)))

    # ------------------------------------------------------------ tuning
    def set_threads(self, threads: int):
        check(lib().ep_set_threads(self._h, threads))

    def set_adjoint_threads(self, threads: int):
        """Threads that compute per CUDA block in the adjoint kernels (default 352)."""
        check(lib().ep_set_adjoint_threads(self._h, threads))

    def set_pipeline(self, stages: int):
        """0: one CUDA block per kernel block; 2..8: persistent pipelined kernel
        with that many shared-memory stages."""
        check(lib().ep_set_pipeline(self._h, stages))

    def pipeline_info(self, D: int = 5, adjoint: bool = False) -> dict:
        """Launch plan of the pipelined kernels (ep_pipeline_info)."""
        v = [ctypes.c_int32() for _ in range(5)]
        check(lib().ep_pipeline_info(self._h, D, int(adjoint), *(ctypes.byref(x) for x in v)))
        return dict(zip(("grid", "per_sm", "threads", "stages", "stage_bytes"), (x.value for x in v)))

    def check_errors(self, stream=None) -> int:
        """Error word of the pipelined kernels (raises EpError when non-zero)."""
        code = ctypes.c_int32()
        check(lib().ep_check_errors(self._h, ctypes.byref(code), _stream(stream)))
        return code.value

    def set_cache(self, mode: int):
        """CACHE_SMEM (staged, default) or CACHE_L1 (read-only data cache, no staging)
        for forward flux steps."""
        check(lib().ep_set_cache(self._h, mode))

    def debug_stall(self, block_index: int):
        """Test hook: make the pipelined kernels' bounded waits expire (-1 turns it off)."""
        check(lib().ep_debug_stall(self._h, block_index))

    def timing(self, enable: int = 2):
        """Start (2 = clear and start), keep (1) or stop (0) per-kernel timing."""
        check(lib().ep_timing(self._h, enable))

    def timing_read(self, kernel_class: int):
        """(total ms, launches) of one kernel class since the last clear."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        check(lib().ep_timing_read(self._h, kernel_class, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ------------------------------------------------------ schedule layout
    def layout_floats(self, D: int) -> int:
        return int(lib().ep_layout_floats(self._h, D))

    def weights_floats(self) -> int:
        """Length of a task-weight buffer in schedule layout."""
        return int(lib().ep_weights_floats(self._h))

    def layout_in(self, x, x_lay, stream=None):
        check(lib().ep_layout_in(self._h, int(x.shape[0]), _vp(x), _vp(x_lay), _stream(stream)))

    def layout_out(self, x_lay, x, stream=None):
        check(lib().ep_layout_out(self._h, int(x.shape[0]), _vp(x_lay), _vp(x), _stream(stream)))

    def weights_in(self, w, w_lay, stream=None):
        check(lib().ep_weights_in(self._h, _vp(w), _vp(w_lay), _stream(stream)))

    def weights_out_add(self, w_lay, w, stream=None):
        check(lib().ep_weights_out_add(self._h, _vp(w_lay), _vp(w), _stream(stream)))

    def step(self, D: int, x_in, x_out, w_lay, out_lay=None, tau: float = 1e-3, stream=None,
             pending: bool = False):
        """One explicit step in schedule layout (ep_step); pending=True leaves the shared
        copies one step behind (ep_step_pending; no out_lay): finish() before reading."""
        if pending:
            if out_lay is not None:
                raise ValueError("a pending step has no flux output")
            check(lib().ep_step_pending(self._h, D, _vp(x_in), _vp(x_out), _vp(w_lay), tau,
                                        _stream(stream)))
        else:
            check(lib().ep_step(self._h, D, _vp(x_in), _vp(x_out), _vp(w_lay), _vp(out_lay), tau,
                                _stream(stream)))

    def finish(self, D: int, x_lay, tau: float = 1e-3, stream=None):
        """Brings the shared copies of a pending state up to date (ep_finish)."""
        check(lib().ep_finish(self._h, D, _vp(x_lay), tau, _stream(stream)))

    # ------------------------------------------------------------ shard halo
    def set_halo(self, ids):
        """Declares the data vertices other shards touch too (ep_set_halo); rebuilds
        the flux layout.  halo_pack / halo_unpack then move their per-step sums."""
        ids = np.ascontiguousarray(ids, np.int32)
        self._halo_n = int(ids.size)
        check(lib().ep_set_halo(self._h, ctypes.c_void_p(ids.ctypes.data), ids.size))

    def halo_pack(self, D: int, buf, stream=None):
        """Sums of the last forward step at the halo vertices into buf (nh x D, device)."""
        check(lib().ep_halo_pack(self._h, D, _vp(buf), _stream(stream)))

    def halo_unpack(self, D: int, buf, stream=None):
        """buf (the sums over all shards) back into this shard's halo sums."""
        check(lib().ep_halo_unpack(self._h, D, _vp(buf), _stream(stream)))

    def spmv_x_in(self, x, x_lay, stream=None):
        check(lib().ep_spmv_x_in(self._h, _vp(x), _vp(x_lay), _stream(stream)))

    def spmv_y_out(self, y_lay, y, stream=None):
        check(lib().ep_spmv_y_out(self._h, _vp(y_lay), _vp(y), _stream(stream)))

    def spmv(self, x_lay, w_lay, y_lay, stream=None):
        """y_lay = A x_lay in schedule layout (bipartite schedules)."""
        check(lib().ep_spmv(self._h, _vp(x_lay), _vp(w_lay), _vp(y_lay), _stream(stream)))

    def adjoint_step(self, D: int, x_lay, w_lay, lam, grad_w_lay, tau: float = 1e-3, stream=None,
                     pending: bool = False):
        """One adjoint step (ep_adjoint_step); pending=True leaves the shared copies of lam
        one step behind (ep_adjoint_step_pending): adjoint_finish() before reading lam."""
        f = lib().ep_adjoint_step_pending if pending else lib().ep_adjoint_step
        check(f(self._h, D, _vp(x_lay), _vp(w_lay), _vp(lam), _vp(grad_w_lay), tau, _stream(stream)))

    def adjoint_finish(self, D: int, lam, tau: float = 1e-3, stream=None):
        check(lib().ep_adjoint_finish(self._h, D, _vp(lam), tau, _stream(stream)))


class PartitionJob:
    """Schedule.partition on a library-owned host thread (ep_partition_start).

    The optimisation thread of Section 4.2: the caller keeps launching its
    kernel under another schedule and polls; ``cancel`` stops the partitioner
    between bisections.  ``test`` takes JOB_TEST_FAIL or JOB_TEST_HOLD.
    """

    def __init__(self, src, dst, n: int, C: int, bipartite: bool = False, threads: int = 0,
                 prescreen: bool = False, test: int = 0):
        src, dst = _edges(src, dst)
        flags = (BIPARTITE if bipartite else 0) | (PRESCREEN if prescreen else 0) | test
        self._h = ctypes.c_void_p()
        check(lib().ep_partition_start(src.ctypes.data, dst.ctypes.data, src.size, n, C, flags,
                                       threads, ctypes.byref(self._h)))
        self.seconds = None

    def wait(self, timeout: float | None = None) -> bool:
        """True once the job has ended; timeout in seconds (0 polls, None waits)."""
        done = ctypes.c_int32()
        ms = -1 if timeout is None else int(round(timeout * 1000))
        check(lib().ep_job_wait(self._h, ms, ctypes.byref(done)))
        return bool(done.value)

    def done(self) -> bool:
        return self.wait(0)

    def take(self) -> Schedule:
        """The finished schedule; raises EpError with the job's code if it failed."""
        h = ctypes.c_void_p()
        sec = ctypes.c_double()
        rc = lib().ep_job_take(self._h, ctypes.byref(h), ctypes.byref(sec))
        self.seconds = sec.value if rc != -1 else None
        check(rc)
        return Schedule(h)

    def cancel(self):
        check(lib().ep_job_cancel(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().ep_job_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
