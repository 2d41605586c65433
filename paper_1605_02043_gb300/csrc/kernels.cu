// kernels.cu -- device code of libepcache (sm_103a).
//
// The software-cache kernel of Section 4 (Fig. 7(d)), restated for GB300:
// every CUDA block takes one schedule block, copies the distinct vertices of
// that block (the vertex set the cost model of Eq. 1 counts once per block)
// from HBM into shared memory, runs its tasks out of shared memory, and
// writes back once per vertex: vertices no other block uses are updated in
// place with plain stores, shared vertices get one vector atomic add into an
// accumulator, applied to every copy by the next step's fix-up or by the
// finish (bnd_update_kernel).  Also here: the SpMV kernel, the cost kernels,
// the layout conversions and the shard-halo moves.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>
#include <unordered_set>

#include "block_distinct.cuh"
#include "flux_common.cuh"
#include "kernels.h"

namespace ep {
namespace dev {
namespace {

// Shared-memory carve-up of one kernel block (the stage layout of the
// pipelined kernels, one stage): state planes, cotangent planes (adjoint),
// slots, slot weights, shared ids, slice offsets.
struct BlockSmem {
  float* x;
  float* lam;
  uint16_t* sidx;
  float* w;
  int32_t* sid;
  uint16_t* soff;
};
__device__ __forceinline__ BlockSmem block_smem(unsigned char* base, const TmaLayout& L) {
  BlockSmem r;
  r.x = reinterpret_cast<float*>(base);
  r.lam = reinterpret_cast<float*>(base + L.off_lam);
  r.sidx = reinterpret_cast<uint16_t*>(base + L.off_sidx);
  r.w = reinterpret_cast<float*>(base + L.off_w);
  r.sid = reinterpret_cast<int32_t*>(base + L.off_sid);
  r.soff = reinterpret_cast<uint16_t*>(base + L.off_soff);
  return r;
}

// copy `bytes` (a multiple of 16) as 16-byte vectors, the whole CUDA block
__device__ __forceinline__ void copy16(void* dst, const void* src, uint32_t bytes) {
  uint4* d = reinterpret_cast<uint4*>(dst);
  const uint4* s = reinterpret_cast<const uint4*>(src);
  for (uint32_t i = threadIdx.x; i < bytes / 16u; i += blockDim.x) d[i] = __ldg(s + i);
}
__device__ __forceinline__ uint32_t up16(uint32_t b) { return (b + 15u) & ~15u; }

template <int D, int K = 0>
__device__ __forceinline__ void copy_run(float* sx, int npos, const float* gx, int64_t n, int lo, int nv) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    copy16(sx + F * npos, gx + F * n + (int64_t)lo * W, up16((uint32_t)nv * W * 4u));
    copy_run<D, K + 1>(sx, npos, gx, n, lo, nv);
  }
}

// The same pieces the pipelined kernels bulk-copy, moved by the CUDA block's
// threads as 16-byte vectors (every piece is 16-byte aligned and padded).
template <int D>
__device__ __forceinline__ void stage_block(const FluxDesc& d, const FluxArgs& a, const float* lam,
                                            const BlockSmem& S, const TmaLayout& L) {
  copy16(S.sidx, a.sidx + d.s0, (uint32_t)d.nslot * 2u);
  copy16(S.w, a.w + d.s0, (uint32_t)d.nslot * 4u);
  copy16(S.soff, a.soff + d.q0, up16((uint32_t)(d.nsl + 1) * 2u));
  copy16(S.sid, a.sid + d.h0, up16((uint32_t)(d.nv - d.ni) * 4u));
  copy_run<D>(S.x, L.npos, a.x_in, a.n_rec, d.rec_lo, d.nv);
  if (lam) copy_run<D>(S.lam, L.npos, lam, a.n_rec, d.rec_lo, d.nv);
}

// ------------------------------------------------------------- flux forward

// One CUDA block per kernel block: stage, bring the pending shared copies up
// to date, then every warp takes slices of 32 positions (pull form,
// flux_common.cuh).  Only the staged copy is read, so the in-place update of
// the interior records cannot overtake a read.
template <int D>
__global__ void __launch_bounds__(1024) flux_fwd_kernel(const FluxArgs a, TmaLayout L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FluxDesc d = a.desc[blockIdx.x];
  const BlockSmem S = block_smem(smem, L);
  const int q = *a.phase;
  stage_block<D>(d, a, nullptr, S, L);
  __syncthreads();
  fixup_copies<D>(d, S.x, L.npos, S.sid, acc_buffer<D>(a, q + 2), acc_buffer<D>(a, q + 1), a.tau,
                  threadIdx.x, blockDim.x);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int sl = warp; sl < d.nsl; sl += nw)
    fwd_block_slice<D>(a, acc_buffer<D>(a, q), d, S.x, L.npos, S.sidx, S.w, S.soff, S.sid, sl, lane);
  advance_phase(a, q);
}

// Read-only-cache variant: the texture-cache kernel of Section 5 (Fig. 7(c)),
// with the read-only data cache (ld.global.nc) in place of texture binding.
// No staging: slots, weights and states are read from global memory through
// that cache, so it runs on a finished state (no pending copies: the previous
// step's accumulator is zero).  Warp w takes slices w, w + W, ..., up to R of
// them, and keeps their sums in registers; writes wait for a block barrier,
// because interior records are updated in place and other warps may still be
// reading them.
template <int D, int R>
__global__ void __launch_bounds__(1024) flux_fwd_ldg_kernel(const FluxArgs a) {
  const FluxDesc d = a.desc[blockIdx.x];
  const int q = *a.phase;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float xp[R][D], acc[R][D];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int sl = warp + i * nw, p = 32 * sl + lane;
#pragma unroll
    for (int c = 0; c < D; ++c) xp[i][c] = acc[i][c] = 0.f;
    if (sl >= d.nsl) continue;
    const int c0 = __ldg(a.soff + d.q0 + sl), K = __ldg(a.soff + d.q0 + sl + 1) - c0;
    if (p < d.nv) rec_load<D, true>(a.x_in, a.n_rec, (int64_t)d.rec_lo + p, xp[i]);
    const int64_t s = (int64_t)d.s0 + 32 * c0 + lane;
    fwd_slice<D, true>(a.x_in, a.n_rec, d.rec_lo, a.sidx + s, a.w + s, K, xp[i], acc[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int sl = warp + i * nw, p = 32 * sl + lane;
    if (sl >= d.nsl || p >= d.nv) continue;
    if (p < d.ni) {
      float xn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) xn[c] = fmaf(a.tau, acc[i][c], xp[i][c]);
      rec_store<D>(a.x_out, a.n_rec, (int64_t)d.rec_lo + p, xn);
      if (a.out) rec_store<D>(a.out, a.n_rec, (int64_t)d.rec_lo + p, acc[i]);
    } else {  // this step's sum, the clearing, and the copy (x_out may be another buffer)
      const int32_t raw = __ldg(a.sid + d.h0 + p - d.ni);
      acc_red<D>(acc_buffer<D>(a, q), raw & kSidMask, acc[i]);
      if (raw < 0) acc_zero<D>(acc_buffer<D>(a, q + 1), raw & kSidMask);
      rec_store<D>(a.x_out, a.n_rec, (int64_t)d.rec_lo + p, xp[i]);
    }
  }
  advance_phase(a, q);
}

// The finish of a pending state, one thread per copy (fold_rec / fold_sid in
// record order: coalesced record accesses, one dependent round trip;
// flux_common.cuh fold_copies and the accumulator rotation).
template <int D>
__global__ void bnd_update_kernel(const FluxArgs a, const float* x_in, float* x_out, float* out) {
  // launched with programmatic serialisation after the edge kernel: wait for
  // it (the accumulators and records it wrote) before reading
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int q = *a.phase;
  fold_copies<D>(a, x_in, x_out, out, acc_buffer<D>(a, q + 2), acc_buffer<D>(a, q + 1),
                 blockIdx.x * (int64_t)blockDim.x + threadIdx.x, a.n_copies,
                 (int64_t)gridDim.x * blockDim.x);
  advance_phase(a, q);
}

// ------------------------------------------------------------- flux adjoint

// One CUDA block per kernel block, the adjoint step (flux_common.cuh adj_*):
// stage the state (finished) and the cotangent (copies pending), bring the
// cotangent copies up to date, compute.
template <int D>
__global__ void __launch_bounds__(1024) flux_adj_kernel(const FluxArgs a, float* lam, float* gw,
                                                        TmaLayout L) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FluxDesc d = a.desc[blockIdx.x];
  const BlockSmem S = block_smem(smem, L);
  const int q = *a.phase;
  stage_block<D>(d, a, lam, S, L);
  __syncthreads();
  fixup_copies<D>(d, S.lam, L.npos, S.sid, acc_buffer<D>(a, q + 2), acc_buffer<D>(a, q + 1), a.tau,
                  threadIdx.x, blockDim.x);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int sl = warp; sl < d.nsl; sl += nw)
    adj_block_slice<D>(a, acc_buffer<D>(a, q), d, S.x, S.lam, L.npos, S.sidx, S.w, S.soff, S.sid, lam,
                       gw, sl, lane);
  advance_phase(a, q);
}

// --------------------------------------------------------------------- SpMV

// SpMV over the edge partition (Section 5.2), one warp per schedule block.
// The block's entries are ranked by row position and cut into 32 equal
// chunks, one per lane, so every lane does the same work whatever the row
// lengths: a lane walks its chunk in order, summing runs of equal rows in a
// register.  A run that neither starts nor ends the chunk is a whole row and
// is stored at once; the first and last runs of the chunks are joined across
// lanes by a segmented scan over the warp.  Row totals go to a shared array
// and leave it in row order (plain stores for rows of this block alone,
// atomics for shared rows).  With the software cache, x of the block's
// columns is staged in shared memory first; the read-only-cache variant
// reads x through the read-only data cache at every entry.
//
// Per-warp shared region: y totals at [0, ceil4(ny)), staged x after them.
constexpr int kSpmvBatch = 4;  // 16-byte chunks of entries (and weights) in flight per lane
constexpr int kSpmvMaxThreads = 256;

__device__ __forceinline__ int spmv_up4(int v) { return (v + 3) & ~3; }

template <bool STAGE>
__device__ __forceinline__ float spmv_x(const SpmvDesc& d, const int32_t* __restrict__ xlist,
                                        const float* __restrict__ x, const float* xs, uint32_t col) {
  if (STAGE) return xs[col];
  const int c = (int)col;
  return __ldg(x + (c < d.n_xo ? d.x_lo + c : __ldg(xlist + d.fx0 + (c - d.n_xo))));
}

// x of the block's columns into xs: four (id, value) load chains in flight
// per lane
__device__ __forceinline__ void spmv_stage_x(const SpmvDesc& d, const SpmvArgs& a, float* xs, int lane) {
  const int nx = d.n_xo + d.n_xf;
  for (int i0 = lane; i0 < nx; i0 += 4 * 32) {
    int32_t r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u;
      r[u] = i >= nx ? -1 : (i < d.n_xo ? d.x_lo + i : __ldg(a.xlist + d.fx0 + (i - d.n_xo)));
    }
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = r[u] >= 0 ? __ldg(a.x + r[u]) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r[u] >= 0) xs[i0 + 32 * u] = v[u];
  }
}

struct SpmvRun {
  int cur = -1, hrow = -1;  // row of the open run; row of the chunk's first run once closed
  float acc = 0.f, hsum = 0.f;
  bool whole = true;  // no run closed yet: the chunk is one run so far
};

__device__ __forceinline__ void spmv_take(SpmvRun& r, float* ys, uint32_t e, float v) {
  const int row = (int)(e >> kRowShift);
  if (row != r.cur) {
    if (r.cur >= 0) {
      if (r.whole) {
        r.hrow = r.cur;
        r.hsum = r.acc;
        r.whole = false;
      } else {
        ys[r.cur] = r.acc;  // a run inside the chunk: the whole row
      }
    }
    r.cur = row;
    r.acc = v;
  } else {
    r.acc += v;
  }
}

// Four entries (one 16-byte chunk) of this lane; j: their rank in the chunk
template <bool STAGE>
__device__ __forceinline__ void spmv_chunk(SpmvRun& run, float* ys, const float* xs, const SpmvDesc& d,
                                           const SpmvArgs& a, uint4 ev, float4 wv, int j, int nj) {
  const uint32_t e[4] = {ev.x, ev.y, ev.z, ev.w};
  const float w[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (j + q < nj) spmv_take(run, ys, e[q], w[q] * spmv_x<STAGE>(d, a.xlist, a.x, xs, e[q] & kColMask));
}

// Joins the chunks' end runs: lane l's first run continues lane l-1's last
// run when both are the same row, and a lane whose chunk is one run passes
// the sum on (segmented inclusive scan of the last-run sums over the lanes).
// Afterwards every row of the block has its total in ys, stored once.
__device__ __forceinline__ void spmv_join(const SpmvRun& run, float* ys, int lane) {
  const unsigned full = 0xffffffffu;
  const int rt = run.cur, rh = run.whole ? run.cur : run.hrow;
  const int rt_prev = __shfl_up_sync(full, rt, 1);
  const bool cont = lane > 0 && rh >= 0 && rh == rt_prev;
  float S = run.acc;
  int F = !(run.whole && cont);  // a segment starts here
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float Sp = __shfl_up_sync(full, S, o);
    const int Fp = __shfl_up_sync(full, F, o);
    if (lane >= o && !F) {
      S += Sp;
      F = Fp;
    }
  }
  const float S_prev = __shfl_up_sync(full, S, 1);
  const int cont_next = __shfl_down_sync(full, (int)cont, 1);
  if (!run.whole) ys[rh] = run.hsum + (cont ? S_prev : 0.f);
  if (rt >= 0 && !(lane < 31 && cont_next)) ys[rt] = S;
}

// Row totals out: four rows in flight per lane
__device__ __forceinline__ void spmv_write_out(const SpmvDesc& d, const SpmvArgs& a, const float* ys,
                                               int lane) {
  const int ny = d.n_yi + d.n_yob + d.n_yf, own = d.n_yi + d.n_yob;
  for (int p0 = lane; p0 < ny; p0 += 4 * 32) {
    int32_t r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + 32 * u;
      r[u] = p >= ny ? -1
                     : (p < d.n_yi ? d.yi_lo + p
                                   : (p < own ? d.yb_lo + (p - d.n_yi)
                                              : __ldg(a.ylist + d.fy0 + (p - own))));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + 32 * u;
      if (r[u] < 0) continue;
      if (p < d.n_yi)
        a.y[r[u]] = ys[p];
      else
        atomicAdd(a.y + r[u], ys[p]);
    }
  }
}

// One warp per schedule block (one pass, no pipeline): the lane's entries and
// weights are loaded straight into registers while x is staged.
template <bool STAGE>
__global__ void __launch_bounds__(kSpmvMaxThreads) spmv_kernel(const SpmvArgs a, int wpb, int cap) {
  extern __shared__ float4 smem4[];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * wpb + wi;
  if (b >= a.k) return;  // warp-uniform; the warps of a CUDA block never synchronise
  const SpmvDesc d = a.desc[b];
  float* ys = reinterpret_cast<float*>(smem4) + (size_t)wi * cap;
  float* xs = ys + spmv_up4(d.n_yi + d.n_yob + d.n_yf);
  const int nj = min(max(d.ne - lane * d.u, 0), d.u);  // this lane's real entries
  // chunk c of this lane: slots i0 + (32 c + lane) * 4 .. + 3
  const uint4* ep = reinterpret_cast<const uint4*>(a.ent + d.i0) + lane;
  const float4* wp = reinterpret_cast<const float4*>(a.w + d.i0) + lane;
  uint4 ev[kSpmvBatch];
  float4 wv[kSpmvBatch];
#pragma unroll
  for (int c = 0; c < kSpmvBatch; ++c)
    if (4 * c < nj) {
      ev[c] = __ldg(ep + 32 * c);
      wv[c] = __ldg(wp + 32 * c);
    }
  if (STAGE) {
    spmv_stage_x(d, a, xs, lane);
    __syncwarp();
  }
  SpmvRun run;
  for (int c0 = 0; 4 * c0 < nj; c0 += kSpmvBatch) {
    if (c0 > 0) {
#pragma unroll
      for (int c = 0; c < kSpmvBatch; ++c)
        if (4 * (c0 + c) < nj) {
          ev[c] = __ldg(ep + 32 * (c0 + c));
          wv[c] = __ldg(wp + 32 * (c0 + c));
        }
    }
#pragma unroll
    for (int c = 0; c < kSpmvBatch; ++c) spmv_chunk<STAGE>(run, ys, xs, d, a, ev[c], wv[c], 4 * (c0 + c), nj);
  }
  spmv_join(run, ys, lane);
  __syncwarp();
  spmv_write_out(d, a, ys, lane);
}

// ------------------------------------------------------------- shard halo

// Halo sums of a shard schedule (one of several that split a schedule's
// blocks): hmap[i] is the shared id of halo vertex i here, or -1 where this
// shard does not touch it.  Pack copies the sums of the last forward edge
// kernel (the accumulator buffer before the current phase) into buf[i][D]
// (zeros for -1); unpack writes buf back after the sum over shards.
template <int D>
__global__ void halo_kernel(const FluxArgs a, const int32_t* __restrict__ hmap, int64_t nh,
                            float* __restrict__ buf, bool pack) {
  float* last = acc_buffer<D>(a, *a.phase + 2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nh;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t h = __ldg(hmap + i);
    float v[D];
    if (pack) {
#pragma unroll
      for (int c = 0; c < D; ++c) v[c] = 0.f;
      if (h >= 0) acc_load<D>(last, h, v);
#pragma unroll
      for (int c = 0; c < D; ++c) buf[i * D + c] = v[c];
    } else if (h >= 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) v[c] = buf[i * D + c];
      acc_store<D>(last, h, v);
    }
  }
}

// ------------------------------------------------------------------- layout

// caller layout [D][n] (by data vertex) <-> planar records (by record id)
template <int D>
__global__ void layout_in_kernel(const int32_t* __restrict__ rec_of, int64_t n, int64_t n_rec,
                                 const float* __restrict__ x, float* __restrict__ x_lay) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    float t[D];
#pragma unroll
    for (int c = 0; c < D; ++c) t[c] = __ldg(x + (size_t)c * n + v);
    rec_store<D>(x_lay, n_rec, __ldg(rec_of + v), t);
  }
}

// flux layout in: x read in vertex order (coalesced; in host memory the GPU
// reads it over the host link), every record of vertex v written (its record
// and the copies of a shared vertex): recs[ptr[v] .. ptr[v + 1])
template <int D>
__global__ void layout_in_csr_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ recs,
                                     int64_t n, int64_t n_rec, const float* __restrict__ x,
                                     float* __restrict__ x_lay) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    float t[D];
#pragma unroll
    for (int c = 0; c < D; ++c) t[c] = x[(size_t)c * n + v];
    for (int32_t i = __ldg(ptr + v), e = __ldg(ptr + v + 1); i < e; ++i) rec_store<D>(x_lay, n_rec, __ldg(recs + i), t);
  }
}

// w read in task order, written to the task's slots (two, -1 for none)
__global__ void weights_scatter_kernel(const int2* __restrict__ slots, int64_t m, const float* __restrict__ w,
                                       float* __restrict__ w_lay) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float v = w[t];
    const int2 sl = __ldg(slots + t);
    if (sl.x >= 0) w_lay[sl.x] = v;
    if (sl.y >= 0) w_lay[sl.y] = v;
  }
}

template <int D>
__global__ void layout_out_kernel(const int32_t* __restrict__ rec_of, int64_t n, int64_t n_rec,
                                  const float* __restrict__ x_lay, float* __restrict__ x) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    float t[D];
    rec_load<D, true>(x_lay, n_rec, __ldg(rec_of + v), t);
#pragma unroll
    for (int c = 0; c < D; ++c) x[(size_t)c * n + v] = t[c];
  }
}

__global__ void gather_kernel(const int32_t* __restrict__ perm, int64_t m, const float* __restrict__ w,
                              float* __restrict__ w_lay) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
  {
    const int32_t t = perm[i];
    w_lay[i] = t >= 0 ? __ldg(w + t) : 0.f;
  }
}

__global__ void scatter_add_kernel(const int32_t* __restrict__ perm, int64_t m,
                                   const float* __restrict__ w_lay, float* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
  {
    const int32_t t = perm[i];
    if (t >= 0) w[t] += w_lay[i];
  }
}

__global__ void gather_add_kernel(const int32_t* __restrict__ slot, int64_t m,
                                  const float* __restrict__ w_lay, float* __restrict__ w) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    w[t] += __ldg(w_lay + __ldg(slot + t));
}

// --------------------------------------------------------------------- cost

// One CUDA block per schedule block: bitonic sort of the block's endpoint ids
// in shared memory, then count distinct ids and mark them touched.
__global__ void cost_block_kernel(const int64_t* __restrict__ block_ptr, const int32_t* __restrict__ eu,
                                  const int32_t* __restrict__ ev, int P, uint8_t* __restrict__ touched,
                                  unsigned long long* __restrict__ loads) {
  extern __shared__ float4 smem4[];
  int32_t* key = reinterpret_cast<int32_t*>(smem4);
  const int64_t e0 = block_ptr[blockIdx.x];
  const int ne = (int)(block_ptr[blockIdx.x + 1] - e0);
  const int nk = 2 * ne;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    key[i] = i < ne ? eu[e0 + i] : i < nk ? ev[e0 + i - ne] : INT_MAX;
  __syncthreads();
  block_bitonic_sort(key, P);
  const unsigned int cnt = count_distinct_sorted(key, nk, [&](int32_t v) { touched[v] = 1; });
  block_sum_add(cnt, loads);
}

__global__ void count_flags_kernel(const uint8_t* __restrict__ f, int64_t nd,
                                   unsigned long long* __restrict__ total) {
  sum_flags(f, nd, total);
}

int grid_for(int64_t work, int tpb) {
  int64_t g = (work + tpb - 1) / tpb;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

// Opens a kernel's dynamic shared-memory limit to the device maximum once
// (a per-kernel attribute shared by all callers); launches above 48 KB need it.
std::mutex g_smem_mu;
std::unordered_set<const void*> g_smem_opened;  // kernels whose limit is open

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // minus the kernel's static shared memory
  if (bytes > (size_t)dyn_max) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_smem_mu);
  const void* key = reinterpret_cast<const void*>(kernel);
  if (g_smem_opened.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e == cudaSuccess) g_smem_opened.insert(key);
  return e;
}

struct Scope {
  Timer* t;
  int cls;
  cudaStream_t st;
  Scope(Timer* t_, int c, cudaStream_t s) : t(t_), cls(c), st(s) {
    if (t) t->begin(cls, st);
  }
  ~Scope() {
    if (t) t->end(cls, st);
  }
};

// PDL launch of the finish (the edge kernel before it may still be draining)
template <int D>
cudaError_t fold_launch(const FluxArgs& a, float* x_out, const float* x_in, float* out, cudaStream_t st) {
  if (a.n_sh <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_for((a.n_copies + kFoldUnroll - 1) / kFoldUnroll, 256));
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bnd_update_kernel<D>, a, x_in, x_out, out);
}

template <int D>
cudaError_t flux_step_t(const FluxArgs& a, cudaStream_t st) {
  const TmaLayout L = tma_layout(a, D, false);
  const size_t smem = (size_t)L.stage_bytes;
  cudaError_t e = allow_smem(flux_fwd_kernel<D>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_FWD, st);
    flux_fwd_kernel<D><<<(unsigned)a.k, a.tpb, smem, st>>>(a, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int D, int R>
void flux_ldg_launch(const FluxArgs& a, int threads, cudaStream_t st) {
  flux_fwd_ldg_kernel<D, R><<<(unsigned)a.k, threads, 0, st>>>(a);
}

template <int D>
cudaError_t flux_step_ldg_t(const FluxArgs& a, cudaStream_t st) {
  const int R = (a.max_nsl + 31) / 32;  // slices per warp
  const int threads = 32 * std::max(1, (a.max_nsl + R - 1) / std::max(R, 1));
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_FWD, st);
    switch (R) {
      case 0:
      case 1: flux_ldg_launch<D, 1>(a, threads, st); break;
      case 2: flux_ldg_launch<D, 2>(a, threads, st); break;
      case 3: flux_ldg_launch<D, 3>(a, threads, st); break;
      case 4: flux_ldg_launch<D, 4>(a, threads, st); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  return cudaSuccess;
}

template <int D>
cudaError_t flux_adj_t(const FluxArgs& a, float* lam, float* gw, cudaStream_t st) {
  const TmaLayout L = tma_layout(a, D, true);
  const size_t smem = (size_t)L.stage_bytes;
  cudaError_t e = allow_smem(flux_adj_kernel<D>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_ADJ, st);
    flux_adj_kernel<D><<<(unsigned)a.k, a.tpb, smem, st>>>(a, lam, gw, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t flux_step(const FluxArgs& a, int D, cudaStream_t st) {
  switch (D) {
    case 1: return flux_step_t<1>(a, st);
    case 2: return flux_step_t<2>(a, st);
    case 3: return flux_step_t<3>(a, st);
    case 4: return flux_step_t<4>(a, st);
    case 5: return flux_step_t<5>(a, st);
    case 6: return flux_step_t<6>(a, st);
    case 7: return flux_step_t<7>(a, st);
    case 8: return flux_step_t<8>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t flux_step_ldg(const FluxArgs& a, int D, cudaStream_t st) {
  switch (D) {
    case 1: return flux_step_ldg_t<1>(a, st);
    case 2: return flux_step_ldg_t<2>(a, st);
    case 3: return flux_step_ldg_t<3>(a, st);
    case 4: return flux_step_ldg_t<4>(a, st);
    case 5: return flux_step_ldg_t<5>(a, st);
    case 6: return flux_step_ldg_t<6>(a, st);
    case 7: return flux_step_ldg_t<7>(a, st);
    case 8: return flux_step_ldg_t<8>(a, st);
  }
  return cudaErrorInvalidValue;
}

#define EP_DISPATCH_D(D, CALL) \
  switch (D) {                    \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    case 7: CALL(7); break;       \
    case 8: CALL(8); break;       \
    default: return cudaErrorInvalidValue; \
  }

// shared-vertex fold after a pipelined edge kernel
cudaError_t bnd_update(const FluxArgs& a, int D, float* x_out, const float* x_in, float* out,
                       cudaStream_t st) {
  if (a.n_sh <= 0) return cudaSuccess;
  Scope sc(a.timer, T_BND, st);
#define EP_BU(DD) return fold_launch<DD>(a, x_out, x_in, out, st)
  switch (D) {
    case 1: EP_BU(1);
    case 2: EP_BU(2);
    case 3: EP_BU(3);
    case 4: EP_BU(4);
    case 5: EP_BU(5);
    case 6: EP_BU(6);
    case 7: EP_BU(7);
    case 8: EP_BU(8);
  }
#undef EP_BU
  return cudaErrorInvalidValue;
}

TmaLayout tma_layout(const FluxArgs& a, int D, bool adjoint) {
  auto up = [](int64_t x, int64_t m) { return (x + m - 1) / m * m; };
  TmaLayout L = {};
  L.npos = (int)up(a.max_nv, 4);
  const int64_t xb = (int64_t)D * L.npos * 4;
  L.off_lam = (int)xb;
  L.off_sidx = (int)(L.off_lam + (adjoint ? xb : 0));
  L.off_w = (int)(L.off_sidx + up((int64_t)a.max_nslot * 2, 16));
  L.off_sid = (int)(L.off_w + (int64_t)a.max_nslot * 4);
  L.off_soff = (int)(L.off_sid + up((int64_t)a.max_nsh * 4, 16));
  L.off_desc = (int)(L.off_soff + up((int64_t)(a.max_nsl + 1) * 2, 16));
  L.stage_bytes = (int)up(L.off_desc + (int64_t)sizeof(FluxDesc), 128);
  L.stages = 1;
  L.stall = -1;
  return L;
}

cudaError_t flux_adjoint_step(const FluxArgs& a, int D, float* lam, float* gw, cudaStream_t st) {
  switch (D) {
    case 1: return flux_adj_t<1>(a, lam, gw, st);
    case 2: return flux_adj_t<2>(a, lam, gw, st);
    case 3: return flux_adj_t<3>(a, lam, gw, st);
    case 4: return flux_adj_t<4>(a, lam, gw, st);
    case 5: return flux_adj_t<5>(a, lam, gw, st);
    case 6: return flux_adj_t<6>(a, lam, gw, st);
    case 7: return flux_adj_t<7>(a, lam, gw, st);
    case 8: return flux_adj_t<8>(a, lam, gw, st);
  }
  return cudaErrorInvalidValue;
}

size_t flux_block_smem(const FluxArgs& a, int D, bool adjoint) {
  return (size_t)tma_layout(a, D, adjoint).stage_bytes;
}

SpmvPlan spmv_plan(const SpmvArgs& a, int smem_optin) {
  SpmvPlan P = {};
  int wpb = std::max(1, std::min(kSpmvMaxThreads / 32, a.tpb / 32));
  P.cap = a.readonly ? (a.max_ny + 3) & ~3 : a.max_nxy;
  const size_t per_warp = (size_t)P.cap * sizeof(float);
  while (wpb > 1 && per_warp * wpb > (size_t)48 * 1024) --wpb;  // room for several CUDA blocks per SM
  P.smem = per_warp * wpb;
  P.wpb = P.smem + 1024 <= (size_t)smem_optin ? wpb : 0;
  return P;
}

cudaError_t spmv(const SpmvArgs& a, cudaStream_t st) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const SpmvPlan P = spmv_plan(a, optin);
  if (P.wpb == 0) return cudaErrorInvalidValue;
  e = a.readonly ? allow_smem(spmv_kernel<false>, P.smem) : allow_smem(spmv_kernel<true>, P.smem);
  if (e != cudaSuccess) return e;
  if (a.ny_zero > 0) {
    e = cudaMemsetAsync(a.y + a.ny_int, 0, (size_t)a.ny_zero * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  if (a.k <= 0) return cudaSuccess;
  Scope sc(a.timer, T_SPMV, st);
  const unsigned grid = (unsigned)((a.k + P.wpb - 1) / P.wpb);
  if (a.readonly)
    spmv_kernel<false><<<grid, 32 * P.wpb, P.smem, st>>>(a, P.wpb, P.cap);
  else
    spmv_kernel<true><<<grid, 32 * P.wpb, P.smem, st>>>(a, P.wpb, P.cap);
  return cudaGetLastError();
}

cudaError_t layout_in(const int32_t* rec_of, int64_t n, int64_t n_rec, int D, const float* x,
                      float* x_lay, cudaStream_t st, Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  const int g = grid_for(n, 256);
#define EP_LIN(DD) layout_in_kernel<DD><<<g, 256, 0, st>>>(rec_of, n, n_rec, x, x_lay)
  EP_DISPATCH_D(D, EP_LIN)
#undef EP_LIN
  return cudaGetLastError();
}

cudaError_t halo_move(const FluxArgs& a, int D, const int32_t* hmap, int64_t nh, float* buf, bool pack,
                      cudaStream_t st) {
  if (nh <= 0) return cudaSuccess;
  const int g = grid_for(nh, 256);
#define EP_HALO(DD) halo_kernel<DD><<<g, 256, 0, st>>>(a, hmap, nh, buf, pack)
  EP_DISPATCH_D(D, EP_HALO)
#undef EP_HALO
  return cudaGetLastError();
}

cudaError_t layout_in_csr(const int32_t* ptr, const int32_t* recs, int64_t n, int64_t n_rec, int D,
                          const float* x, float* x_lay, cudaStream_t st, Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  const int g = grid_for(n, 256);
#define EP_LIN(DD) layout_in_csr_kernel<DD><<<g, 256, 0, st>>>(ptr, recs, n, n_rec, x, x_lay)
  EP_DISPATCH_D(D, EP_LIN)
#undef EP_LIN
  return cudaGetLastError();
}

cudaError_t weights_scatter(const int32_t* slots, int64_t m, const float* w, float* w_lay, cudaStream_t st,
                            Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  weights_scatter_kernel<<<grid_for(m, 256), 256, 0, st>>>(reinterpret_cast<const int2*>(slots), m, w, w_lay);
  return cudaGetLastError();
}

cudaError_t layout_out(const int32_t* rec_of, int64_t n, int64_t n_rec, int D, const float* x_lay,
                       float* x, cudaStream_t st, Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  const int g = grid_for(n, 256);
#define EP_LOUT(DD) layout_out_kernel<DD><<<g, 256, 0, st>>>(rec_of, n, n_rec, x_lay, x)
  EP_DISPATCH_D(D, EP_LOUT)
#undef EP_LOUT
  return cudaGetLastError();
}

cudaError_t gather(const int32_t* perm, int64_t m, const float* w, float* w_lay, cudaStream_t st,
                   Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  gather_kernel<<<grid_for(m, 256), 256, 0, st>>>(perm, m, w, w_lay);
  return cudaGetLastError();
}

cudaError_t scatter_add(const int32_t* perm, int64_t m, const float* w_lay, float* w, cudaStream_t st,
                        Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  scatter_add_kernel<<<grid_for(m, 256), 256, 0, st>>>(perm, m, w_lay, w);
  return cudaGetLastError();
}

cudaError_t gather_add(const int32_t* slot, int64_t m, const float* w_lay, float* w, cudaStream_t st,
                       Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  gather_add_kernel<<<grid_for(m, 256), 256, 0, st>>>(slot, m, w_lay, w);
  return cudaGetLastError();
}

cudaError_t cost(const CostArgs& a, cudaStream_t st) {
  int P = 2;
  while (P < 2 * a.max_ne) P <<= 1;
  const size_t smem = (size_t)P * sizeof(int32_t);
  cudaError_t e = allow_smem(cost_block_kernel, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.touched, 0, (size_t)a.nd, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counters, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int tpb = P >= 1024 ? 1024 : (P < 32 ? 32 : P);  // whole warps for the shuffles
  Scope sc(a.timer, T_COST, st);
  cost_block_kernel<<<(unsigned)a.k, tpb, smem, st>>>(a.block_ptr, a.eu, a.ev, P, a.touched, a.counters);
  count_flags_kernel<<<grid_for(a.nd, 256), 256, 0, st>>>(a.touched, a.nd, a.counters + 1);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace ep
