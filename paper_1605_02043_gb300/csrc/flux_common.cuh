// flux_common.cuh -- device pieces shared by every flux kernel (sm_103a).
//
// The interaction is the particle kernel of the cfd example (Section 1):
// task e = (u, v) with weight w_e gives f_e = w_e (x_v - x_u) / (1 + |x_v - x_u|^2),
// out_u += f_e, out_v -= f_e.  The kernels compute it in pull form: the lane
// that owns position p sums c (x_o - x_p), c = w / (1 + |x_o - x_p|^2), over the
// slots of p; IEEE subtraction is exactly antisymmetric, so the two endpoints
// of a task add exactly +f_e and -f_e.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace ep {
namespace dev {

// The D components of a record live in planes of width 4, 2 and 1
// (D = 4a + 2b + c).  Plane k starts at component first(k): in a buffer of
// n records it is the float range [first(k) * n, (first(k) + width(k)) * n).
template <int D>
struct Planes {
  static constexpr int A = D / 4, B = (D % 4) / 2, C1 = D % 2;
  static constexpr int NP = A + B + C1;
  __host__ __device__ static constexpr int width(int k) { return k < A ? 4 : (k < A + B ? 2 : 1); }
  __host__ __device__ static constexpr int first(int k) {
    return k < A ? 4 * k : (k < A + B ? 4 * A + 2 * (k - A) : 4 * A + 2 * B);
  }
};

// Accumulator records of the shared vertices: array of structures with a
// 16-byte (D <= 4) or 32-byte stride, so one record is one 32-byte sector.
__host__ __device__ constexpr int acc_stride(int D) { return D <= 4 ? 4 : 8; }

template <int W>
__device__ __forceinline__ void vld(const float* p, float* v) {
  if constexpr (W == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else if constexpr (W == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x, v[1] = t.y;
  } else {
    v[0] = *p;
  }
}
template <int W>
__device__ __forceinline__ void vld_nc(const float* __restrict__ p, float* v) {
  if constexpr (W == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else if constexpr (W == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x, v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}
template <int W>
__device__ __forceinline__ void vst(float* p, const float* v) {
  if constexpr (W == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if constexpr (W == 2)
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  else
    *p = v[0];
}
// fire-and-forget vector reductions into global memory (no value returned,
// so the issuing warp never waits for them)
template <int W>
__device__ __forceinline__ void vred(float* p, const float* v) {
  if constexpr (W == 4)
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
  else if constexpr (W == 2)
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v[0]), "f"(v[1]) : "memory");
  else
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v[0]) : "memory");
}

// Record r of a planar buffer of n records <-> registers v[0..D), one vector
// access per plane.  NC: through the read-only data cache.
template <int D, bool NC = false, int K = 0>
__device__ __forceinline__ void rec_load(const float* base, int64_t n, int64_t r, float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    if constexpr (NC)
      vld_nc<W>(base + F * n + r * W, v + F);
    else
      vld<W>(base + F * n + r * W, v + F);
    rec_load<D, NC, K + 1>(base, n, r, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void rec_store(float* base, int64_t n, int64_t r, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vst<W>(base + F * n + r * W, v + F);
    rec_store<D, K + 1>(base, n, r, v);
  }
}
// accumulator record h (array of structures) <-> registers
template <int D, int K = 0>
__device__ __forceinline__ void acc_red(float* bacc, int64_t h, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vred<W>(bacc + h * acc_stride(D) + F, v + F);
    acc_red<D, K + 1>(bacc, h, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void acc_load(const float* bacc, int64_t h, float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vld<W>(bacc + h * acc_stride(D) + F, v + F);
    acc_load<D, K + 1>(bacc, h, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void acc_store(float* bacc, int64_t h, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vst<W>(bacc + h * acc_stride(D) + F, v + F);
    acc_store<D, K + 1>(bacc, h, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void acc_zero(float* bacc, int64_t h) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    const float z[4] = {0.f, 0.f, 0.f, 0.f};
    vst<W>(bacc + h * acc_stride(D) + F, z);
    acc_zero<D, K + 1>(bacc, h);
  }
}

// One slot of the forward pull: acc += w (x_o - x_p) / (1 + |x_o - x_p|^2).
template <int D, bool NC>
__device__ __forceinline__ void fwd_entry(const float* xs, int64_t n, int64_t base, uint16_t e, float wt,
                                          const float* xp, float* acc) {
  float xo[D];
  rec_load<D, NC>(xs, n, base + (e & kSlotPos), xo);
  float q = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    xo[c] -= xp[c];
    q = fmaf(xo[c], xo[c], q);
  }
  const float coef = __fdividef(wt, 1.f + q);
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = fmaf(coef, xo[c], acc[c]);
}

// Forward pull of one lane over the K columns of its slice.  xs: the state
// planes (n records, positions offset by `base`), ix / wv: the lane's first
// slot (the next column is 32 slots further).  Unused slots add exactly zero.
// kSlotUnroll slots per iteration: their loads are independent, so they are
// all in flight before the arithmetic.
constexpr int kSlotUnroll = 2;
template <int D, bool NC>
__device__ __forceinline__ void fwd_slice(const float* xs, int64_t n, int64_t base,
                                          const uint16_t* ix, const float* wv, int K,
                                          const float* xp, float* acc) {
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = 0.f;
  int k = 0;
  for (; k + kSlotUnroll <= K; k += kSlotUnroll) {
    uint16_t e[kSlotUnroll];
    float wt[kSlotUnroll];
#pragma unroll
    for (int u = 0; u < kSlotUnroll; ++u) {
      e[u] = NC ? __ldg(ix + 32 * (k + u)) : ix[32 * (k + u)];
      wt[u] = NC ? __ldg(wv + 32 * (k + u)) : wv[32 * (k + u)];
    }
#pragma unroll
    for (int u = 0; u < kSlotUnroll; ++u) fwd_entry<D, NC>(xs, n, base, e[u], wt[u], xp, acc);
  }
  for (; k < K; ++k) {
    const uint16_t e = NC ? __ldg(ix + 32 * k) : ix[32 * k];
    const float wt = NC ? __ldg(wv + 32 * k) : wv[32 * k];
    fwd_entry<D, NC>(xs, n, base, e, wt, xp, acc);
  }
}

// Adjoint pull of one lane (reverse step at state x, cotangent lam): for the
// slot to other position o, d = x_o - x_p, g = lam_p - lam_o, q = |d|^2,
// acc -= w (g / (1 + q) - 2 d (d.g) / (1 + q)^2); the source-side slot of a
// task adds tau (d.g) / (1 + q) to the task's weight gradient (gslot: that
// slot's weight-gradient element; one writer per task).
template <int D>
__device__ __forceinline__ void adj_slice(const float* xs, const float* ls, int64_t n,
                                          const uint16_t* ix, const float* wv, int K,
                                          const float* xp, const float* lp, float* acc,
                                          float* __restrict__ gslot, float tau) {
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = 0.f;
  for (int k = 0; k < K; ++k) {  // an unused slot (w = 0, own position) adds zero
    const uint16_t e = ix[32 * k];
    const float we = wv[32 * k];
    const int o = e & kSlotPos;
    float xo[D], lo[D];
    rec_load<D>(xs, n, o, xo);
    rec_load<D>(ls, n, o, lo);
    float q = 0.f, dg = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      xo[c] -= xp[c];        // d
      lo[c] = lp[c] - lo[c];  // g
      q = fmaf(xo[c], xo[c], q);
      dg = fmaf(xo[c], lo[c], dg);
    }
    const float inv = __fdividef(1.f, 1.f + q);
    const float two = 2.f * dg * inv * inv;
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] -= we * (lo[c] * inv - two * xo[c]);
    // fire-and-forget reduction: no load on the critical path
    if (e & kSlotSrc) atomicAdd(gslot + 32 * k, tau * dg * inv);
  }
}

// One slice of a forward kernel block staged in shared memory (xs: state
// planes of npos positions, ix / wv / soff / ssid: the block's slots, slot
// weights, slice offsets and shared ids; the shared copies already brought up
// to date by fixup_copies): lane `lane` sums the flux at its position and
// writes back, x_out = x + tau * flux in place for a vertex only this block
// uses (and out = flux if requested); for a shared vertex one vector
// reduction of its partial flux into this step's accumulator, and its
// up-to-date value into this block's copy.
template <int D>
__device__ __forceinline__ void fwd_block_slice(const FluxArgs& a, float* bacc, const FluxDesc& d,
                                                const float* xs, int npos, const uint16_t* ix,
                                                const float* wv, const uint16_t* soff,
                                                const int32_t* ssid, int sl, int lane) {
  const int p = 32 * sl + lane;
  const int c0 = soff[sl], K = soff[sl + 1] - c0;
  float xp[D], acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) xp[c] = 0.f;
  if (p < d.nv) rec_load<D>(xs, npos, p, xp);
  fwd_slice<D, false>(xs, npos, 0, ix + 32 * c0 + lane, wv + 32 * c0 + lane, K, xp, acc);
  if (p >= d.nv) return;
  if (p < d.ni) {
    float xn[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xn[c] = fmaf(a.tau, acc[c], xp[c]);
    rec_store<D>(a.x_out, a.n_rec, (int64_t)d.rec_lo + p, xn);
    if (a.out) rec_store<D>(a.out, a.n_rec, (int64_t)d.rec_lo + p, acc);
  } else {
    acc_red<D>(bacc, ssid[p - d.ni] & kSidMask, acc);
    rec_store<D>(a.x_out, a.n_rec, (int64_t)d.rec_lo + p, xp);  // this copy, brought up to date
  }
}

// One slice of an adjoint kernel block staged in shared memory (xs, ls: state
// and cotangent planes, the cotangent copies already brought up to date):
// lam_p += tau * acc in place for a vertex only this block uses; for a shared
// vertex one reduction into this step's accumulator and its up-to-date value
// into this block's copy; gw is the weight gradient in slot layout.
template <int D>
__device__ __forceinline__ void adj_block_slice(const FluxArgs& a, float* bacc, const FluxDesc& d,
                                                const float* xs, const float* ls, int npos,
                                                const uint16_t* ix, const float* wv,
                                                const uint16_t* soff, const int32_t* ssid, float* lam,
                                                float* gw, int sl, int lane) {
  const int p = 32 * sl + lane;
  const int c0 = soff[sl], K = soff[sl + 1] - c0;
  float xp[D], lp[D], acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) xp[c] = lp[c] = 0.f;
  if (p < d.nv) {
    rec_load<D>(xs, npos, p, xp);
    rec_load<D>(ls, npos, p, lp);
  }
  adj_slice<D>(xs, ls, npos, ix + 32 * c0 + lane, wv + 32 * c0 + lane, K, xp, lp, acc,
               gw + d.s0 + 32 * c0 + lane, a.tau);
  if (p >= d.nv) return;
  if (p < d.ni) {
#pragma unroll
    for (int c = 0; c < D; ++c) lp[c] = fmaf(a.tau, acc[c], lp[c]);
    rec_store<D>(lam, a.n_rec, (int64_t)d.rec_lo + p, lp);
  } else {
    acc_red<D>(bacc, ssid[p - d.ni] & kSidMask, acc);
    rec_store<D>(lam, a.n_rec, (int64_t)d.rec_lo + p, lp);  // this copy, brought up to date
  }
}

// Shared vertices between steps.  Each kernel block keeps its own copy of
// every shared vertex it uses; an edge kernel adds the block's partial sums
// for them into an accumulator and leaves the copies one step behind
// ("pending"): the next edge kernel brings each staged copy up to date
// (x += tau * accumulator of the previous step) before it computes, and a
// finish pass does the same in memory when the state itself is needed.  The
// accumulators rotate through three buffers, with the phase Q (0..2) of each
// kind (forward, adjoint) in device memory, so a captured CUDA graph replays
// correctly whatever its number of steps:
//   an edge kernel at phase Q  reads buffer Q+2 (the previous step's sums),
//                              adds into buffer Q, and the first copy of each
//                              shared vertex clears it in buffer Q+1;
//   a finish at phase Q        reads buffer Q+2 into every copy and clears
//                              buffer Q+1;
//   both then advance the phase to Q+1 (indices mod 3).
// The buffer an edge kernel clears was last read by the step before it, the
// one it adds into was cleared by the step before it, and a finish leaves the
// buffer the next step reads cleared, so no buffer is ever read and cleared
// by the same launch.
__device__ __forceinline__ int acc_slot(int q) { return q % 3; }
template <int D>
__device__ __forceinline__ float* acc_buffer(const FluxArgs& a, int q) {
  return a.bacc + acc_slot(q) * a.n_sh * acc_stride(D);
}

// Brings the staged copies of shared positions [ni, nv) up to date in shared
// memory (xs, npos positions per plane): x += tau * prev[h]; the first copy of
// h clears h in `next`.  Positions ni + i0, ni + i0 + stride, ..., up to four
// per iteration with their loads in flight together.
template <int D>
__device__ __forceinline__ void fixup_copies(const FluxDesc& d, float* xs, int npos, const int32_t* ssid,
                                             const float* prev, float* next, float tau, int i0,
                                             int stride) {
  const int nsh = d.nv - d.ni;
  for (int i = i0; i < nsh; i += 4 * stride) {
    int32_t raw[4];
    float acc[4][D];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = i + u * stride;
      raw[u] = j < nsh ? ssid[j] : 0;
      if (j < nsh) acc_load<D>(prev, raw[u] & kSidMask, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = i + u * stride;
      if (j >= nsh) continue;
      float x[D];
      rec_load<D>(xs, npos, d.ni + j, x);
#pragma unroll
      for (int c = 0; c < D; ++c) x[c] = fmaf(tau, acc[u][c], x[c]);
      rec_store<D>(xs, npos, d.ni + j, x);
      if (raw[u] < 0) acc_zero<D>(next, raw[u] & kSidMask);
    }
  }
}

// The finish over copies i0, i0 + stride, ... below i1, U copies per
// iteration (their loads are in flight together).  Copy r of shared vertex h:
// x_out[r] = x_in[r] + tau * prev[h] (every copy holds the same value, so every
// copy ends with the same new value), out[r] = prev[h] if out is not null;
// the first copy of h clears h in `next`.
constexpr int kFoldUnroll = 2;
template <int D, int U = kFoldUnroll>
__device__ __forceinline__ void fold_copies(const FluxArgs& a, const float* x_in, float* x_out,
                                            float* out, const float* prev, float* next, int64_t i0,
                                            int64_t i1, int64_t stride) {
  for (int64_t i = i0; i < i1; i += U * stride) {
    int32_t raw[U];
    int64_t r[U];
    float acc[U][D], x[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = i + u * stride;
      raw[u] = j < i1 ? __ldg(a.fold_sid + j) : 0;
      r[u] = j < i1 ? __ldg(a.fold_rec + j) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (r[u] >= 0) {
        acc_load<D>(prev, raw[u] & kSidMask, acc[u]);
        rec_load<D>(x_in, a.n_rec, r[u], x[u]);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (r[u] >= 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) x[u][c] = fmaf(a.tau, acc[u][c], x[u][c]);
        rec_store<D>(x_out, a.n_rec, r[u], x[u]);
        if (out) rec_store<D>(out, a.n_rec, r[u], acc[u]);
        if (raw[u] < 0) acc_zero<D>(next, raw[u] & kSidMask);
      }
  }
}

// End of a launch that uses the phase: the last CUDA block to get here
// advances it (every block has read it by then).  Called by every thread.
__device__ __forceinline__ void advance_phase(const FluxArgs& a, int q) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1) {
      *a.phase = acc_slot(q + 1);
      *a.done = 0;
    }
  }
}

}  // namespace dev
}  // namespace ep
