// kernels.cu -- device code of libepcache (sm_103a).
//
// The software-cache kernel of Section 4 (Fig. 7(d)), restated for GB300:
// every CUDA block takes one schedule block, copies the distinct vertices of
// that block (the vertex set the cost model of Eq. 1 counts once per block)
// from HBM into shared memory, runs its tasks out of shared memory, and
// writes back once per vertex: vertices no other block uses are updated in
// place with plain stores, shared vertices get one vector atomic add into an
// accumulator that a second, streaming kernel folds into the state.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>
#include <unordered_set>

#include "kernels.h"

namespace ep {
namespace dev {
namespace {

template <int V>
struct VecOf;
template <>
struct VecOf<1> {
  using T = float;
};
template <>
struct VecOf<2> {
  using T = float2;
};
template <>
struct VecOf<4> {
  using T = float4;
};

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

template <int W>
__device__ __forceinline__ void vload(const float* p, float* v) {
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
__device__ __forceinline__ void vload_g(const float* __restrict__ p, float* v) {
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
__device__ __forceinline__ void vstore(float* p, const float* v) {
  if constexpr (W == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if constexpr (W == 2)
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  else
    *p = v[0];
}
template <int W>
__device__ __forceinline__ void vred(float* p, const float* v) {
  if constexpr (W == 4)
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  else if constexpr (W == 2)
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
  else
    atomicAdd(p, v[0]);
}

// Record r of a planar buffer of n records <-> registers v[0..D), one vector
// access per plane (planes unrolled at compile time).
template <int D, bool GLOBAL, int K = 0>
__device__ __forceinline__ void rec_load(const float* base, int64_t n, int64_t r, float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    const float* q = base + F * n + r * W;
    if constexpr (GLOBAL)
      vload_g<W>(q, v + F);
    else
      vload<W>(q, v + F);
    rec_load<D, GLOBAL, K + 1>(base, n, r, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void rec_store(float* base, int64_t n, int64_t r, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vstore<W>(base + F * n + r * W, v + F);
    rec_store<D, K + 1>(base, n, r, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void rec_red(float* base, int64_t n, int64_t r, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    vred<W>(base + F * n + r * W, v + F);
    rec_red<D, K + 1>(base, n, r, v);
  }
}

// record at shared position p of a flux block, -1 for an unused position
__device__ __forceinline__ int32_t flux_rec(const FluxDesc& d, const int32_t* __restrict__ flist,
                                            int p) {
  if (p >= d.pi && p < d.pi + d.n_int) return d.int_lo + (p - d.pi);
  if (p >= d.pb && p < d.pb + d.n_ob) return d.bnd_lo + (p - d.pb);
  if (p >= d.pf && p < d.pf + d.nf) return __ldg(flist + d.f0 + (p - d.pf));
  return -1;
}

// Shared-memory carve-up of a flux block: planes of npos positions each
// (npos a multiple of 4 keeps every plane 16-byte aligned), then weights,
// incidence entries and position offsets.
struct FluxSmem {
  float* x;
  float* lam;
  float* w;
  uint32_t* ent;
  uint16_t* ptr;
  int npos;
};
template <int D>
__device__ __forceinline__ FluxSmem flux_smem(const FluxDesc& d, bool with_lam) {
  extern __shared__ float4 smem4[];
  FluxSmem s;
  s.npos = (d.np + 3) & ~3;
  s.x = reinterpret_cast<float*>(smem4);
  s.lam = s.x + D * s.npos;
  s.w = with_lam ? s.lam + D * s.npos : s.lam;
  s.ent = reinterpret_cast<uint32_t*>(s.w + ((d.ne + 3) & ~3));  // 16-byte aligned pieces
  s.ptr = reinterpret_cast<uint16_t*>(s.ent + ((d.nent + 3) & ~3));
  return s;
}

template <int D>
__device__ __forceinline__ void stage_block(const FluxDesc& d, const FluxSmem& s,
                                            const int32_t* __restrict__ flist,
                                            const uint32_t* __restrict__ inc,
                                            const uint16_t* __restrict__ ptr,
                                            const float* __restrict__ w, const float* x, int64_t n_rec,
                                            const float* lam) {
  // independent loads first, so no warp waits on a foreign id before issuing
  // them; the per-block pieces are 16-byte aligned and padded, so they move
  // as 16-byte vectors
  const int nw = (d.ne + 3) >> 2, ne4 = (d.nent + 3) >> 2, np8 = (d.np + 1 + 7) >> 3;
  for (int i = threadIdx.x; i < nw; i += blockDim.x)
    reinterpret_cast<float4*>(s.w)[i] = __ldg(reinterpret_cast<const float4*>(w + d.w0) + i);
  for (int i = threadIdx.x; i < ne4; i += blockDim.x)
    reinterpret_cast<uint4*>(s.ent)[i] = __ldg(reinterpret_cast<const uint4*>(inc + d.i0) + i);
  for (int i = threadIdx.x; i < np8; i += blockDim.x)
    reinterpret_cast<uint4*>(s.ptr)[i] = __ldg(reinterpret_cast<const uint4*>(ptr + d.q0) + i);
  for (int p = threadIdx.x; p < d.np; p += blockDim.x) {
    const int32_t r = flux_rec(d, flist, p);
    if (r < 0) continue;
    float v[D];
    rec_load<D, true>(x, n_rec, r, v);
    rec_store<D>(s.x, s.npos, p, v);
    if (lam) {
      rec_load<D, false>(lam, n_rec, r, v);
      rec_store<D>(s.lam, s.npos, p, v);
    }
  }
}

// ------------------------------------------------------------- flux forward

// One CUDA block per schedule block.  After staging, the thread of position p
// sums the flux of every task at p over p's incidence list, reading the other
// endpoint from shared memory: d = x_o - x_p, f = w d / (1 + |d|^2).  The
// difference is exactly antisymmetric in IEEE arithmetic, so both endpoints of
// a task see +f and -f of the same value.
template <int D>
__global__ void __launch_bounds__(1024) flux_fwd_kernel(
    const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
    const uint32_t* __restrict__ inc, const uint16_t* __restrict__ ptr, const float* __restrict__ w,
    const float* x_in, float* x_out, float* __restrict__ bacc, float* __restrict__ out,
    int64_t n_rec, int64_t n_int, int64_t n_bnd, float tau) {
  const FluxDesc d = desc[blockIdx.x];
  const FluxSmem s = flux_smem<D>(d, false);
  stage_block<D>(d, s, flist, inc, ptr, w, x_in, n_rec, nullptr);
  __syncthreads();
  for (int p = threadIdx.x; p < d.np; p += blockDim.x) {
    const int k0 = s.ptr[p], k1 = s.ptr[p + 1];
    if (k0 == k1) continue;  // unused position
    float xp[D], acc[D];
    rec_load<D, false>(s.x, s.npos, p, xp);
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.f;
    for (int k = k0; k < k1; ++k) {
      const uint32_t e = s.ent[k];
      float xo[D];
      rec_load<D, false>(s.x, s.npos, (int)(e & kPosMask), xo);
      float dd[D], q = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dd[c] = xo[c] - xp[c];
        q = fmaf(dd[c], dd[c], q);
      }
      const float coef = __fdividef(s.w[(e >> kTaskShift) & 0xffffu], 1.f + q);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = fmaf(coef, dd[c], acc[c]);
    }
    const int32_t r = flux_rec(d, flist, p);
    if (p < d.pi + d.n_int) {
      float xn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) xn[c] = fmaf(tau, acc[c], xp[c]);
      rec_store<D>(x_out, n_rec, r, xn);
      if (out) rec_store<D>(out, n_rec, r, acc);
    } else {
      rec_red<D>(bacc, n_bnd, r - n_int, acc);
    }
  }
}

// Read-only-cache variant: the texture-cache kernel of Section 5 (Fig. 7(c)),
// with the read-only data cache (ld.global.nc) in place of texture binding.
// No staging: every read of a block's incidence, weights and states goes to
// global memory through that cache.  Thread t handles positions t, t + T,
// ..., t + (R-1) T of its block and keeps their sums in registers; writes
// wait for a block barrier, because interior records are updated in place
// and other threads of the same block may still be reading them.  Foreign
// and boundary records are never written by this kernel.
template <int D, int R>
__global__ void __launch_bounds__(1024) flux_fwd_ldg_kernel(
    const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
    const uint32_t* __restrict__ inc, const uint16_t* __restrict__ ptr, const float* __restrict__ w,
    const float* x_in, float* x_out, float* __restrict__ bacc, float* __restrict__ out,
    int64_t n_rec, int64_t n_int, int64_t n_bnd, float tau) {
  const FluxDesc d = desc[blockIdx.x];
  float xp[R][D], acc[R][D];
  int32_t rec[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = (int)threadIdx.x + i * (int)blockDim.x;
    rec[i] = -1;
#pragma unroll
    for (int c = 0; c < D; ++c) acc[i][c] = 0.f;
    if (p >= d.np) continue;
    const int k0 = __ldg(ptr + d.q0 + p), k1 = __ldg(ptr + d.q0 + p + 1);
    if (k0 == k1) continue;  // unused position
    rec[i] = flux_rec(d, flist, p);
    rec_load<D, true>(x_in, n_rec, rec[i], xp[i]);
    for (int k = k0; k < k1; ++k) {
      const uint32_t e = __ldg(inc + d.i0 + k);
      float xo[D];
      rec_load<D, true>(x_in, n_rec, flux_rec(d, flist, (int)(e & kPosMask)), xo);
      float dd[D], q = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dd[c] = xo[c] - xp[i][c];
        q = fmaf(dd[c], dd[c], q);
      }
      const float coef = __fdividef(__ldg(w + d.w0 + ((e >> kTaskShift) & 0xffffu)), 1.f + q);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[i][c] = fmaf(coef, dd[c], acc[i][c]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = (int)threadIdx.x + i * (int)blockDim.x;
    if (rec[i] < 0) continue;
    if (p < d.pi + d.n_int) {
      float xn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) xn[c] = fmaf(tau, acc[i][c], xp[i][c]);
      rec_store<D>(x_out, n_rec, rec[i], xn);
      if (out) rec_store<D>(out, n_rec, rec[i], acc[i]);
    } else {
      rec_red<D>(bacc, n_bnd, rec[i] - n_int, acc[i]);
    }
  }
}

// shared records: x_out = x_in + tau * acc; out = acc; acc = 0 (plane by plane)
template <int D>
__global__ void bnd_update_kernel(const float* x_in, float* x_out, float* __restrict__ bacc,
                                  float* __restrict__ out, int64_t n_rec, int64_t n_int,
                                  int64_t n_bnd, float tau) {
  // launched with programmatic serialisation after the edge kernel: wait for
  // it (the accumulators and interior records it wrote) before reading
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bnd;
       i += (int64_t)gridDim.x * blockDim.x) {
    float a[D], x[D];
    rec_load<D, false>(bacc, n_bnd, i, a);
    rec_load<D, false>(x_in, n_rec, n_int + i, x);
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = fmaf(tau, a[c], x[c]);
    rec_store<D>(x_out, n_rec, n_int + i, x);
    if (out) rec_store<D>(out, n_rec, n_int + i, a);
#pragma unroll
    for (int c = 0; c < D; ++c) a[c] = 0.f;
    rec_store<D>(bacc, n_bnd, i, a);
  }
}

// ------------------------------------------------------------- flux adjoint

// Reverse step: at position p with other endpoint o of a task,
// d = x_o - x_p, g = lam_p - lam_o, q = |d|^2,
// contribution to lam_p: -w (g/(1+q) - 2 d (d.g)/(1+q)^2), and the src-side
// entry adds tau (d.g)/(1+q) to the task's weight gradient.
template <int D>
__global__ void __launch_bounds__(1024) flux_adj_kernel(
    const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
    const uint32_t* __restrict__ inc, const uint16_t* __restrict__ ptr, const float* __restrict__ w,
    const float* __restrict__ x, float* lam, float* __restrict__ gw, float* __restrict__ bacc,
    int64_t n_rec, int64_t n_int, int64_t n_bnd, float tau) {
  const FluxDesc d = desc[blockIdx.x];
  const FluxSmem s = flux_smem<D>(d, true);
  stage_block<D>(d, s, flist, inc, ptr, w, x, n_rec, lam);
  __syncthreads();
  for (int p = threadIdx.x; p < d.np; p += blockDim.x) {
    const int k0 = s.ptr[p], k1 = s.ptr[p + 1];
    if (k0 == k1) continue;
    float xp[D], lp[D], acc[D];
    rec_load<D, false>(s.x, s.npos, p, xp);
    rec_load<D, false>(s.lam, s.npos, p, lp);
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.f;
    for (int k = k0; k < k1; ++k) {
      const uint32_t e = s.ent[k];
      const int o = (int)(e & kPosMask);
      const int t = (int)((e >> kTaskShift) & 0xffffu);
      float xo[D], lo[D];
      rec_load<D, false>(s.x, s.npos, o, xo);
      rec_load<D, false>(s.lam, s.npos, o, lo);
      float dd[D], g[D], q = 0.f, dg = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dd[c] = xo[c] - xp[c];
        g[c] = lp[c] - lo[c];
        q = fmaf(dd[c], dd[c], q);
        dg = fmaf(dd[c], g[c], dg);
      }
      const float inv = __fdividef(1.f, 1.f + q);
      const float we = s.w[t];
      const float two = 2.f * dg * inv * inv;
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] -= we * (g[c] * inv - two * dd[c]);
      // one writer per task: a fire-and-forget reduction instead of a load in the loop
      if (e & kSrcBit) atomicAdd(gw + d.w0 + t, tau * dg * inv);
    }
    const int32_t r = flux_rec(d, flist, p);
    if (p < d.pi + d.n_int) {
#pragma unroll
      for (int c = 0; c < D; ++c) lp[c] = fmaf(tau, acc[c], lp[c]);
      rec_store<D>(lam, n_rec, r, lp);
    } else {
      rec_red<D>(bacc, n_bnd, r - n_int, acc);
    }
  }
}

// --------------------------------------------------------------------- SpMV

// One CUDA block per schedule block, pull form: x of the block's columns is
// staged in shared memory; every row position sums w * x over its list.
// Rows with more than 32 entries (hubs of a power-law matrix) take a whole
// warp each; the others one thread each.
__device__ __forceinline__ void spmv_write(const SpmvDesc& d, const int32_t* __restrict__ ylist,
                                           float* __restrict__ y, int p, float acc) {
  if (p < d.n_yi) {
    y[d.yi_lo + p] = acc;
  } else {
    const int own = d.n_yi + d.n_yob;
    const int32_t r = p < own ? d.yb_lo + (p - d.n_yi) : __ldg(ylist + d.fy0 + (p - own));
    atomicAdd(y + r, acc);
  }
}

__global__ void __launch_bounds__(1024) spmv_kernel(
    const SpmvDesc* __restrict__ desc, const int32_t* __restrict__ xlist,
    const int32_t* __restrict__ ylist, const uint32_t* __restrict__ inc,
    const uint16_t* __restrict__ ptr, const float* __restrict__ w, const float* __restrict__ x,
    float* __restrict__ y) {
  extern __shared__ float4 smem4[];
  const SpmvDesc d = desc[blockIdx.x];
  const int nx = d.n_xo + d.n_xf, ny = d.n_yi + d.n_yob + d.n_yf;
  float* xs = reinterpret_cast<float*>(smem4);
  float* ws = xs + ((nx + 3) & ~3);
  uint32_t* es = reinterpret_cast<uint32_t*>(ws + ((d.ne + 3) & ~3));
  uint16_t* ps = reinterpret_cast<uint16_t*>(es + d.ne);
  // weights, entries and row offsets: four loads in flight per thread
  for (int i0 = threadIdx.x; i0 < d.ne; i0 += 4 * blockDim.x) {
    float wv[4];
    uint32_t ev[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      wv[u] = i < d.ne ? __ldg(w + d.w0 + i) : 0.f;
      ev[u] = i < d.ne ? __ldg(inc + d.i0 + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i < d.ne) {
        ws[i] = wv[u];
        es[i] = ev[u];
      }
    }
  }
  for (int i0 = threadIdx.x; i0 <= ny; i0 += 4 * blockDim.x) {
    uint16_t pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      pv[u] = i <= ny ? __ldg(ptr + d.q0 + i) : (uint16_t)0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i <= ny) ps[i] = pv[u];
    }
  }
  // x entries: four (id, value) load chains in flight per thread
  for (int i0 = threadIdx.x; i0 < nx; i0 += 4 * blockDim.x) {
    int32_t r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      r[u] = i >= nx ? -1 : (i < d.n_xo ? d.x_lo + i : __ldg(xlist + d.fx0 + (i - d.n_xo)));
    }
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = r[u] >= 0 ? __ldg(x + r[u]) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r[u] >= 0) xs[i0 + u * (int)blockDim.x] = v[u];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = warp; p < ny; p += nw) {
    const int k0 = ps[p], k1 = ps[p + 1];
    if (k1 - k0 <= 32) continue;  // warp-uniform
    float acc = 0.f;
    for (int q = k0 + lane; q < k1; q += 32) {
      const uint32_t e = es[q];
      acc = fmaf(ws[e >> kTaskShift], xs[e & kPosMask], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) spmv_write(d, ylist, y, p, acc);
  }
  for (int p = threadIdx.x; p < ny; p += blockDim.x) {
    const int k0 = ps[p], k1 = ps[p + 1];
    if (k1 - k0 > 32 || k1 == k0) continue;
    float acc = 0.f;
    for (int q = k0; q < k1; ++q) {
      const uint32_t e = es[q];
      acc = fmaf(ws[e >> kTaskShift], xs[e & kPosMask], acc);
    }
    spmv_write(d, ylist, y, p, acc);
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

// --------------------------------------------------------------------- cost

// One CUDA block per schedule block: bitonic sort of the block's endpoint ids
// in shared memory, then count distinct ids and mark them touched.
__global__ void cost_block_kernel(const int64_t* __restrict__ block_ptr, const int32_t* __restrict__ eu,
                                  const int32_t* __restrict__ ev, int P, uint8_t* __restrict__ touched,
                                  unsigned long long* __restrict__ loads) {
  extern __shared__ float4 smem4[];
  int32_t* key = reinterpret_cast<int32_t*>(smem4);
  __shared__ unsigned int warp_sum[32];
  const int64_t e0 = block_ptr[blockIdx.x];
  const int ne = (int)(block_ptr[blockIdx.x + 1] - e0);
  const int nk = 2 * ne;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    key[i] = i < ne ? eu[e0 + i] : i < nk ? ev[e0 + i - ne] : INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = key[i], b = key[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  unsigned int cnt = 0;
  for (int i = threadIdx.x; i < nk; i += blockDim.x)
    if (i == 0 || key[i] != key[i - 1]) {
      ++cnt;
      touched[key[i]] = 1;
    }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned int v = threadIdx.x < (blockDim.x >> 5) ? warp_sum[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loads, (unsigned long long)v);
  }
}

__global__ void count_flags_kernel(const uint8_t* __restrict__ f, int64_t nd,
                                   unsigned long long* __restrict__ total) {
  unsigned int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    cnt += f[i];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(total, (unsigned long long)cnt);
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

size_t flux_smem_bytes(const FluxArgs& a, int D, int copies) {
  const size_t npos = ((size_t)a.max_np + 3) & ~(size_t)3;
  const auto up = [](size_t v, size_t m) { return (v + m - 1) / m * m; };
  return (size_t)copies * D * npos * sizeof(float) + up(a.max_ne, 4) * sizeof(float) +
         up(a.max_nent, 4) * sizeof(uint32_t) + up((size_t)a.max_np + 1, 8) * sizeof(uint16_t) + 16;
}

template <int D>
cudaError_t flux_step_t(const FluxArgs& a, cudaStream_t st) {
  const size_t smem = flux_smem_bytes(a, D, 1);
  cudaError_t e = allow_smem(flux_fwd_kernel<D>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_FWD, st);
    flux_fwd_kernel<D><<<(unsigned)a.k, a.tpb, smem, st>>>(a.desc, a.flist, a.inc, a.ptr, a.w, a.x_in,
                                                          a.x_out, a.bacc, a.out, a.n_rec, a.n_int,
                                                          a.n_bnd, a.tau);
  }
  if (a.n_bnd > 0) {
    Scope sc(a.timer, T_BND, st);
    bnd_update_kernel<D><<<grid_for(a.n_bnd, 256), 256, 0, st>>>(a.x_in, a.x_out, a.bacc, a.out,
                                                                 a.n_rec, a.n_int, a.n_bnd, a.tau);
  }
  return cudaGetLastError();
}

template <int D, int R>
void flux_ldg_launch(const FluxArgs& a, int threads, cudaStream_t st) {
  flux_fwd_ldg_kernel<D, R><<<(unsigned)a.k, threads, 0, st>>>(a.desc, a.flist, a.inc, a.ptr, a.w,
                                                              a.x_in, a.x_out, a.bacc, a.out,
                                                              a.n_rec, a.n_int, a.n_bnd, a.tau);
}

template <int D>
cudaError_t flux_step_ldg_t(const FluxArgs& a, cudaStream_t st) {
  const int R = (a.max_np + 1023) / 1024;  // positions per thread
  const int threads = std::max(32, (((a.max_np + R - 1) / R) + 31) / 32 * 32);
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
  }
  if (a.n_bnd > 0) {
    Scope sc(a.timer, T_BND, st);
    bnd_update_kernel<D><<<grid_for(a.n_bnd, 256), 256, 0, st>>>(a.x_in, a.x_out, a.bacc, a.out,
                                                                 a.n_rec, a.n_int, a.n_bnd, a.tau);
  }
  return cudaGetLastError();
}

template <int D>
cudaError_t flux_adj_t(const FluxArgs& a, float* lam, float* gw, cudaStream_t st) {
  const size_t smem = flux_smem_bytes(a, D, 2);
  cudaError_t e = allow_smem(flux_adj_kernel<D>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_ADJ, st);
    flux_adj_kernel<D><<<(unsigned)a.k, a.tpb, smem, st>>>(a.desc, a.flist, a.inc, a.ptr, a.w, a.x_in,
                                                          lam, gw, a.bacc, a.n_rec, a.n_int, a.n_bnd,
                                                          a.tau);
  }
  if (a.n_bnd > 0) {
    Scope sc(a.timer, T_BND, st);
    bnd_update_kernel<D><<<grid_for(a.n_bnd, 256), 256, 0, st>>>(lam, lam, a.bacc, nullptr, a.n_rec,
                                                                 a.n_int, a.n_bnd, a.tau);
  }
  return cudaGetLastError();
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

// shared-vertex fold after a pipelined edge kernel: x_out = x_in + tau*bacc
cudaError_t bnd_update(const FluxArgs& a, int D, float* x_out, const float* x_in, float* out,
                       cudaStream_t st) {
  if (a.n_bnd <= 0) return cudaSuccess;
  Scope sc(a.timer, T_BND, st);
  const int g = grid_for(a.n_bnd, 256);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
#define EP_BU(DD)                                                                        \
  e = cudaLaunchKernelEx(&cfg, bnd_update_kernel<DD>, x_in, x_out, a.bacc, out, a.n_rec, \
                         a.n_int, a.n_bnd, a.tau)
  EP_DISPATCH_D(D, EP_BU)
#undef EP_BU
  return e != cudaSuccess ? e : cudaGetLastError();
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

// Read-only-cache SpMV (EP-text of Section 5): the same row-pull form with
// nothing staged; x, the task weights, entries and offsets are read through
// the read-only data cache.  y is written as in spmv_kernel.
__global__ void __launch_bounds__(1024) spmv_ldg_kernel(
    const SpmvDesc* __restrict__ desc, const int32_t* __restrict__ xlist,
    const int32_t* __restrict__ ylist, const uint32_t* __restrict__ inc,
    const uint16_t* __restrict__ ptr, const float* __restrict__ w, const float* __restrict__ x,
    float* __restrict__ y) {
  const SpmvDesc d = desc[blockIdx.x];
  const int ny = d.n_yi + d.n_yob + d.n_yf;
  const uint32_t* es = inc + d.i0;
  const uint16_t* ps = ptr + d.q0;
  const float* ws = w + d.w0;
  auto xval = [&](uint32_t e) {
    const int i = (int)(e & kPosMask);
    return __ldg(x + (i < d.n_xo ? d.x_lo + i : __ldg(xlist + d.fx0 + (i - d.n_xo))));
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = warp; p < ny; p += nw) {
    const int k0 = __ldg(ps + p), k1 = __ldg(ps + p + 1);
    if (k1 - k0 <= 32) continue;  // warp-uniform
    float acc = 0.f;
    for (int q = k0 + lane; q < k1; q += 32) {
      const uint32_t e = __ldg(es + q);
      acc = fmaf(__ldg(ws + (e >> kTaskShift)), xval(e), acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) spmv_write(d, ylist, y, p, acc);
  }
  for (int p = threadIdx.x; p < ny; p += blockDim.x) {
    const int k0 = __ldg(ps + p), k1 = __ldg(ps + p + 1);
    if (k1 - k0 > 32 || k1 == k0) continue;
    float acc = 0.f;
    for (int q = k0; q < k1; ++q) {
      const uint32_t e = __ldg(es + q);
      acc = fmaf(__ldg(ws + (e >> kTaskShift)), xval(e), acc);
    }
    spmv_write(d, ylist, y, p, acc);
  }
}

size_t flux_block_smem(const FluxArgs& a, int D, bool adjoint) {
  return flux_smem_bytes(a, D, adjoint ? 2 : 1);
}

size_t spmv_block_smem(const SpmvArgs& a) {
  return (size_t)(a.max_nx + 4) * sizeof(float) + (size_t)(a.max_ne + 4) * 8 +
         (size_t)(a.max_ny + 1) * sizeof(uint16_t) + 16;
}

cudaError_t spmv(const SpmvArgs& a, cudaStream_t st) {
  const size_t smem = spmv_block_smem(a);
  cudaError_t e = allow_smem(spmv_kernel, smem);
  if (e != cudaSuccess) return e;
  if (a.ny_zero > 0) {
    e = cudaMemsetAsync(a.y + a.ny_int, 0, (size_t)a.ny_zero * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  if (a.k > 0) {
    Scope sc(a.timer, T_SPMV, st);
    if (a.readonly)
      spmv_ldg_kernel<<<(unsigned)a.k, a.tpb, 0, st>>>(a.desc, a.xlist, a.ylist, a.inc, a.ptr, a.w,
                                                       a.x, a.y);
    else
      spmv_kernel<<<(unsigned)a.k, a.tpb, smem, st>>>(a.desc, a.xlist, a.ylist, a.inc, a.ptr, a.w,
                                                      a.x, a.y);
  }
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
