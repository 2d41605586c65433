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

// a record of R floats is R/V chunks of a V-wide vector
template <int R>
struct Rec {
  static constexpr int V = R >= 4 ? 4 : R;
  static constexpr int NC = R / V;
  using T = typename VecOf<V>::T;
};

__device__ __forceinline__ float lane(const float& v, int) { return v; }
__device__ __forceinline__ float lane(const float2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ float lane(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ float axpy(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ float2 axpy(float a, float2 x, float2 y) {
  return make_float2(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y));
}
__device__ __forceinline__ float4 axpy(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
template <typename T>
__device__ __forceinline__ T zero_of();
template <>
__device__ __forceinline__ float zero_of<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ float4 zero_of<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Global accumulation of lanes [c*V, c*V+V) of a record, only lanes < D.
template <int D, int V>
__device__ __forceinline__ void red_chunk(float* dst, int c, const typename VecOf<V>::T& a) {
  if (c * V + V <= D) {
    if constexpr (V == 4)
      atomicAdd(reinterpret_cast<float4*>(dst), a);
    else if constexpr (V == 2)
      atomicAdd(reinterpret_cast<float2*>(dst), a);
    else
      atomicAdd(dst, lane(a, 0));
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (c * V + l < D) atomicAdd(dst + l, lane(a, l));
  }
}

// record id of local slot `slot` in a flux block
__device__ __forceinline__ int32_t flux_rec(const FluxDesc& d, const int32_t* __restrict__ flist,
                                            int slot) {
  const int own = d.n_int + d.n_ob;
  return slot < d.n_int ? d.int_lo + slot
         : slot < own   ? d.bnd_lo + (slot - d.n_int)
                        : __ldg(flist + d.f0 + (slot - own));
}

// ------------------------------------------------------------- flux forward

template <int D, int R>
__global__ void flux_fwd_kernel(const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
                                const uint32_t* __restrict__ loc, const float* __restrict__ w,
                                const float* __restrict__ x_in, float* __restrict__ x_out,
                                float* __restrict__ bacc, float* __restrict__ out, int32_t n_int,
                                float tau) {
  using RT = Rec<R>;
  using T = typename RT::T;
  extern __shared__ float4 smem4[];
  const FluxDesc d = desc[blockIdx.x];
  const int nv = d.n_int + d.n_ob + d.nf;
  float* xs = reinterpret_cast<float*>(smem4);
  float* acc = xs + (size_t)nv * R;
  for (int i = threadIdx.x; i < nv * RT::NC; i += blockDim.x) {
    const int slot = i / RT::NC, c = i % RT::NC;
    const int32_t r = flux_rec(d, flist, slot);
    reinterpret_cast<T*>(xs + slot * R)[c] =
        __ldg(reinterpret_cast<const T*>(x_in + (size_t)r * R) + c);
    reinterpret_cast<T*>(acc + slot * R)[c] = zero_of<T>();
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d.ne; j += blockDim.x) {
    const uint32_t p = __ldg(loc + d.e0 + j);
    const int u = (int)(p & 0xffffu), v = (int)(p >> 16);
    const float we = __ldg(w + d.e0 + j);
    float dd[D];
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      dd[c] = xs[v * R + c] - xs[u * R + c];
      s = fmaf(dd[c], dd[c], s);
    }
    const float coef = we / (1.f + s);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float f = coef * dd[c];
      atomicAdd(acc + u * R + c, f);
      atomicAdd(acc + v * R + c, -f);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv * RT::NC; i += blockDim.x) {
    const int slot = i / RT::NC, c = i % RT::NC;
    const T a = reinterpret_cast<const T*>(acc + slot * R)[c];
    if (slot < d.n_int) {
      const int32_t r = d.int_lo + slot;
      const T xv = reinterpret_cast<const T*>(xs + slot * R)[c];
      reinterpret_cast<T*>(x_out + (size_t)r * R)[c] = axpy(tau, a, xv);
      if (out) reinterpret_cast<T*>(out + (size_t)r * R)[c] = a;
    } else {
      const int32_t r = flux_rec(d, flist, slot);
      red_chunk<D, RT::V>(bacc + (size_t)(r - n_int) * R + c * RT::V, c, a);
    }
  }
}

// shared records: x_out = x_in + tau * acc; out = acc; acc = 0
template <int R>
__global__ void bnd_update_kernel(const float* __restrict__ x_in, float* __restrict__ x_out,
                                  float* __restrict__ bacc, float* __restrict__ out, int64_t n_int,
                                  int64_t n_bnd, float tau) {
  using RT = Rec<R>;
  using T = typename RT::T;
  const int64_t total = n_bnd * RT::NC;
  const T* xi = reinterpret_cast<const T*>(x_in + (size_t)n_int * R);
  T* xo = reinterpret_cast<T*>(x_out + (size_t)n_int * R);
  T* ba = reinterpret_cast<T*>(bacc);
  T* oo = out ? reinterpret_cast<T*>(out + (size_t)n_int * R) : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T a = ba[i];
    xo[i] = axpy(tau, a, xi[i]);
    if (oo) oo[i] = a;
    ba[i] = zero_of<T>();
  }
}

// ------------------------------------------------------------- flux adjoint

template <int D, int R>
__global__ void flux_adj_kernel(const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
                                const uint32_t* __restrict__ loc, const float* __restrict__ w,
                                const float* __restrict__ x, float* __restrict__ lam,
                                float* __restrict__ gw, float* __restrict__ bacc, int32_t n_int,
                                float tau) {
  using RT = Rec<R>;
  using T = typename RT::T;
  extern __shared__ float4 smem4[];
  const FluxDesc d = desc[blockIdx.x];
  const int nv = d.n_int + d.n_ob + d.nf;
  float* xs = reinterpret_cast<float*>(smem4);
  float* ls = xs + (size_t)nv * R;
  float* acc = ls + (size_t)nv * R;
  for (int i = threadIdx.x; i < nv * RT::NC; i += blockDim.x) {
    const int slot = i / RT::NC, c = i % RT::NC;
    const int32_t r = flux_rec(d, flist, slot);
    reinterpret_cast<T*>(xs + slot * R)[c] = __ldg(reinterpret_cast<const T*>(x + (size_t)r * R) + c);
    reinterpret_cast<T*>(ls + slot * R)[c] = reinterpret_cast<const T*>(lam + (size_t)r * R)[c];
    reinterpret_cast<T*>(acc + slot * R)[c] = zero_of<T>();
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d.ne; j += blockDim.x) {
    const uint32_t p = __ldg(loc + d.e0 + j);
    const int u = (int)(p & 0xffffu), v = (int)(p >> 16);
    const float we = __ldg(w + d.e0 + j);
    float dd[D], gb[D];
    float s = 0.f, dg = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      dd[c] = xs[v * R + c] - xs[u * R + c];
      gb[c] = ls[u * R + c] - ls[v * R + c];
      s = fmaf(dd[c], dd[c], s);
      dg = fmaf(dd[c], gb[c], dg);
    }
    const float inv = 1.f / (1.f + s);
    gw[d.e0 + j] += tau * dg * inv;
    const float two = 2.f * dg * inv * inv;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float h = we * (gb[c] * inv - two * dd[c]);
      atomicAdd(acc + v * R + c, h);
      atomicAdd(acc + u * R + c, -h);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv * RT::NC; i += blockDim.x) {
    const int slot = i / RT::NC, c = i % RT::NC;
    const T a = reinterpret_cast<const T*>(acc + slot * R)[c];
    if (slot < d.n_int) {
      const int32_t r = d.int_lo + slot;
      const T lv = reinterpret_cast<const T*>(ls + slot * R)[c];
      reinterpret_cast<T*>(lam + (size_t)r * R)[c] = axpy(tau, a, lv);
    } else {
      const int32_t r = flux_rec(d, flist, slot);
      red_chunk<D, RT::V>(bacc + (size_t)(r - n_int) * R + c * RT::V, c, a);
    }
  }
}

// --------------------------------------------------------------------- SpMV

__global__ void spmv_kernel(const SpmvDesc* __restrict__ desc, const int32_t* __restrict__ xlist,
                            const int32_t* __restrict__ ylist, const uint32_t* __restrict__ loc,
                            const float* __restrict__ w, const float* __restrict__ x,
                            float* __restrict__ y) {
  extern __shared__ float4 smem4[];
  const SpmvDesc d = desc[blockIdx.x];
  const int nx = d.n_xo + d.n_xf, ny = d.n_yi + d.n_yob + d.n_yf;
  float* xs = reinterpret_cast<float*>(smem4);
  float* ys = xs + nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x)
    xs[i] = __ldg(x + (i < d.n_xo ? d.x_lo + i : __ldg(xlist + d.fx0 + (i - d.n_xo))));
  for (int i = threadIdx.x; i < ny; i += blockDim.x) ys[i] = 0.f;
  __syncthreads();
  for (int j = threadIdx.x; j < d.ne; j += blockDim.x) {
    const uint32_t p = __ldg(loc + d.e0 + j);
    atomicAdd(ys + (p & 0xffffu), __ldg(w + d.e0 + j) * xs[p >> 16]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ny; i += blockDim.x) {
    if (i < d.n_yi) {
      y[d.yi_lo + i] = ys[i];
    } else {
      const int own = d.n_yi + d.n_yob;
      const int32_t r = i < own ? d.yb_lo + (i - d.n_yi) : __ldg(ylist + d.fy0 + (i - own));
      atomicAdd(y + r, ys[i]);
    }
  }
}

// ------------------------------------------------------------------- layout

template <int R>
__global__ void layout_in_kernel(const int32_t* __restrict__ rec_of, int64_t n, int D,
                                 const float* __restrict__ x, float* __restrict__ x_lay) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    float t[R];
#pragma unroll
    for (int c = 0; c < R; ++c) t[c] = c < D ? x[(size_t)c * n + v] : 0.f;
    using RT = Rec<R>;
    using T = typename RT::T;
    T* dst = reinterpret_cast<T*>(x_lay + (size_t)rec_of[v] * R);
#pragma unroll
    for (int c = 0; c < RT::NC; ++c) dst[c] = reinterpret_cast<const T*>(t)[c];
  }
}

template <int R>
__global__ void layout_out_kernel(const int32_t* __restrict__ rec_of, int64_t n, int D,
                                  const float* __restrict__ x_lay, float* __restrict__ x) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    using RT = Rec<R>;
    using T = typename RT::T;
    float t[R];
    const T* src = reinterpret_cast<const T*>(x_lay + (size_t)rec_of[v] * R);
#pragma unroll
    for (int c = 0; c < RT::NC; ++c) reinterpret_cast<T*>(t)[c] = src[c];
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (c < D) x[(size_t)c * n + v] = t[c];
  }
}

__global__ void gather_kernel(const int32_t* __restrict__ perm, int64_t m, const float* __restrict__ w,
                              float* __restrict__ w_lay) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    w_lay[i] = __ldg(w + perm[i]);
}

__global__ void scatter_add_kernel(const int32_t* __restrict__ perm, int64_t m,
                                   const float* __restrict__ w_lay, float* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    w[perm[i]] += w_lay[i];
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

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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

template <int D, int R>
cudaError_t flux_step_t(const FluxArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)a.max_nv * R * sizeof(float) * 2;
  cudaError_t e = allow_smem(flux_fwd_kernel<D, R>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_FWD, st);
    flux_fwd_kernel<D, R><<<(unsigned)a.k, a.tpb, smem, st>>>(
        a.desc, a.flist, a.loc, a.w, a.x_in, a.x_out, a.bacc, a.out, (int32_t)a.n_int, a.tau);
  }
  if (a.n_bnd > 0) {
    Scope sc(a.timer, T_BND, st);
    bnd_update_kernel<R><<<grid_for(a.n_bnd * Rec<R>::NC, 256), 256, 0, st>>>(
        a.x_in, a.x_out, a.bacc, a.out, a.n_int, a.n_bnd, a.tau);
  }
  return cudaGetLastError();
}

template <int D, int R>
cudaError_t flux_adj_t(const FluxArgs& a, float* lam, float* gw, cudaStream_t st) {
  const size_t smem = (size_t)a.max_nv * R * sizeof(float) * 3;
  cudaError_t e = allow_smem(flux_adj_kernel<D, R>, smem);
  if (e != cudaSuccess) return e;
  if (a.k > 0) {
    Scope sc(a.timer, T_EDGE_ADJ, st);
    flux_adj_kernel<D, R><<<(unsigned)a.k, a.tpb, smem, st>>>(a.desc, a.flist, a.loc, a.w, a.x_in,
                                                             lam, gw, a.bacc, (int32_t)a.n_int, a.tau);
  }
  if (a.n_bnd > 0) {
    Scope sc(a.timer, T_BND, st);
    bnd_update_kernel<R><<<grid_for(a.n_bnd * Rec<R>::NC, 256), 256, 0, st>>>(
        lam, lam, a.bacc, nullptr, a.n_int, a.n_bnd, a.tau);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t flux_step(const FluxArgs& a, int D, cudaStream_t st) {
  switch (D) {
    case 1: return flux_step_t<1, 1>(a, st);
    case 2: return flux_step_t<2, 2>(a, st);
    case 3: return flux_step_t<3, 4>(a, st);
    case 4: return flux_step_t<4, 4>(a, st);
    case 5: return flux_step_t<5, 8>(a, st);
    case 6: return flux_step_t<6, 8>(a, st);
    case 7: return flux_step_t<7, 8>(a, st);
    case 8: return flux_step_t<8, 8>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t flux_adjoint_step(const FluxArgs& a, int D, float* lam, float* gw, cudaStream_t st) {
  switch (D) {
    case 1: return flux_adj_t<1, 1>(a, lam, gw, st);
    case 2: return flux_adj_t<2, 2>(a, lam, gw, st);
    case 3: return flux_adj_t<3, 4>(a, lam, gw, st);
    case 4: return flux_adj_t<4, 4>(a, lam, gw, st);
    case 5: return flux_adj_t<5, 8>(a, lam, gw, st);
    case 6: return flux_adj_t<6, 8>(a, lam, gw, st);
    case 7: return flux_adj_t<7, 8>(a, lam, gw, st);
    case 8: return flux_adj_t<8, 8>(a, lam, gw, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t spmv(const SpmvArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.max_nx + a.max_ny) * sizeof(float);
  cudaError_t e = allow_smem(spmv_kernel, smem);
  if (e != cudaSuccess) return e;
  if (a.ny_zero > 0) {
    e = cudaMemsetAsync(a.y + a.ny_int, 0, (size_t)a.ny_zero * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  if (a.k > 0) {
    Scope sc(a.timer, T_SPMV, st);
    spmv_kernel<<<(unsigned)a.k, a.tpb, smem, st>>>(a.desc, a.xlist, a.ylist, a.loc, a.w, a.x, a.y);
  }
  return cudaGetLastError();
}

cudaError_t layout_in(const int32_t* rec_of, int64_t n, int D, int R, const float* x, float* x_lay,
                      cudaStream_t st, Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  const int g = grid_for(n, 256);
  switch (R) {
    case 1: layout_in_kernel<1><<<g, 256, 0, st>>>(rec_of, n, D, x, x_lay); break;
    case 2: layout_in_kernel<2><<<g, 256, 0, st>>>(rec_of, n, D, x, x_lay); break;
    case 4: layout_in_kernel<4><<<g, 256, 0, st>>>(rec_of, n, D, x, x_lay); break;
    case 8: layout_in_kernel<8><<<g, 256, 0, st>>>(rec_of, n, D, x, x_lay); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t layout_out(const int32_t* rec_of, int64_t n, int D, int R, const float* x_lay, float* x,
                       cudaStream_t st, Timer* t) {
  Scope sc(t, T_LAYOUT, st);
  const int g = grid_for(n, 256);
  switch (R) {
    case 1: layout_out_kernel<1><<<g, 256, 0, st>>>(rec_of, n, D, x_lay, x); break;
    case 2: layout_out_kernel<2><<<g, 256, 0, st>>>(rec_of, n, D, x_lay, x); break;
    case 4: layout_out_kernel<4><<<g, 256, 0, st>>>(rec_of, n, D, x_lay, x); break;
    case 8: layout_out_kernel<8><<<g, 256, 0, st>>>(rec_of, n, D, x_lay, x); break;
    default: return cudaErrorInvalidValue;
  }
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
