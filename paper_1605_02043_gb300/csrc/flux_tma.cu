// flux_tma.cu -- persistent, pipelined flux kernels (sm_103a).
//
// Same computation as the one-block-per-CUDA-block kernels in kernels.cu
// (the software-cache kernel of Section 4 with the partition of Section 3),
// organised so that loading the next schedule blocks overlaps computing the
// current one.  Each persistent CUDA block owns NS shared-memory stages:
//   producer (one thread)  deals schedule blocks round-robin and copies each
//                  block's contiguous pieces (incidence entries, position
//                  offsets, weights, foreign ids, and the 16-byte aligned part
//                  of its two owned record runs in every state plane) with
//                  1-D TMA bulk copies that complete on the stage's "full"
//                  mbarrier;
//   consumer warps gather block j+1's foreign records and the ragged ends of
//                  its runs with cp.async, then compute every position of
//                  block j from shared memory, write back, and arrive on the
//                  stage's "empty" mbarrier so the producer can refill it.
// Every wait is bounded by a clock budget; on expiry the kernel records an
// error code and returns instead of hanging (consumers decide together, so
// none is left behind in a named barrier).
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace ep {
namespace dev {
namespace {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kErrTimeoutFull = 1;
constexpr int kErrTimeoutEmpty = 2;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}
// true in every consumer thread if `fail` is true in any of them (named barrier 1)
__device__ __forceinline__ bool consumers_any(bool fail, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)fail), "r"(nthreads)
      : "memory");
  return r != 0;
}

// ------------------------------------------------------------ plane helpers

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
__device__ __forceinline__ void ld_sv(const float* p, float* v) {
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
__device__ __forceinline__ void st_gv(float* p, const float* v) {
  if constexpr (W == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if constexpr (W == 2)
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  else
    *p = v[0];
}
template <int W>
__device__ __forceinline__ void red_gv(float* p, const float* v) {
  if constexpr (W == 4)
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  else if constexpr (W == 2)
    atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
  else
    atomicAdd(p, v[0]);
}

// shared record at position p (planes of npos positions) -> registers
template <int D, int K = 0>
__device__ __forceinline__ void srec_load(const float* base, int npos, int p, float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    ld_sv<W>(base + F * npos + p * W, v + F);
    srec_load<D, K + 1>(base, npos, p, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void grec_store(float* base, int64_t n, int64_t r, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    st_gv<W>(base + F * n + r * W, v + F);
    grec_store<D, K + 1>(base, n, r, v);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void grec_red(float* base, int64_t n, int64_t r, const float* v) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    red_gv<W>(base + F * n + r * W, v + F);
    grec_red<D, K + 1>(base, n, r, v);
  }
}
// cp.async of one record (all planes) from global record r to shared position p
template <int D, int K = 0>
__device__ __forceinline__ void rec_cp_async(float* sbase, int npos, int p, const float* gbase,
                                             int64_t n, int64_t r) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    cp_async<W * 4>(sbase + F * npos + p * W, gbase + F * n + r * W);
    rec_cp_async<D, K + 1>(sbase, npos, p, gbase, n, r);
  }
}

// ------------------------------------------------------------ stage layout

struct StageRefs {
  float* x;
  float* lam;
  float* w;
  uint32_t* ent;
  uint16_t* ptr;
  int32_t* flist;
  FluxDesc* desc;
  int32_t* block;
};

__device__ __forceinline__ StageRefs stage_refs(unsigned char* base, const TmaLayout& L, int s) {
  unsigned char* p = base + (size_t)s * L.stage_bytes;
  StageRefs r;
  r.x = reinterpret_cast<float*>(p);
  r.lam = reinterpret_cast<float*>(p + L.off_lam);
  r.w = reinterpret_cast<float*>(p + L.off_w);
  r.ent = reinterpret_cast<uint32_t*>(p + L.off_ent);
  r.ptr = reinterpret_cast<uint16_t*>(p + L.off_ptr);
  r.flist = reinterpret_cast<int32_t*>(p + L.off_flist);
  r.desc = reinterpret_cast<FluxDesc*>(p + L.off_desc);
  r.block = reinterpret_cast<int32_t*>(p + L.off_desc + sizeof(FluxDesc));
  return r;
}

__device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__device__ __forceinline__ int pad8(int x) { return (x + 7) & ~7; }

// Bulk pieces of one owned run [lo, lo + cnt) at shared positions from p0:
// runs start on 4-record boundaries and are followed by unused gap records up
// to the next boundary, so every plane moves as whole 16-byte chunks
// (ceil(cnt / (4 / width)) of them).  `issue` false only sums the bytes.
template <int D, int K = 0>
__device__ __forceinline__ uint32_t run_bulk(const float* gx, int64_t n, int lo, int cnt, int p0,
                                             float* sx, int npos, uint64_t* bar, bool issue) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    constexpr int G = 4 / W;  // records per 16 bytes
    const uint32_t bytes = (uint32_t)((cnt + G - 1) / G) * 16u;
    if (issue && bytes) bulk_load(sx + F * npos + p0 * W, gx + F * n + (int64_t)lo * W, bytes, bar);
    return bytes + run_bulk<D, K + 1>(gx, n, lo, cnt, p0, sx, npos, bar, issue);
  }
  return 0;
}

// Producer (one thread): bulk copies of schedule block b into stage S.
template <int D>
__device__ __forceinline__ void produce(const FluxDesc& d, int b, const int32_t* __restrict__ flist,
                                        const uint32_t* __restrict__ inc,
                                        const uint16_t* __restrict__ ptr, const float* __restrict__ w,
                                        const float* x, const float* lam, int64_t n_rec,
                                        const StageRefs& S, const TmaLayout& L, uint64_t* full) {
  *S.desc = d;
  *S.block = b;
  const uint32_t b_ent = (uint32_t)pad4(d.nent) * 4u;
  const uint32_t b_ptr = (uint32_t)pad8(d.np + 1) * 2u;
  const uint32_t b_w = (uint32_t)pad4(d.ne) * 4u;
  const uint32_t b_f = (uint32_t)pad4(d.nf) * 4u;
  uint32_t bytes = b_ent + b_ptr + b_w + b_f;
  bytes += run_bulk<D>(x, n_rec, d.int_lo, d.n_int, d.pi, S.x, L.npos, full, false);
  bytes += run_bulk<D>(x, n_rec, d.bnd_lo, d.n_ob, d.pb, S.x, L.npos, full, false);
  if (lam) {
    bytes += run_bulk<D>(lam, n_rec, d.int_lo, d.n_int, d.pi, S.lam, L.npos, full, false);
    bytes += run_bulk<D>(lam, n_rec, d.bnd_lo, d.n_ob, d.pb, S.lam, L.npos, full, false);
  }
  mbar_arrive_tx(full, bytes);
  if (b_ent) bulk_load(S.ent, inc + d.i0, b_ent, full);
  bulk_load(S.ptr, ptr + d.q0, b_ptr, full);
  if (b_w) bulk_load(S.w, w + d.w0, b_w, full);
  if (b_f) bulk_load(S.flist, flist + d.f0, b_f, full);
  run_bulk<D>(x, n_rec, d.int_lo, d.n_int, d.pi, S.x, L.npos, full, true);
  run_bulk<D>(x, n_rec, d.bnd_lo, d.n_ob, d.pb, S.x, L.npos, full, true);
  if (lam) {
    run_bulk<D>(lam, n_rec, d.int_lo, d.n_int, d.pi, S.lam, L.npos, full, true);
    run_bulk<D>(lam, n_rec, d.bnd_lo, d.n_ob, d.pb, S.lam, L.npos, full, true);
  }
}

// Producer warp, all lanes: pull a later schedule block into L2 so that its
// stage fill later hits L2 (contiguous pieces with bulk prefetches, foreign
// records one line each).
template <int D, int K = 0>
__device__ __forceinline__ void run_prefetch(const float* gx, int64_t n, int lo, int cnt) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    const int a = lo / (4 / W) * (4 / W);
    const int e = (lo + cnt + 4 / W - 1) / (4 / W) * (4 / W);
    if (e > a) bulk_prefetch_l2(gx + F * n + (int64_t)a * W, (uint32_t)(e - a) * W * 4);
    run_prefetch<D, K + 1>(gx, n, lo, cnt);
  }
}
template <int D, int K = 0>
__device__ __forceinline__ void rec_prefetch(const float* gx, int64_t n, int64_t r) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    prefetch_l2(gx + F * n + r * W);
    rec_prefetch<D, K + 1>(gx, n, r);
  }
}
template <int D>
__device__ __forceinline__ void prefetch_block(const FluxDesc& d, const int32_t* __restrict__ flist,
                                               const uint32_t* __restrict__ inc,
                                               const uint16_t* __restrict__ ptr,
                                               const float* __restrict__ w, const float* x,
                                               const float* lam, int64_t n_rec, int lane) {
  if (lane == 0) {
    bulk_prefetch_l2(inc + d.i0, (uint32_t)pad4(d.nent) * 4u);
    bulk_prefetch_l2(ptr + d.q0, (uint32_t)pad8(d.np + 1) * 2u);
    bulk_prefetch_l2(w + d.w0, (uint32_t)pad4(d.ne) * 4u);
    if (d.nf) bulk_prefetch_l2(flist + d.f0, (uint32_t)pad4(d.nf) * 4u);
  } else if (lane == 1) {
    run_prefetch<D>(x, n_rec, d.int_lo, d.n_int);
    run_prefetch<D>(x, n_rec, d.bnd_lo, d.n_ob);
    if (lam) {
      run_prefetch<D>(lam, n_rec, d.int_lo, d.n_int);
      run_prefetch<D>(lam, n_rec, d.bnd_lo, d.n_ob);
    }
  }
  for (int i = lane; i < d.nf; i += 32) {
    const int32_t r = __ldg(flist + d.f0 + i);
    rec_prefetch<D>(x, n_rec, r);
    if (lam) rec_prefetch<D>(lam, n_rec, r);
  }
}

// Consumers: cp.async of the foreign records (everything the bulk copies
// leave out), thread `ct` of `nct`.
template <int D>
__device__ __forceinline__ void gather(const StageRefs& S, const TmaLayout& L, const float* x,
                                       const float* lam, int64_t n_rec, int ct, int nct) {
  const FluxDesc& d = *S.desc;
  for (int i = ct; i < d.nf; i += nct) {
    const int32_t r = S.flist[i];
    rec_cp_async<D>(S.x, L.npos, d.pf + i, x, n_rec, r);
    if (lam) rec_cp_async<D>(S.lam, L.npos, d.pf + i, lam, n_rec, r);
  }
}

__device__ __forceinline__ int32_t pos_rec(const FluxDesc& d, const int32_t* sflist, int p) {
  if (p < d.pi + d.n_int) return d.int_lo + (p - d.pi);
  if (p < d.pb + d.n_ob) return d.bnd_lo + (p - d.pb);
  return sflist[p - d.pf];
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Shared scaffolding of the persistent kernels.  Schedule blocks are dealt
// round-robin (block j of this CUDA block is blockIdx.x + j * gridDim.x).
// `consume(S, ct, nct)` computes one stage.
template <int D, bool ADJ, typename Consume>
__device__ __forceinline__ void pipeline(const FluxDesc* __restrict__ desc,
                                         const int32_t* __restrict__ flist,
                                         const uint32_t* __restrict__ inc,
                                         const uint16_t* __restrict__ ptr,
                                         const float* __restrict__ w, const float* x,
                                         const float* lam, int64_t n_rec, int64_t k,
                                         int* __restrict__ err, const TmaLayout L, Consume consume) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  // launched with programmatic serialisation: wait for the previous kernel
  // on the stream (its writes to x, lam and the accumulators) first
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ int done;  // schedule blocks finished by the consumers
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nspec = L.ahead > 0 ? 2 : 1;                 // producer (+ prefetch) warps
  const int ncw = (int)(blockDim.x >> 5) - nspec;        // consumer warps
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    done = 0;
    for (int s = 0; s < L.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], (uint32_t)ncw);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    if (lane != 0) return;
    int64_t b = blockIdx.x;
    FluxDesc dn;
    if (b < k) dn = desc[b];
    for (int j = 0;; ++j, b += G) {
      const int s = j % L.stages;
      if (j >= L.stages && !mbar_wait(&empty[s], (uint32_t)((j / L.stages) - 1) & 1u)) {
        atomicOr(err, kErrTimeoutEmpty);
        return;
      }
      const StageRefs S = stage_refs(smem, L, s);
      if (b >= k) {
        *S.block = -1;
        mbar_arrive(&full[s]);
        return;
      }
      if (j == L.stall) return;  // test hook: this stage is never filled
      const FluxDesc d = dn;
      if (b + G < k) dn = desc[b + G];  // next descriptor in flight while copying this one
      produce<D>(d, (int)b, flist, inc, ptr, w, x, ADJ ? lam : nullptr, n_rec, S, L, &full[s]);
    }
  }
  if (L.ahead > 0 && warp == 1) {
    // prefetch warp: keeps the schedule blocks up to L.ahead past the one being
    // computed in L2; paced by the consumers' progress counter
    const long long t0 = clock64();
    int64_t b = blockIdx.x;
    for (int j = 0; b < k; ++j, b += G) {
      while (j - *(volatile int*)&done > L.ahead) {
        __nanosleep(200);
        if (clock64() - t0 > kWaitCycles) return;  // pacing only; nothing waits on this warp
      }
      prefetch_block<D>(desc[b], flist, inc, ptr, w, x, ADJ ? lam : nullptr, n_rec, lane);
    }
    return;
  }
  // consumers
  const int ct = (int)threadIdx.x - 32 * nspec, nct = ncw * 32;
  if (consumers_any(!mbar_wait(&full[0], 0u), nct)) {
    if (ct == 0) atomicOr(err, kErrTimeoutFull);
    return;
  }
  {
    const StageRefs S0 = stage_refs(smem, L, 0);
    if (*S0.block < 0) return;
    gather<D>(S0, L, x, ADJ ? lam : nullptr, n_rec, ct, nct);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int j = 0;; ++j) {
    const int s = j % L.stages, s1 = (j + 1) % L.stages;
    const StageRefs S = stage_refs(smem, L, s);
    // start gathering the next block before computing this one
    if (consumers_any(!mbar_wait(&full[s1], (uint32_t)((j + 1) / L.stages) & 1u), nct)) {
      if (ct == 0) atomicOr(err, kErrTimeoutFull);
      asm volatile("cp.async.wait_all;" ::: "memory");
      return;
    }
    const StageRefs S1 = stage_refs(smem, L, s1);
    const bool more = *S1.block >= 0;
    if (more) gather<D>(S1, L, x, ADJ ? lam : nullptr, n_rec, ct, nct);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    consumer_sync(nct);
    consume(S, ct, nct);
    // the stage was written through the generic proxy (cp.async) and will be
    // refilled through the async proxy (bulk copies)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (ct == 0) *(volatile int*)&done = j + 1;
    if (!more) break;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ------------------------------------------------------------------ forward

template <int D>
__global__ void __launch_bounds__(1024) flux_fwd_tma_kernel(
    const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
    const uint32_t* __restrict__ inc, const uint16_t* __restrict__ ptr, const float* __restrict__ w,
    const float* x_in, float* x_out, float* __restrict__ bacc, float* __restrict__ out, int64_t n_rec,
    int64_t n_int, int64_t n_bnd, float tau, int64_t k, int* err, TmaLayout L) {
  auto consume = [&](const StageRefs& S, int ct, int nct) {
    const FluxDesc d = *S.desc;
    for (int p = ct; p < d.np; p += nct) {
      const int k0 = S.ptr[p], k1 = S.ptr[p + 1];
      if (k0 == k1) continue;  // unused position
      float xp[D], acc[D];
      srec_load<D>(S.x, L.npos, p, xp);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = 0.f;
      // two entries per iteration: their loads are independent
      int q = k0;
      for (; q + 1 < k1; q += 2) {
        const uint32_t e0 = S.ent[q], e1 = S.ent[q + 1];
        float xa[D], xb[D];
        srec_load<D>(S.x, L.npos, (int)(e0 & kPosMask), xa);
        srec_load<D>(S.x, L.npos, (int)(e1 & kPosMask), xb);
        const float wa = S.w[(e0 >> kTaskShift) & 0xffffu], wb = S.w[(e1 >> kTaskShift) & 0xffffu];
        float qa = 0.f, qb = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          xa[c] -= xp[c];
          xb[c] -= xp[c];
          qa = fmaf(xa[c], xa[c], qa);
          qb = fmaf(xb[c], xb[c], qb);
        }
        const float ca = __fdividef(wa, 1.f + qa), cb = __fdividef(wb, 1.f + qb);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = fmaf(cb, xb[c], fmaf(ca, xa[c], acc[c]));
      }
      if (q < k1) {
        const uint32_t e = S.ent[q];
        float xo[D];
        srec_load<D>(S.x, L.npos, (int)(e & kPosMask), xo);
        float s2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          xo[c] -= xp[c];
          s2 = fmaf(xo[c], xo[c], s2);
        }
        const float coef = __fdividef(S.w[(e >> kTaskShift) & 0xffffu], 1.f + s2);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = fmaf(coef, xo[c], acc[c]);
      }
      const int32_t r = pos_rec(d, S.flist, p);
      if (p < d.pi + d.n_int) {
        float xn[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xn[c] = fmaf(tau, acc[c], xp[c]);
        grec_store<D>(x_out, n_rec, r, xn);
        if (out) grec_store<D>(out, n_rec, r, acc);
      } else {
        grec_red<D>(bacc, n_bnd, r - n_int, acc);
      }
    }
  };
  pipeline<D, false>(desc, flist, inc, ptr, w, x_in, nullptr, n_rec, k, err, L, consume);
}

// ------------------------------------------------------------------ adjoint

template <int D>
__global__ void __launch_bounds__(1024) flux_adj_tma_kernel(
    const FluxDesc* __restrict__ desc, const int32_t* __restrict__ flist,
    const uint32_t* __restrict__ inc, const uint16_t* __restrict__ ptr, const float* __restrict__ w,
    const float* x, float* lam, float* __restrict__ gw, float* __restrict__ bacc, int64_t n_rec,
    int64_t n_int, int64_t n_bnd, float tau, int64_t k, int* err, TmaLayout L) {
  auto consume = [&](const StageRefs& S, int ct, int nct) {
    const FluxDesc d = *S.desc;
    for (int p = ct; p < d.np; p += nct) {
      const int k0 = S.ptr[p], k1 = S.ptr[p + 1];
      if (k0 == k1) continue;
      float xp[D], lp[D], acc[D];
      srec_load<D>(S.x, L.npos, p, xp);
      srec_load<D>(S.lam, L.npos, p, lp);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = 0.f;
      for (int q = k0; q < k1; ++q) {
        const uint32_t e = S.ent[q];
        const int o = (int)(e & kPosMask);
        const int t = (int)((e >> kTaskShift) & 0xffffu);
        float xo[D], lo[D];
        srec_load<D>(S.x, L.npos, o, xo);
        srec_load<D>(S.lam, L.npos, o, lo);
        float dd[D], g[D], s2 = 0.f, dg = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          dd[c] = xo[c] - xp[c];
          g[c] = lp[c] - lo[c];
          s2 = fmaf(dd[c], dd[c], s2);
          dg = fmaf(dd[c], g[c], dg);
        }
        const float inv = __fdividef(1.f, 1.f + s2);
        const float we = S.w[t];
        const float two = 2.f * dg * inv * inv;
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] -= we * (g[c] * inv - two * dd[c]);
        // one writer per task: a fire-and-forget reduction instead of a load in the loop
        if (e & kSrcBit) atomicAdd(gw + d.w0 + t, tau * dg * inv);
      }
      const int32_t r = pos_rec(d, S.flist, p);
      if (p < d.pi + d.n_int) {
#pragma unroll
        for (int c = 0; c < D; ++c) lp[c] = fmaf(tau, acc[c], lp[c]);
        grec_store<D>(lam, n_rec, r, lp);
      } else {
        grec_red<D>(bacc, n_bnd, r - n_int, acc);
      }
    }
  };
  pipeline<D, true>(desc, flist, inc, ptr, w, x, lam, n_rec, k, err, L, consume);
}

// Launch configuration with programmatic stream serialisation: the kernel may
// be scheduled while the previous kernel on the stream drains; it waits for
// that kernel's completion (griddepcontrol.wait) before touching memory.
struct PdlConfig {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  PdlConfig(dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
};

template <int D>
cudaError_t launch_fwd(const FluxArgs& a, const TmaPlan& P, cudaStream_t st) {
  PdlConfig c(P.grid, P.threads, P.smem, st);  // shared-memory limit raised when the plan was made
  return cudaLaunchKernelEx(&c.cfg, flux_fwd_tma_kernel<D>, a.desc, a.flist, a.inc, a.ptr, a.w,
                            a.x_in, a.x_out, a.bacc, a.out, a.n_rec, a.n_int, a.n_bnd, a.tau, a.k,
                            P.err, P.L);
}

template <int D>
cudaError_t launch_adj(const FluxArgs& a, const TmaPlan& P, float* lam, float* gw, cudaStream_t st) {
  PdlConfig c(P.grid, P.threads, P.smem, st);
  return cudaLaunchKernelEx(&c.cfg, flux_adj_tma_kernel<D>, a.desc, a.flist, a.inc, a.ptr, a.w,
                            (const float*)a.x_in, lam, gw, a.bacc, a.n_rec, a.n_int, a.n_bnd, a.tau,
                            a.k, P.err, P.L);
}

}  // namespace

#define EP_TMA_DISPATCH(D, CALL) \
  switch (D) {                   \
    case 1: return CALL(1);      \
    case 2: return CALL(2);      \
    case 3: return CALL(3);      \
    case 4: return CALL(4);      \
    case 5: return CALL(5);      \
    case 6: return CALL(6);      \
    case 7: return CALL(7);      \
    case 8: return CALL(8);      \
  }                              \
  return cudaErrorInvalidValue;

cudaError_t flux_fwd_tma(const FluxArgs& a, const TmaPlan& P, int D, cudaStream_t st) {
#define EP_F(DD) launch_fwd<DD>(a, P, st)
  EP_TMA_DISPATCH(D, EP_F)
#undef EP_F
}

cudaError_t flux_adj_tma(const FluxArgs& a, const TmaPlan& P, int D, float* lam, float* gw,
                         cudaStream_t st) {
#define EP_A(DD) launch_adj<DD>(a, P, lam, gw, st)
  EP_TMA_DISPATCH(D, EP_A)
#undef EP_A
}

const void* flux_tma_kernel_ptr(int D, bool adjoint) {
  switch (D) {
    case 1: return adjoint ? (const void*)flux_adj_tma_kernel<1> : (const void*)flux_fwd_tma_kernel<1>;
    case 2: return adjoint ? (const void*)flux_adj_tma_kernel<2> : (const void*)flux_fwd_tma_kernel<2>;
    case 3: return adjoint ? (const void*)flux_adj_tma_kernel<3> : (const void*)flux_fwd_tma_kernel<3>;
    case 4: return adjoint ? (const void*)flux_adj_tma_kernel<4> : (const void*)flux_fwd_tma_kernel<4>;
    case 5: return adjoint ? (const void*)flux_adj_tma_kernel<5> : (const void*)flux_fwd_tma_kernel<5>;
    case 6: return adjoint ? (const void*)flux_adj_tma_kernel<6> : (const void*)flux_fwd_tma_kernel<6>;
    case 7: return adjoint ? (const void*)flux_adj_tma_kernel<7> : (const void*)flux_fwd_tma_kernel<7>;
    case 8: return adjoint ? (const void*)flux_adj_tma_kernel<8> : (const void*)flux_fwd_tma_kernel<8>;
  }
  return nullptr;
}

}  // namespace dev
}  // namespace ep
