// flux_tma.cu -- persistent, pipelined flux kernels (sm_103a).
//
// The software-cache kernel of Section 4 (Fig. 7(d)) under the partition of
// Section 3, organised so that loading later kernel blocks overlaps
// computing the current one.  Each persistent CUDA block owns NS
// shared-memory stages:
//   producer (one thread)  deals kernel blocks round-robin and copies each
//                  block's contiguous pieces (its record run in every state
//                  plane, its slots and slot weights, its shared ids and slice
//                  offsets) with 1-D TMA bulk copies that complete on the
//                  stage's "full" mbarrier.  With every shared vertex
//                  replicated in each block that uses it, a block's vertex set
//                  is one run of records, so a stage fills in one round trip
//                  with no dependent gather;
//   fix-up warps   bring the staged copies of shared vertices up to date
//                  with the previous step's sums (the copies lag one step)
//                  and mark the stage "ready";
//   consumer warps each take whole slices (32 positions) of a stage, sum the
//                  flux of every position from shared memory (pull form),
//                  write back (interior vertices in place; shared vertices
//                  one vector reduction into this step's accumulator, which
//                  the next step or the finish applies to every copy, and
//                  the up-to-date copy), and arrive on the stage's "empty"
//                  mbarrier.  Warps move through the
//                  stages independently (no block-wide barrier per kernel
//                  block); slices are dealt so that every warp gets the same
//                  share over the run.
// Every wait is bounded by a clock budget; on expiry the kernel records an
// error code and returns instead of hanging.
#include <cuda_runtime.h>

#include <cstdint>

#include "flux_common.cuh"
#include "kernels.h"
#include "tma_sync.cuh"

namespace ep {
namespace dev {
namespace {

constexpr int kErrTimeoutFull = 1;
constexpr int kErrTimeoutEmpty = 2;

// ------------------------------------------------------------ stage layout

struct StageRefs {
  float* x;
  float* lam;
  uint16_t* sidx;
  float* w;
  int32_t* sid;
  uint16_t* soff;
  FluxDesc* desc;
};

__device__ __forceinline__ StageRefs stage_refs(unsigned char* base, const TmaLayout& L, int s) {
  unsigned char* p = base + (size_t)s * L.stage_bytes;
  StageRefs r;
  r.x = reinterpret_cast<float*>(p);
  r.lam = reinterpret_cast<float*>(p + L.off_lam);
  r.sidx = reinterpret_cast<uint16_t*>(p + L.off_sidx);
  r.w = reinterpret_cast<float*>(p + L.off_w);
  r.sid = reinterpret_cast<int32_t*>(p + L.off_sid);
  r.soff = reinterpret_cast<uint16_t*>(p + L.off_soff);
  r.desc = reinterpret_cast<FluxDesc*>(p + L.off_desc);
  return r;
}

__device__ __forceinline__ uint32_t up16(uint32_t bytes) { return (bytes + 15u) & ~15u; }

// Bulk pieces of the record run [lo, lo + nv) in every plane: the run starts
// on a 4-record boundary, so each plane moves as whole 16-byte chunks.
// `issue` false only sums the bytes.
template <int D, int K = 0>
__device__ __forceinline__ uint32_t run_bulk(const float* gx, int64_t n, int lo, int nv, float* sx,
                                             int npos, uint64_t* bar, bool issue) {
  if constexpr (K < Planes<D>::NP) {
    constexpr int W = Planes<D>::width(K), F = Planes<D>::first(K);
    const uint32_t bytes = up16((uint32_t)nv * W * 4u);
    if (issue) bulk_load(sx + F * npos, gx + F * n + (int64_t)lo * W, bytes, bar);
    return bytes + run_bulk<D, K + 1>(gx, n, lo, nv, sx, npos, bar, issue);
  }
  return 0;
}

// Producer (one thread): bulk copies of kernel block `d` into stage S.
template <int D>
__device__ __forceinline__ void produce(const FluxDesc& d, const FluxArgs& a, const float* lam,
                                        const StageRefs& S, const TmaLayout& L, uint64_t* full) {
  *S.desc = d;
  const uint32_t b_ix = (uint32_t)d.nslot * 2u, b_w = (uint32_t)d.nslot * 4u;
  const uint32_t b_sid = up16((uint32_t)(d.nv - d.ni) * 4u);
  const uint32_t b_so = up16((uint32_t)(d.nsl + 1) * 2u);
  uint32_t bytes = b_ix + b_w + b_sid + b_so;
  bytes += run_bulk<D>(a.x_in, a.n_rec, d.rec_lo, d.nv, S.x, L.npos, full, false);
  if (lam) bytes += run_bulk<D>(lam, a.n_rec, d.rec_lo, d.nv, S.lam, L.npos, full, false);
  mbar_arrive_tx(full, bytes);
  run_bulk<D>(a.x_in, a.n_rec, d.rec_lo, d.nv, S.x, L.npos, full, true);
  if (lam) run_bulk<D>(lam, a.n_rec, d.rec_lo, d.nv, S.lam, L.npos, full, true);
  bulk_load(S.sidx, a.sidx + d.s0, b_ix, full);
  bulk_load(S.w, a.w + d.s0, b_w, full);
  bulk_load(S.soff, a.soff + d.q0, b_so, full);
  if (b_sid) bulk_load(S.sid, a.sid + d.h0, b_sid, full);
}

// Shared scaffolding of the persistent kernels.  Kernel blocks are dealt
// round-robin (block j of this CUDA block is blockIdx.x + j * gridDim.x).
//   warp 0, lane 0: producer, fills the stages with bulk copies ("full");
//   warps 1..kFixupWarps: fix-up, bring the staged copies of shared vertices
//           up to date from the previous step's accumulator (flux_common.cuh)
//           while the consumers work on earlier stages, then mark the stage
//           "ready".  With F = min(kFixupWarps, stages) of them at work,
//           fix-up warp f owns the stages s with s % F == f and takes their
//           fills in order: a parity wait only tells the current phase from
//           the one before it, so every fill of a stage must be awaited by
//           one thread in order (F warps keep F stages' gathers in flight);
//   the other warps: consumers, consume(S, d, slice, lane, acc) computes and writes
//           back one slice, adding the partial sums of shared vertices into
//           this step's accumulator; the last consumer warp done with a stage
//           lets the producer refill it ("empty").
// fix: the planes (state, or cotangent for the adjoint) whose copies are
// pending.  Ends with the phase advance.
template <int D, bool ADJ, typename Consume>
__device__ __forceinline__ void pipeline(const FluxArgs& a, const float* lam_in, int* err,
                                         const TmaLayout L, Consume consume) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], ready[kMaxStages], empty[kMaxStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncw = (int)(blockDim.x >> 5) - 1 - kFixupWarps;  // consumer warps
  const int64_t G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < L.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 1);
      mbar_init(&empty[s], (uint32_t)ncw);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // launched with programmatic serialisation: wait for the previous kernel on
  // the stream (its writes to the state and the accumulators) first
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int q = *a.phase;
  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;  // stage fills issued: fill i went to stage i % stages
      int64_t b = blockIdx.x;
      FluxDesc dn;
      if (b < a.k) dn = a.desc[b];
      for (int j = 0;; ++j, b += G) {
        const int s = j % L.stages;
        if (j >= L.stages && !mbar_wait(&empty[s], (uint32_t)((j / L.stages) - 1) & 1u)) {
          atomicOr(err, kErrTimeoutEmpty);
          break;
        }
        const StageRefs S = stage_refs(smem, L, s);
        if (b >= a.k) {  // end markers, one in every stage (each fix-up warp owns stages)
          S.desc->nv = -1;
          mbar_arrive(&full[s]);
          ++issued;
          if (b >= a.k + (int64_t)(L.stages - 1) * G) break;
          continue;
        }
        if (j == L.stall) break;  // test hook: this stage is never filled
        const FluxDesc d = dn;
        if (b + G < a.k) dn = a.desc[b + G];  // next descriptor in flight while copying this one
        produce<D>(d, a, ADJ ? lam_in : nullptr, S, L, &full[s]);
        ++issued;
      }
      // never leave the CTA with copies in flight: wait (bounded) for the last
      // fill of every stage
      for (int s = 0; s < L.stages && s < issued; ++s) {
        const int fills = (issued - s + L.stages - 1) / L.stages;
        mbar_wait(&full[s], (uint32_t)(fills - 1) & 1u);
      }
    }
    __syncwarp();
  } else if (warp <= kFixupWarps) {
    const float* prev = acc_buffer<D>(a, q + 2);
    float* next = acc_buffer<D>(a, q + 1);
    const int nfix = min(kFixupWarps, L.stages);  // a warp past nfix owns no stage
    for (int j = 0; warp - 1 < nfix; ++j) {
      const int s = j % L.stages;
      if (s % nfix != warp - 1) continue;
      const uint32_t par = (uint32_t)(j / L.stages) & 1u;
      const bool ok = mbar_wait(&full[s], par);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(err, kErrTimeoutFull);
        break;
      }
      const StageRefs S = stage_refs(smem, L, s);
      const FluxDesc d = *S.desc;
      if (d.nv >= 0) {
        fixup_copies<D>(d, ADJ ? S.lam : S.x, L.npos, S.sid, prev, next, a.tau, lane, 32);
        // the stage is written through the generic proxy here and refilled
        // through the async proxy later
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
      if (d.nv < 0) break;
    }
  } else {
    float* acc = acc_buffer<D>(a, q);
    const int cw = warp - 1 - kFixupWarps;
    int rot = 0;  // slices dealt so far, mod ncw
    int s = 0;
    uint32_t par = 0;
    for (;;) {
      const bool ok = mbar_wait(&ready[s], par) && mbar_wait(&full[s], par);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(err, kErrTimeoutFull);
        break;
      }
      const StageRefs S = stage_refs(smem, L, s);
      const FluxDesc d = *S.desc;
      if (d.nv < 0) break;
      int sl = cw - rot;
      if (sl < 0) sl += ncw;
      for (; sl < d.nsl; sl += ncw) consume(S, d, sl, lane, acc);
      rot += d.nsl;
      while (rot >= ncw) rot -= ncw;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (++s == L.stages) s = 0, par ^= 1u;
    }
  }
  advance_phase(a, q);
}

// ------------------------------------------------------------------ forward

template <int D>
__global__ void __maxnreg__(56) flux_fwd_tma_kernel(const FluxArgs a, int* err,
                                                    TmaLayout L) {
  auto consume = [&](const StageRefs& S, const FluxDesc& d, int sl, int lane, float* bacc) {
    fwd_block_slice<D>(a, bacc, d, S.x, L.npos, S.sidx, S.w, S.soff, S.sid, sl, lane);
  };
  pipeline<D, false>(a, nullptr, err, L, consume);
}

// ------------------------------------------------------------------ adjoint

template <int D>
__global__ void __launch_bounds__(1024) flux_adj_tma_kernel(const FluxArgs a, float* lam, float* gw,
                                                            int* err, TmaLayout L) {
  auto consume = [&](const StageRefs& S, const FluxDesc& d, int sl, int lane, float* bacc) {
    adj_block_slice<D>(a, bacc, d, S.x, S.lam, L.npos, S.sidx, S.w, S.soff, S.sid, lam, gw, sl, lane);
  };
  pipeline<D, true>(a, lam, err, L, consume);
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
  return cudaLaunchKernelEx(&c.cfg, flux_fwd_tma_kernel<D>, a, P.err, P.L);
}

template <int D>
cudaError_t launch_adj(const FluxArgs& a, const TmaPlan& P, float* lam, float* gw, cudaStream_t st) {
  PdlConfig c(P.grid, P.threads, P.smem, st);
  return cudaLaunchKernelEx(&c.cfg, flux_adj_tma_kernel<D>, a, lam, gw, P.err, P.L);
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
