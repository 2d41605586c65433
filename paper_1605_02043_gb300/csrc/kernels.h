// kernels.h -- launchers of the device code (internal to libepcache).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace ep {
namespace dev {

// Optional per-launch timing hook (events recorded on the launch stream).
struct Timer {
  virtual void begin(int cls, cudaStream_t st) = 0;
  virtual void end(int cls, cudaStream_t st) = 0;
  virtual ~Timer() = default;
};
enum { T_EDGE_FWD = 0, T_BND = 1, T_EDGE_ADJ = 2, T_SPMV = 3, T_LAYOUT = 4, T_COST = 5 };

struct FluxArgs {
  const FluxDesc* desc;
  int64_t k;             // kernel blocks
  const uint16_t* sidx;  // slots
  const uint16_t* soff;  // slice offsets
  const int32_t* sid;    // shared ids of the shared positions
  const float* w;        // task weights in slot layout
  const float* x_in;     // state in schedule layout (planar, n_rec records)
  float* x_out;          // may equal x_in
  float* bacc;           // 3 x n_sh accumulator records (acc_stride(D) floats each) of this kind
  int* phase;            // accumulator phase of this kind (0..2)
  int* done;             // CUDA blocks finished (the last one advances the phase)
  float* out;            // flux in schedule layout or nullptr
  const int32_t* fold_rec;  // every copy of a shared vertex: its record and shared id
  const int32_t* fold_sid;
  int64_t n_copies;
  int64_t n_rec, n_sh;
  float tau;
  int32_t max_nv, max_nslot, max_nsh, max_nsl;
  int tpb;
  Timer* timer;
};

struct SpmvArgs {
  const SpmvDesc* desc;
  int64_t k;
  const int32_t* xlist;
  const int32_t* ylist;
  const uint32_t* ent;   // entries, (row position << 16) | x position
  const float* w;        // weight layout (one weight per entry, same index)
  const float* x;        // x records
  float* y;              // y records; [ny_int, ny_int + ny_zero) zeroed first
  int64_t ny_int, ny_zero;
  int32_t max_nx, max_ny, max_nxy;
  int32_t u;              // entries per lane (every block's runs: 32 u slots)
  int tpb;                // threads per CUDA block (one warp per schedule block)
  bool readonly = false;  // x read through the read-only cache, not staged
  Timer* timer;
};

struct CostArgs {
  const int64_t* block_ptr;
  int64_t k;
  const int32_t* eu;  // endpoint ids in schedule order
  const int32_t* ev;
  int32_t max_ne;
  uint8_t* touched;   // nd bytes of workspace
  int64_t nd;
  unsigned long long* counters;  // [0] loads, [1] touched
  Timer* timer;
};

// Persistent pipelined kernels (flux_tma.cu): per-stage shared-memory layout
// (byte offsets, all multiples of 16) and launch plan.
constexpr int kMaxStages = 8;
// fix-up warps of the pipelined flux kernels (warps 1..kFixupWarps; one
// producer warp and the consumer warps besides)
constexpr int kFixupWarps = 2;
struct TmaLayout {
  int npos;  // positions per state plane (multiple of 4)
  int off_lam, off_sidx, off_w, off_sid, off_soff, off_desc;
  int stage_bytes;
  int stages;
  int stall;  // test hook: leave the stage of this block index unfilled (-1: off)
};
struct TmaPlan {
  TmaLayout L;
  int grid, threads, per_sm;
  size_t smem;
  int* err;  // error word (bit 0: a "full" wait expired, bit 1: an "empty" wait expired)
  bool fits = true;  // false: two stages exceed shared memory; use the one-block kernel
};
// bytes of one stage (state copies: 1 forward, 2 adjoint) and its layout
TmaLayout tma_layout(const FluxArgs& a, int D, bool adjoint);
cudaError_t flux_fwd_tma(const FluxArgs& a, const TmaPlan& P, int D, cudaStream_t st);
cudaError_t flux_adj_tma(const FluxArgs& a, const TmaPlan& P, int D, float* lam, float* gw,
                         cudaStream_t st);
const void* flux_tma_kernel_ptr(int D, bool adjoint);

cudaError_t flux_step(const FluxArgs& a, int D, cudaStream_t st);
// read-only-cache variant (no staging); needs max_np <= 4096
cudaError_t flux_step_ldg(const FluxArgs& a, int D, cudaStream_t st);
// finish of a pending state: every copy r of shared vertex h becomes
// x_out[r] = x_in[r] + tau * prev[h]; out[r] (if not null) = prev[h]
// (flux_common.cuh: the accumulator rotation)
cudaError_t bnd_update(const FluxArgs& a, int D, float* x_out, const float* x_in, float* out,
                       cudaStream_t st);
cudaError_t flux_adjoint_step(const FluxArgs& a, int D, float* lam, float* gw, cudaStream_t st);
cudaError_t spmv(const SpmvArgs& a, cudaStream_t st);
// shared memory the one-block kernels stage for the schedule's largest block
size_t flux_block_smem(const FluxArgs& a, int D, bool adjoint);
// SpMV launch shape: warps (schedule blocks) per CUDA block and the shared
// memory of one CUDA block; 0 warps when one warp's share does not fit
struct SpmvPlan {
  int wpb;      // warps per CUDA block (0: does not fit)
  int cap;      // floats of the per-warp x / y region
  size_t smem;  // dynamic shared memory per CUDA block
};
SpmvPlan spmv_plan(const SpmvArgs& a, int smem_optin);
// SpMV layout in (one record per vertex): x_lay[rec_of[v]] <- x[v]
cudaError_t layout_in(const int32_t* rec_of, int64_t n, int64_t n_rec, int D, const float* x,
                      float* x_lay, cudaStream_t st, Timer* t);
cudaError_t layout_out(const int32_t* rec_of, int64_t n, int64_t n_rec, int D, const float* x_lay,
                       float* x, cudaStream_t st, Timer* t);
// halo sums of a shard schedule (forward kind): pack the last edge kernel's
// sums of halo vertices i (shared id hmap[i], -1: not here) into buf[i][D], or
// unpack buf into them
cudaError_t halo_move(const FluxArgs& a, int D, const int32_t* hmap, int64_t nh, float* buf, bool pack,
                      cudaStream_t st);
// vertex- and task-ordered input forms: x plane by plane in vertex order into
// every record of each vertex (CSR ptr/recs; the flux layout in), and w in
// task order into the task's two slots (slots[2 t], slots[2 t + 1], -1 for
// none; for weights in host memory)
cudaError_t layout_in_csr(const int32_t* ptr, const int32_t* recs, int64_t n, int64_t n_rec, int D,
                          const float* x, float* x_lay, cudaStream_t st, Timer* t);
cudaError_t weights_scatter(const int32_t* slots, int64_t m, const float* w, float* w_lay, cudaStream_t st,
                            Timer* t);
cudaError_t gather(const int32_t* perm, int64_t m, const float* w, float* w_lay, cudaStream_t st,
                   Timer* t);
cudaError_t scatter_add(const int32_t* perm, int64_t m, const float* w_lay, float* w, cudaStream_t st,
                        Timer* t);
// w[t] += w_lay[slot[t]] for t < m
cudaError_t gather_add(const int32_t* slot, int64_t m, const float* w_lay, float* w, cudaStream_t st,
                       Timer* t);
cudaError_t cost(const CostArgs& a, cudaStream_t st);

}  // namespace dev
}  // namespace ep
