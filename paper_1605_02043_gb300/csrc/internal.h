// internal.h -- shared declarations of libepcache (not part of the C ABI).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace ep {

// Flux kernels: one descriptor per schedule block.  The block's vertices sit
// at shared-memory positions
//   [pi, pi + n_int)   records used by this block only (p_v = 1), contiguous
//                      from int_lo;
//   [pb, pb + n_ob)    records first touched by this block and used by later
//                      blocks too, contiguous from bnd_lo;
//   [pf, pf + nf)      records owned by earlier blocks, flist[f0 .. f0 + nf);
// with pi = int_lo mod 4 and pb = bnd_lo mod 4 (mod 4), so that a 16-byte
// aligned run of records in a state plane maps to a 16-byte aligned run in
// shared memory.  Positions outside the three runs are unused.  Every
// position p in [0, np) has the incidence entries inc[i0 + ptr[q0 + p] ..
// i0 + ptr[q0 + p + 1]): (other position) | (task << 15) | (p is src << 31).
// The task weights of the block are w_lay[w0 .. w0 + ne).  Every per-block
// segment (entries, offsets, foreign ids, weights) starts on a 16-byte
// boundary and is zero-padded to a multiple of 16 bytes, so it can be moved
// with one bulk copy.
struct FluxDesc {
  int32_t w0, ne;        // task weights w_lay[w0, w0 + ne)
  int32_t int_lo, n_int;
  int32_t bnd_lo, n_ob;
  int32_t f0, nf;
  int32_t pi, pb, pf, np;
  int32_t i0, q0, nent, pad;
};
static_assert(sizeof(FluxDesc) == 64, "FluxDesc layout");

// Incidence entry fields
constexpr uint32_t kPosMask = 0x7fffu;
constexpr int kTaskShift = 15;
constexpr uint32_t kSrcBit = 0x80000000u;

// SpMV kernels (bipartite): x records are read only, y records accumulate.
// x positions: [0, n_xo) the run x_lo.., then n_xf ids from xlist[fx0..].
// y positions: [0, n_yi) the single-block rows yi_lo.., [n_yi, n_yi + n_yob)
// the run yb_lo.. of shared rows first touched here, then n_yf ids from
// ylist[fy0..]; within each class rows are ordered by descending list length.
// Row position p has entries ent[i0 + ptr[q0 + p] .. i0 + ptr[q0 + p + 1]):
// (x position) | (task << 15); task weights are w_lay[w0 .. w0 + ne).
struct SpmvDesc {
  int32_t w0, ne;
  int32_t x_lo, n_xo, fx0, n_xf;
  int32_t yi_lo, n_yi, yb_lo, n_yob, fy0, n_yf;
  int32_t i0, q0, pad[2];
};
static_assert(sizeof(SpmvDesc) == 64, "SpmvDesc layout");

// Host part of a schedule plus the kernel layout derived from it.
struct HostSchedule {
  int64_t m = 0, n = 0, nd = 0, k = 0;
  int32_t C = 0;
  uint32_t flags = 0;
  int32_t origin = 0;             // how the task order was chosen (kOrigin*)
  std::vector<int32_t> src, dst;  // caller's task list
  std::vector<int32_t> part;      // block of every task
  std::vector<int64_t> block_ptr, vert_ptr;
  std::vector<int32_t> edge_perm, vert_list, relabel;
  int64_t loads = 0, touched = 0;
  int32_t max_ne = 0;

  // flux layout (non-bipartite)
  int64_t n_rec = 0;        // records per state plane: nd rounded up to a multiple of 4
  int64_t n_int = 0;        // records [0, n_int) are single-block vertices
  int64_t n_bnd = 0;        // records [n_int, n_int + n_bnd) are shared
  std::vector<int32_t> rec_of;  // data vertex -> record (all nd vertices)
  std::vector<FluxDesc> fdesc;
  std::vector<int32_t> flist;
  std::vector<uint32_t> inc;   // incidence entries (flux)
  std::vector<uint16_t> ptr;   // per-position entry offsets within a block (flux)
  int32_t max_nv = 0;          // max positions per block
  int32_t max_nent = 0;        // max incidence entries per block
  int32_t max_nf = 0;          // max foreign records per block
  int64_t w_pad = 0;           // length of the padded weight layout
  std::vector<int32_t> wmap;   // weight slot -> task id (-1 for padding)

  // spmv layout (bipartite): x records 0..n-1, y records 0..n-1
  int64_t ny_int = 0, ny_bnd = 0;
  std::vector<int32_t> xrec_of, yrec_of;  // by column / row index
  std::vector<SpmvDesc> sdesc;
  std::vector<int32_t> xlist, ylist;
  std::vector<uint32_t> sinc;   // SpMV row entries
  std::vector<uint16_t> sptr;   // SpMV row offsets
  int32_t max_nx = 0, max_ny = 0;
};

// prescreen.cpp: checks made before partitioning (Section 4 workflow).
// Origins match EP_ORIGIN_* in epcache.h.
constexpr int32_t kOriginPartition = 0, kOriginDefault = 1, kOriginPath = 2, kOriginStar = 3,
                  kOriginLowReuse = 4;
struct PrescreenResult {
  int64_t touched = 0, degree_sum = 0, max_degree = 0;
  int32_t origin = kOriginPartition;
  std::vector<int32_t> order;  // path preset: the tasks in walk order
};
PrescreenResult prescreen(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, bool bip);

// partition.cpp.  Returns false (part unfinished) when *stop became non-zero
// during the run.
bool partition_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                     uint32_t flags, int threads, int32_t* part,
                     const std::atomic<int>* stop = nullptr);

// schedule.cpp: everything after the partition (Definition 4, vertex lists,
// cpack, cost, kernel layout).  Returns an empty string or an error message.
std::string build_schedule(HostSchedule& s, int threads);

// State layout: the D components of a record are split into planes of
// width 4, 2 and 1 (D = 4a + 2b + c); plane k holds n_rec records of its
// width contiguously, so a state buffer is n_rec * D floats without padding.
inline int32_t record_floats(int32_t D) { return D; }
// planes of a D-wide record: count, first component and width of each
inline int planes_of(int32_t D, int32_t first[4], int32_t width[4]) {
  int np = 0, c = 0;
  for (int i = 0; i < D / 4; ++i, c += 4) first[np] = c, width[np++] = 4;
  if (D % 4 >= 2) first[np] = c, width[np++] = 2, c += 2;
  if (D % 2) first[np] = c, width[np++] = 1;
  return np;
}

}  // namespace ep
