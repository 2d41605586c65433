// internal.h -- shared declarations of libepcache (not part of the C ABI).
#pragma once

#include <atomic>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace ep {

// Flux kernels: one descriptor per kernel block (a schedule block, or a piece
// of an oversize one).  The block's vertices V_b sit at positions [0, nv):
//   [0, ni)    vertices no other kernel block uses (p_v = 1), in-place update;
//   [ni, nv)   shared vertices (p_v > 1); each kernel block holds its own copy
//              (replica) of every shared vertex it uses, so position p is always
//              the state record rec_lo + p and a block's vertex set is one
//              contiguous run; sid_list[h0 + p - ni] is the shared id h that
//              indexes the accumulators (kSidFirst marks the first copy of h).
// Within each class positions are ordered by descending in-block degree.
// Incidence in sliced-ELL form: slice j holds the positions [32 j, 32 j + 32);
// its incidence entries occupy K_j = soff[q0 + j + 1] - soff[q0 + j] columns
// of 32 slots, slot = s0 + 32 * soff[q0 + j] + 32 * column + lane, so that a
// warp reads one column with one access per array.  A slot holds the other
// endpoint's position (bits 0-14) and a source flag (bit 15: this position is
// the task's first endpoint), and the task weight in the same slot of the
// weight layout; an unused slot has weight 0 and names some position of the
// block (one that spreads the slice's loads over the shared-memory banks), so
// its term is exactly zero.  Every task has one slot at each
// endpoint (one for a self loop), so the forward flux is computed from either
// side without signs (pull form).  Every per-block segment starts on a 16-byte
// boundary and is padded to a multiple of 16 bytes (one bulk copy each).
struct FluxDesc {
  int32_t rec_lo, nv, ni, nsl;  // record run, positions, interior positions, slices
  int32_t s0, nslot;            // slots [s0, s0 + nslot), both multiples of 32
  int32_t h0, q0;               // shared ids sid_list[h0 ..], slice offsets soff[q0 ..]
  int32_t ne;                   // tasks of the block
  int32_t pad[7];
};
static_assert(sizeof(FluxDesc) == 64, "FluxDesc layout");

// Slot fields (flux)
constexpr uint16_t kSlotPos = 0x7fffu;
constexpr uint16_t kSlotSrc = 0x8000u;
constexpr int32_t kSidFirst = INT32_MIN;   // sid_list: first copy of this shared vertex
constexpr int32_t kSidMask = 0x7fffffff;

// SpMV entry fields: (row position << 16) | x position
constexpr int kRowShift = 16;
constexpr uint32_t kColMask = 0xffffu;

// SpMV kernels (bipartite): x records are read only, y records accumulate.
// x positions: [0, n_xo) the run x_lo.., then n_xf ids from xlist[fx0..].
// y positions: [0, n_yi) the single-block rows yi_lo.., [n_yi, n_yi + n_yob)
// the run yb_lo.. of shared rows first touched here, then n_yf ids from
// ylist[fy0..]; within each class rows are ordered by descending list length.
// The block's ne entries, ranked by row position, go to lane t / u of a warp
// (u entries per lane, a multiple of 4, the same for every block) and are
// stored 4 by 4 interleaved over the lanes (spmv_slot), so that one 16-byte
// load per lane reads 512 consecutive bytes; the task weight of the entry in
// slot j is w_lay[i0 + j].  Every block's runs hold 32 * u slots (padding:
// entry 0, weight 0), so block b's start at i0 = 32 * u * b.
struct SpmvDesc {
  int32_t i0, ne, u;
  int32_t x_lo, n_xo, fx0, n_xf;
  int32_t yi_lo, n_yi, yb_lo, n_yob, fy0, n_yf;
  int32_t pad[3];
};
static_assert(sizeof(SpmvDesc) == 64, "SpmvDesc layout");
// slot (from i0) of the entry ranked t in row order, u entries per lane
inline int32_t spmv_slot(int32_t t, int32_t u) {
  const int32_t lane = t / u, j = t % u;
  return ((j >> 2) * 32 + lane) * 4 + (j & 3);
}

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

  // flux layout (non-bipartite), built over the kernel blocks
  int64_t n_rec = 0;         // records per state plane (multiple of 4)
  int64_t n_run = 0;         // records [0, n_run) are block runs; untouched vertices follow
  int64_t n_sh = 0;          // shared vertices (accumulator records)
  std::vector<int32_t> rec_of;    // data vertex -> its record (a shared vertex: its first copy)
  std::vector<int32_t> vrec;      // record -> data vertex (-1: padding)
  std::vector<int32_t> cptr, crec;  // copies of shared vertex s: crec[cptr[s] .. cptr[s+1])
  std::vector<int32_t> sid_list;  // shared id of every shared position, per block
  std::vector<int32_t> fold_rec, fold_sid;  // every copy: its record and shared id (fold order)
  std::vector<uint16_t> sidx;     // slot entries
  std::vector<uint16_t> soff;     // slice column offsets, per block
  std::vector<int32_t> gslot;     // task -> its source-side slot
  std::vector<FluxDesc> fdesc;
  int32_t max_nv = 0, max_nslot = 0, max_nsh = 0, max_nsl = 0;
  int64_t w_pad = 0;           // slots of the weight layout
  std::vector<int32_t> wmap;   // weight slot -> task id (-1 for padding)
  std::vector<int32_t> halo;   // data vertices forced onto the shared path (a shard's halo)

  // spmv layout (bipartite): x records 0..n-1, y records 0..n-1
  int64_t ny_int = 0, ny_bnd = 0;
  std::vector<int32_t> xrec_of, yrec_of;  // by column / row index
  std::vector<SpmvDesc> sdesc;
  std::vector<int32_t> xlist, ylist;
  std::vector<uint32_t> sent;   // SpMV entries (padded runs, see SpmvDesc)
  int32_t max_nx = 0, max_ny = 0;
  int32_t max_nxy = 0;  // largest x + y positions of a block, each rounded up to 4
  int32_t spmv_u = 0;   // entries per lane (every block: 32 * spmv_u slots)
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
// The flux layout again (after `halo` changed); non-bipartite schedules only.
std::string rebuild_flux_layout(HostSchedule& s);

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
