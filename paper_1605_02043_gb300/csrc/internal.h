// internal.h -- shared declarations of libepcache (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace ep {

// Flux kernels: one descriptor per schedule block.  A block's local slots are
//   [0, n_int)                  records used by this block only (p_v = 1),
//                               contiguous from int_lo;
//   [n_int, n_int + n_ob)       records first touched by this block and used
//                               by later blocks too, contiguous from bnd_lo;
//   [n_int + n_ob, ... + nf)    records owned by earlier blocks, listed in
//                               flist[f0 .. f0 + nf).
struct FluxDesc {
  int32_t e0, ne;
  int32_t int_lo, n_int;
  int32_t bnd_lo, n_ob;
  int32_t f0, nf;
};
static_assert(sizeof(FluxDesc) == 32, "FluxDesc layout");

// SpMV kernels (bipartite): x records are read only, y records accumulate.
//   x slots: [0, n_xo) contiguous from x_lo, then n_xf from xlist[fx0..]
//   y slots: [0, n_yi) interior from yi_lo, [n_yi, n_yi + n_yob) from yb_lo,
//            then n_yf from ylist[fy0..]
struct SpmvDesc {
  int32_t e0, ne;
  int32_t x_lo, n_xo, fx0, n_xf;
  int32_t yi_lo, n_yi, yb_lo, n_yob, fy0, n_yf;
  int32_t pad[4];
};
static_assert(sizeof(SpmvDesc) == 64, "SpmvDesc layout");

// Host part of a schedule plus the kernel layout derived from it.
struct HostSchedule {
  int64_t m = 0, n = 0, nd = 0, k = 0;
  int32_t C = 0;
  uint32_t flags = 0;
  std::vector<int32_t> src, dst;  // caller's task list
  std::vector<int32_t> part;      // block of every task
  std::vector<int64_t> block_ptr, vert_ptr;
  std::vector<int32_t> edge_perm, vert_list, relabel;
  int64_t loads = 0, touched = 0;
  int32_t max_ne = 0;

  // flux layout (non-bipartite)
  int64_t n_int = 0;        // records [0, n_int) are single-block vertices
  int64_t n_bnd = 0;        // records [n_int, n_int + n_bnd) are shared
  std::vector<int32_t> rec_of;  // data vertex -> record (all nd vertices)
  std::vector<FluxDesc> fdesc;
  std::vector<int32_t> flist;
  int32_t max_nv = 0;

  // spmv layout (bipartite): x records 0..n-1, y records 0..n-1
  int64_t ny_int = 0, ny_bnd = 0;
  std::vector<int32_t> xrec_of, yrec_of;  // by column / row index
  std::vector<SpmvDesc> sdesc;
  std::vector<int32_t> xlist, ylist;
  int32_t max_nx = 0, max_ny = 0;

  std::vector<uint32_t> loc;  // per task in edge_perm order: slot(u) | slot(v) << 16
};

// partition.cpp
void partition_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                     uint32_t flags, int threads, int32_t* part);

// schedule.cpp: everything after the partition (Definition 4, vertex lists,
// cpack, cost, kernel layout).  Returns an empty string or an error message.
std::string build_schedule(HostSchedule& s, int threads);

inline int32_t record_floats(int32_t D) {
  return D <= 1 ? 1 : D <= 2 ? 2 : D <= 4 ? 4 : 8;
}

}  // namespace ep
