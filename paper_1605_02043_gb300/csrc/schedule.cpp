// schedule.cpp -- from a task partition to the arrays the kernels use.
//
//   reconstruction   tasks grouped by block, ascending id inside a block
//                    (Definition 4);
//   vertex lists     distinct data vertices of each block in first-touch
//                    order (the block's share of the data, Section 4 Fig. 7);
//   cpack            ids in order of first appearance over blocks (Section
//                    4.1, after Ding and Kennedy), untouched vertices last;
//   cost             loads = sum_b |V_b|, vertex cut = loads - touched (Eq. 1);
//   kernel layout    the cpack order split into vertices one block uses
//                    (updated in place by that block) and shared vertices
//                    (accumulated by atomics), with per-block descriptors,
//                    incidence lists in shared-memory positions, foreign-id
//                    lists and padded weights (flux), or row lists (SpMV).
#include <algorithm>
#include <climits>
#include <thread>

#include "internal.h"

namespace ep {
namespace {

// Endpoint pair of task e as data-vertex ids (bipartite: y_i -> n + i).
inline void task_ends(const HostSchedule& s, int64_t e, int32_t& u, int32_t& v) {
  const bool bip = (s.flags & 1u) != 0;
  u = bip ? (int32_t)(s.n + s.src[e]) : s.src[e];
  v = s.dst[e];
}

// Per-block first-touch vertex lists, computed block-parallel with one stamp
// array per worker, then concatenated.
void vertex_lists(HostSchedule& s, int threads) {
  const int64_t k = s.k;
  std::vector<int64_t> count(k, 0);
  std::vector<std::vector<int32_t>> chunks(threads);
  std::vector<int64_t> lo(threads + 1);
  for (int t = 0; t <= threads; ++t) lo[t] = k * t / threads;
  auto work = [&](int t) {
    std::vector<int32_t> stamp(s.nd, -1);
    auto& out = chunks[t];
    for (int64_t b = lo[t]; b < lo[t + 1]; ++b) {
      const int64_t before = (int64_t)out.size();
      for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
        int32_t u, v;
        task_ends(s, s.edge_perm[i], u, v);
        if (stamp[u] != (int32_t)b) {
          stamp[u] = (int32_t)b;
          out.push_back(u);
        }
        if (stamp[v] != (int32_t)b) {
          stamp[v] = (int32_t)b;
          out.push_back(v);
        }
      }
      count[b] = (int64_t)out.size() - before;
    }
  };
  if (threads == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
  }
  s.vert_ptr.assign(k + 1, 0);
  for (int64_t b = 0; b < k; ++b) s.vert_ptr[b + 1] = s.vert_ptr[b] + count[b];
  s.vert_list.clear();
  s.vert_list.reserve(s.vert_ptr[k]);
  for (auto& c : chunks) s.vert_list.insert(s.vert_list.end(), c.begin(), c.end());
  s.loads = s.vert_ptr[k];
}

void cpack(HostSchedule& s) {
  s.relabel.assign(s.nd, -1);
  int32_t next = 0;
  for (int32_t v : s.vert_list)
    if (s.relabel[v] < 0) s.relabel[v] = next++;
  s.touched = next;
  for (int64_t v = 0; v < s.nd; ++v)
    if (s.relabel[v] < 0) s.relabel[v] = next++;
}

// Number of blocks using each vertex (p_v) and the first such block.
void usage(const HostSchedule& s, std::vector<int32_t>& p, std::vector<int32_t>& owner) {
  p.assign(s.nd, 0);
  owner.assign(s.nd, -1);
  for (int64_t b = 0; b < s.k; ++b)
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      if (p[v]++ == 0) owner[v] = (int32_t)b;
    }
}

// In-block degree of every vertex of block b (tasks of b touching it).
void block_degrees(const HostSchedule& s, int64_t b, std::vector<int32_t>& deg) {
  for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
    int32_t u, v;
    task_ends(s, s.edge_perm[i], u, v);
    ++deg[u];
    if (v != u) ++deg[v];
  }
}

// The vertices of V_b satisfying `pick`, first-touch order, then stably
// sorted by descending in-block degree (so warps see similar list lengths).
template <typename Pick>
void class_order(const HostSchedule& s, int64_t b, const std::vector<int32_t>& deg, Pick pick,
                 std::vector<int32_t>& out) {
  out.clear();
  for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i)
    if (pick(s.vert_list[i])) out.push_back(s.vert_list[i]);
  std::stable_sort(out.begin(), out.end(), [&](int32_t a, int32_t c) { return deg[a] > deg[c]; });
}

std::string flux_layout_blocks(HostSchedule& s) {
  std::vector<int32_t> p, owner;
  usage(s, p, owner);
  s.rec_of.assign(s.nd, -1);
  s.fdesc.assign(s.k, FluxDesc{});
  std::vector<int32_t> deg(s.nd, 0), cls;
  // Every run starts on a multiple of 4 records (gap records stay unused), so
  // a run is a whole number of 16-byte chunks in every state plane.
  auto align4 = [](int32_t v) { return (v + 3) & ~3; };
  int32_t next = 0;
  for (int64_t b = 0; b < s.k; ++b) {
    block_degrees(s, b, deg);
    next = align4(next);
    s.fdesc[b].int_lo = next;
    class_order(s, b, deg, [&](int32_t v) { return owner[v] == b && p[v] == 1; }, cls);
    for (int32_t v : cls) s.rec_of[v] = next++;
    s.fdesc[b].n_int = next - s.fdesc[b].int_lo;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
  }
  next = align4(next);
  s.n_int = next;
  for (int64_t b = 0; b < s.k; ++b) {
    block_degrees(s, b, deg);
    next = align4(next);
    s.fdesc[b].bnd_lo = next;
    class_order(s, b, deg, [&](int32_t v) { return owner[v] == b && p[v] > 1; }, cls);
    for (int32_t v : cls) s.rec_of[v] = next++;
    s.fdesc[b].n_ob = next - s.fdesc[b].bnd_lo;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
  }
  next = align4(next);
  s.n_bnd = next - s.n_int;
  for (int64_t v = 0; v < s.nd; ++v)
    if (s.rec_of[v] < 0) s.rec_of[v] = next++;
  s.n_rec = align4(next);  // keeps every plane of a state buffer 16-byte aligned
  // shared-memory positions, foreign lists and per-position incidence lists
  s.flist.clear();
  s.inc.clear();
  s.ptr.clear();
  s.max_nv = 0;
  s.max_nent = 0;
  s.max_nf = 0;
  s.wmap.clear();
  auto pad_to = [](auto& v, size_t mult) {
    while (v.size() % mult) v.push_back(0);
  };
  std::vector<int32_t> pos(s.nd, -1);
  std::vector<int32_t> cnt;
  std::vector<uint32_t> ent;
  for (int64_t b = 0; b < s.k; ++b) {
    FluxDesc& d = s.fdesc[b];
    d.ne = (int32_t)(s.block_ptr[b + 1] - s.block_ptr[b]);
    while (s.wmap.size() % 4) s.wmap.push_back(-1);
    d.w0 = (int32_t)s.wmap.size();
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) s.wmap.push_back(s.edge_perm[i]);
    pad_to(s.flist, 4);
    d.f0 = (int32_t)s.flist.size();
    // runs are 4-aligned: positions [0, n_int), [pb, pb + n_ob), [pf, pf + nf)
    // with pb and pf rounded up to multiples of 4 (room for whole 16-byte chunks)
    d.pi = 0;
    d.pb = (d.n_int + 3) & ~3;
    d.pf = d.pb + ((d.n_ob + 3) & ~3);
    int32_t nf = 0;
    block_degrees(s, b, deg);
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      const int32_t r = s.rec_of[v];
      if (owner[v] == b) pos[v] = r < s.n_int ? d.pi + (r - d.int_lo) : d.pb + (r - d.bnd_lo);
    }
    class_order(s, b, deg, [&](int32_t v) { return owner[v] != b; }, cls);
    for (int32_t v : cls) {
      pos[v] = d.pf + nf++;
      s.flist.push_back(s.rec_of[v]);
    }
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
    d.nf = nf;
    s.max_nf = std::max(s.max_nf, nf);
    d.np = d.pf + nf;
    if (d.np > (int32_t)kPosMask + 1) return "block touches too many vertices";
    s.max_nv = std::max(s.max_nv, d.np);
    // incidence: every task appears at both endpoints (once for a self loop),
    // in task order within a position
    cnt.assign(d.np + 1, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      ++cnt[pos[u] + 1];
      if (v != u) ++cnt[pos[v] + 1];
    }
    for (int32_t p = 0; p < d.np; ++p) cnt[p + 1] += cnt[p];
    d.nent = cnt[d.np];
    pad_to(s.inc, 4);
    pad_to(s.ptr, 8);
    d.i0 = (int32_t)s.inc.size();
    d.q0 = (int32_t)s.ptr.size();
    for (int32_t p = 0; p <= d.np; ++p) s.ptr.push_back((uint16_t)cnt[p]);
    pad_to(s.ptr, 8);
    ent.assign(d.nent, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      const uint32_t j = (uint32_t)(i - s.block_ptr[b]) << kTaskShift;
      ent[cnt[pos[u]]++] = (uint32_t)pos[v] | j | kSrcBit;
      if (v != u) ent[cnt[pos[v]]++] = (uint32_t)pos[u] | j;
    }
    s.inc.insert(s.inc.end(), ent.begin(), ent.end());
    pad_to(s.inc, 4);
    s.max_nent = std::max(s.max_nent, d.nent);
    if (s.inc.size() >= (size_t)INT32_MAX || s.ptr.size() >= (size_t)INT32_MAX ||
        s.wmap.size() >= (size_t)INT32_MAX)
      return "schedule too large";
  }
  pad_to(s.flist, 4);
  while (s.wmap.size() % 4) s.wmap.push_back(-1);
  s.w_pad = (int64_t)s.wmap.size();
  return "";
}

// Kernel blocks of the flux layout.  A schedule block whose vertex set is
// far above the typical one (more than 3/2 of the median |V_b|) is cut in
// task order into halves, recursively, until every piece is within that
// size; each piece is then laid out as a block of its own (vertices shared
// by the pieces become shared vertices).  The schedule and its cost are
// unchanged; the kernels' shared-memory stages, sized for the largest kernel
// block, get smaller.  Returns false when no block needs cutting.
struct Pieces {
  int64_t k = 0;
  std::vector<int64_t> block_ptr, vert_ptr;
  std::vector<int32_t> vert_list;
};

bool cut_large_blocks(const HostSchedule& s, Pieces& out) {
  if (s.k < 2) return false;
  std::vector<int64_t> sz(s.k);
  for (int64_t b = 0; b < s.k; ++b) sz[b] = s.vert_ptr[b + 1] - s.vert_ptr[b];
  const int64_t biggest = *std::max_element(sz.begin(), sz.end());
  std::nth_element(sz.begin(), sz.begin() + s.k / 2, sz.end());
  const int64_t limit = std::max<int64_t>(64, sz[s.k / 2] * 3 / 2);
  if (biggest <= limit) return false;
  std::vector<int32_t> stamp(s.nd, -1);
  int32_t piece = 0;
  out.block_ptr.assign(1, 0);
  out.vert_ptr.assign(1, 0);
  out.vert_list.clear();
  // first-touch vertex list of tasks [lo, hi) appended to out.vert_list
  auto touch = [&](int64_t lo, int64_t hi) {
    const size_t before = out.vert_list.size();
    for (int64_t i = lo; i < hi; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      if (stamp[u] != piece) {
        stamp[u] = piece;
        out.vert_list.push_back(u);
      }
      if (stamp[v] != piece) {
        stamp[v] = piece;
        out.vert_list.push_back(v);
      }
    }
    return (int64_t)(out.vert_list.size() - before);
  };
  std::vector<std::pair<int64_t, int64_t>> todo;
  for (int64_t b = 0; b < s.k; ++b) {
    todo.assign(1, {s.block_ptr[b], s.block_ptr[b + 1]});
    while (!todo.empty()) {  // depth first, left half first: pieces stay in task order
      const auto [lo, hi] = todo.back();
      todo.pop_back();
      const size_t mark = out.vert_list.size();
      const int64_t nv = touch(lo, hi);
      if (nv > limit && hi - lo > 1) {
        out.vert_list.resize(mark);
        ++piece;  // fresh stamps for the halves
        const int64_t mid = lo + (hi - lo + 1) / 2;
        todo.push_back({mid, hi});
        todo.push_back({lo, mid});
        continue;
      }
      ++piece;
      out.block_ptr.push_back(hi);
      out.vert_ptr.push_back((int64_t)out.vert_list.size());
    }
  }
  out.k = (int64_t)out.block_ptr.size() - 1;
  return true;
}

std::string flux_layout(HostSchedule& s) {
  Pieces pc;
  const bool cut = cut_large_blocks(s, pc);
  if (cut) {
    std::swap(s.k, pc.k);
    s.block_ptr.swap(pc.block_ptr);
    s.vert_ptr.swap(pc.vert_ptr);
    s.vert_list.swap(pc.vert_list);
  }
  std::string err = flux_layout_blocks(s);
  if (cut) {  // the schedule itself is the uncut one
    std::swap(s.k, pc.k);
    s.block_ptr.swap(pc.block_ptr);
    s.vert_ptr.swap(pc.vert_ptr);
    s.vert_list.swap(pc.vert_list);
  }
  return err;
}

std::string spmv_layout(HostSchedule& s) {
  std::vector<int32_t> p, owner;
  usage(s, p, owner);
  const int32_t n = (int32_t)s.n;
  s.xrec_of.assign(n, -1);
  s.yrec_of.assign(n, -1);
  s.sdesc.assign(s.k, SpmvDesc{});
  std::vector<int32_t> deg(s.nd, 0), cls;
  // x records: cpack order restricted to columns
  int32_t nx = 0;
  for (int64_t b = 0; b < s.k; ++b) {
    SpmvDesc& d = s.sdesc[b];
    d.x_lo = nx;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      if (v < n && owner[v] == b) s.xrec_of[v] = nx++;
    }
    d.n_xo = nx - d.x_lo;
  }
  for (int32_t j = 0; j < n; ++j)
    if (s.xrec_of[j] < 0) s.xrec_of[j] = nx++;
  // y records: single-block rows first, then shared rows; longest lists first
  int32_t ny = 0;
  for (int64_t b = 0; b < s.k; ++b) {
    SpmvDesc& d = s.sdesc[b];
    block_degrees(s, b, deg);
    d.yi_lo = ny;
    class_order(s, b, deg, [&](int32_t v) { return v >= n && owner[v] == b && p[v] == 1; }, cls);
    for (int32_t v : cls) s.yrec_of[v - n] = ny++;
    d.n_yi = ny - d.yi_lo;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
  }
  s.ny_int = ny;
  for (int64_t b = 0; b < s.k; ++b) {
    SpmvDesc& d = s.sdesc[b];
    block_degrees(s, b, deg);
    d.yb_lo = ny;
    class_order(s, b, deg, [&](int32_t v) { return v >= n && owner[v] == b && p[v] > 1; }, cls);
    for (int32_t v : cls) s.yrec_of[v - n] = ny++;
    d.n_yob = ny - d.yb_lo;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
  }
  s.ny_bnd = ny - s.ny_int;
  for (int32_t i = 0; i < n; ++i)
    if (s.yrec_of[i] < 0) s.yrec_of[i] = ny++;
  s.xlist.clear();
  s.ylist.clear();
  s.sinc.clear();
  s.sptr.clear();
  s.wmap.clear();
  s.max_nx = s.max_ny = 0;
  s.max_nent = 0;
  std::vector<int32_t> pos(s.nd, -1), cnt;
  std::vector<uint32_t> ent;
  for (int64_t b = 0; b < s.k; ++b) {
    SpmvDesc& d = s.sdesc[b];
    d.ne = (int32_t)(s.block_ptr[b + 1] - s.block_ptr[b]);
    while (s.wmap.size() % 4) s.wmap.push_back(-1);
    d.w0 = (int32_t)s.wmap.size();
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) s.wmap.push_back(s.edge_perm[i]);
    d.fx0 = (int32_t)s.xlist.size();
    d.fy0 = (int32_t)s.ylist.size();
    int32_t nxf = 0;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      if (v >= n) continue;
      if (owner[v] == b)
        pos[v] = s.xrec_of[v] - d.x_lo;
      else {
        pos[v] = d.n_xo + nxf++;
        s.xlist.push_back(s.xrec_of[v]);
      }
    }
    d.n_xf = nxf;
    block_degrees(s, b, deg);
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      if (v < n || owner[v] != b) continue;
      const int32_t r = s.yrec_of[v - n];
      pos[v] = r < s.ny_int ? r - d.yi_lo : d.n_yi + (r - d.yb_lo);
    }
    class_order(s, b, deg, [&](int32_t v) { return v >= n && owner[v] != b; }, cls);
    int32_t nyf = 0;
    for (int32_t v : cls) {
      pos[v] = d.n_yi + d.n_yob + nyf++;
      s.ylist.push_back(s.yrec_of[v - n]);
    }
    d.n_yf = nyf;
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
    const int32_t nxs = d.n_xo + nxf, nys = d.n_yi + d.n_yob + nyf;
    if (nxs > (int32_t)kPosMask + 1 || nys > 65535) return "block touches too many vertices";
    s.max_nx = std::max(s.max_nx, nxs);
    s.max_ny = std::max(s.max_ny, nys);
    // row lists: (x position) | (task << 15), tasks in schedule order
    cnt.assign(nys + 1, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      ++cnt[pos[u] + 1];
    }
    for (int32_t q = 0; q < nys; ++q) cnt[q + 1] += cnt[q];
    d.i0 = (int32_t)s.sinc.size();
    d.q0 = (int32_t)s.sptr.size();
    for (int32_t q = 0; q <= nys; ++q) s.sptr.push_back((uint16_t)cnt[q]);
    ent.assign(d.ne, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      ent[cnt[pos[u]]++] = (uint32_t)pos[v] | ((uint32_t)(i - s.block_ptr[b]) << kTaskShift);
    }
    s.sinc.insert(s.sinc.end(), ent.begin(), ent.end());
    s.max_nent = std::max(s.max_nent, d.ne);
    if (s.sinc.size() >= (size_t)INT32_MAX) return "schedule too large";
  }
  while (s.wmap.size() % 4) s.wmap.push_back(-1);
  s.w_pad = (int64_t)s.wmap.size();
  return "";
}

}  // namespace

std::string build_schedule(HostSchedule& s, int threads) {
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, s.k));
  // reconstruction (Definition 4): counting sort by block keeps ascending ids
  s.block_ptr.assign(s.k + 1, 0);
  for (int64_t e = 0; e < s.m; ++e) ++s.block_ptr[s.part[e] + 1];
  s.max_ne = 0;
  for (int64_t b = 0; b < s.k; ++b) {
    s.max_ne = std::max<int32_t>(s.max_ne, (int32_t)s.block_ptr[b + 1]);
    s.block_ptr[b + 1] += s.block_ptr[b];
  }
  s.edge_perm.assign(s.m, 0);
  {
    std::vector<int64_t> cur(s.block_ptr.begin(), s.block_ptr.end() - 1);
    for (int64_t e = 0; e < s.m; ++e) s.edge_perm[cur[s.part[e]]++] = (int32_t)e;
  }
  vertex_lists(s, threads);
  cpack(s);
  return (s.flags & 1u) ? spmv_layout(s) : flux_layout(s);
}

}  // namespace ep
