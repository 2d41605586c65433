// schedule.cpp -- from a task partition to the arrays the kernels use.
//
//   reconstruction   tasks grouped by block, ascending id inside a block
//                    (Definition 4);
//   vertex lists     distinct data vertices of each block in first-touch
//                    order (the block's share of the data, Section 4 Fig. 7);
//   cpack            ids in order of first appearance over blocks (Section
//                    4.1, after Ding and Kennedy), untouched vertices last;
//   cost             loads = sum_b |V_b|, vertex cut = loads - touched (Eq. 1);
//   kernel layout    flux: one contiguous record run per kernel block with
//                    the vertices only that block uses (updated in place)
//                    followed by its own copies of the shared vertices
//                    (accumulated by atomics, refreshed by the fold), the
//                    incidence in sliced-ELL slots with one weight per slot,
//                    and the copy lists of the shared vertices; SpMV: row
//                    lists over x records staged by owner and foreign ids.
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

struct SlotEntry {
  int32_t o;  // the other position
  int32_t e;  // task
  bool src;   // source side of the task (owns its weight-gradient element)
};

// Places the entries of slice j (positions 32 j + l, l < 32) in its columns.
// Column by column, each lane takes one of its remaining entries so that the
// 32 lanes read their other positions from different shared-memory banks as
// far as the lists allow: different (o mod 8) within each group of 8 lanes
// (a 16-byte load is served 8 lanes at a time, 4 banks each) and different
// (o mod 32) over the slice (4-byte loads).  A lane with fewer entries than
// columns leaves slots unused; an unused slot has weight 0, so its term is
// exactly zero whatever position it names, and it takes a free bank too.
void place_slice(HostSchedule& s, const FluxDesc& d, int32_t j, const std::vector<int32_t>& ent_ptr,
                 std::vector<SlotEntry>& ents) {
  const int32_t c0 = s.soff[d.q0 + j], K = s.soff[d.q0 + j + 1] - c0;
  int32_t lo[32], hi[32];
  for (int l = 0; l < 32; ++l) {
    const int32_t p = 32 * j + l;
    lo[l] = p < d.nv ? ent_ptr[p] : 0;
    hi[l] = p < d.nv ? ent_ptr[p + 1] : 0;
  }
  const int32_t npad = std::min(d.nv, 32);  // unused slots name one of the first 32 positions
  for (int32_t c = 0; c < K; ++c) {
    uint32_t used32 = 0;
    uint32_t used8[4] = {0, 0, 0, 0};
    auto score = [&](int l, int32_t o) {
      return 2 * (int)((used8[l >> 3] >> (o & 7)) & 1u) + (int)((used32 >> (o & 31)) & 1u);
    };
    // lanes that must place an entry in every remaining column go first
    uint32_t forced_mask = 0;
    for (int l = 0; l < 32; ++l)
      if (hi[l] - lo[l] == K - c) forced_mask |= 1u << l;
    for (int pass = 0; pass < 2; ++pass)
      for (int l = 0; l < 32; ++l) {
        const int32_t rem = hi[l] - lo[l];
        const bool forced = (forced_mask >> l) & 1u;
        if ((pass == 0) != forced) continue;
        int32_t best = -1, bs = 4;
        for (int32_t i = lo[l]; i < hi[l] && bs > 0; ++i) {
          const int sc = score(l, ents[i].o);
          if (sc < bs) best = i, bs = sc;
        }
        int32_t pad = 0, ps = 4;
        if (!forced)
          for (int32_t o = 0; o < npad && ps > 0; ++o) {
            const int sc = score(l, o);
            if (sc < ps) pad = o, ps = sc;
          }
        const int64_t slot = (int64_t)d.s0 + 32 * ((int64_t)c0 + c) + l;
        int32_t o;
        if (rem > 0 && (forced || bs <= ps)) {
          std::swap(ents[lo[l]], ents[best]);
          const SlotEntry& t = ents[lo[l]++];
          o = t.o;
          s.sidx[slot] = (uint16_t)((uint32_t)t.o | (t.src ? kSlotSrc : 0u));
          s.wmap[slot] = t.e;
          if (t.src) s.gslot[t.e] = (int32_t)slot;
        } else {
          o = pad;
          s.sidx[slot] = (uint16_t)pad;  // weight slot stays -1: weight 0
        }
        used8[l >> 3] |= 1u << (o & 7);
        used32 |= 1u << (o & 31);
      }
  }
}

std::string flux_layout_blocks(HostSchedule& s) {
  std::vector<int32_t> p, owner;
  usage(s, p, owner);
  // halo vertices of a shard (touched by other shards' tasks too) take the
  // shared path even when one block here uses them: their sums must go
  // through an accumulator that the exchange can reach
  for (int32_t v : s.halo)
    if (v >= 0 && v < s.nd && p[v] == 1) p[v] = 2;
  auto align4 = [](int64_t v) { return (v + 3) & ~(int64_t)3; };
  auto pad_to = [](auto& v, size_t mult, auto fill) {
    while (v.size() % mult) v.push_back(fill);
  };
  // shared ids in order of first appearance over the kernel blocks
  std::vector<int32_t> sid(s.nd, -1);
  int64_t n_sh = 0;
  for (int64_t b = 0; b < s.k; ++b)
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) {
      const int32_t v = s.vert_list[i];
      if (p[v] > 1 && sid[v] < 0) sid[v] = (int32_t)n_sh++;
    }
  s.n_sh = n_sh;
  s.fdesc.assign(s.k, FluxDesc{});
  s.rec_of.assign(s.nd, -1);
  s.sid_list.clear();
  s.sidx.clear();
  s.soff.clear();
  s.wmap.clear();
  s.gslot.assign(s.m, -1);
  s.max_nv = s.max_nslot = s.max_nsh = s.max_nsl = 0;
  std::vector<std::vector<int32_t>> copies(n_sh);
  std::vector<int32_t> deg(s.nd, 0), ord, pos(s.nd, -1), cls, col, ent_ptr;
  std::vector<SlotEntry> ents;
  int64_t next = 0;  // next free record
  for (int64_t b = 0; b < s.k; ++b) {
    FluxDesc& d = s.fdesc[b];
    d.ne = (int32_t)(s.block_ptr[b + 1] - s.block_ptr[b]);
    block_degrees(s, b, deg);
    // positions: interior vertices, then shared ones, each by descending degree
    class_order(s, b, deg, [&](int32_t v) { return p[v] == 1; }, ord);
    d.ni = (int32_t)ord.size();
    class_order(s, b, deg, [&](int32_t v) { return p[v] > 1; }, cls);
    ord.insert(ord.end(), cls.begin(), cls.end());
    d.nv = (int32_t)ord.size();
    if (d.nv > (int32_t)kSlotPos) return "block touches too many vertices";
    next = align4(next);
    d.rec_lo = (int32_t)next;
    for (int32_t q = 0; q < d.nv; ++q) {
      const int32_t v = ord[q];
      pos[v] = q;
      const int32_t r = (int32_t)(next + q);
      if (owner[v] == b) s.rec_of[v] = r;  // first copy of a shared vertex
      if (q >= d.ni) copies[sid[v]].push_back(r);
    }
    next += d.nv;
    // shared ids of positions [ni, nv); the first copy of each shared vertex
    // (in its first block) carries kSidFirst
    pad_to(s.sid_list, 4, (int32_t)0);
    d.h0 = (int32_t)s.sid_list.size();
    for (int32_t q = d.ni; q < d.nv; ++q)
      s.sid_list.push_back(sid[ord[q]] | (owner[ord[q]] == b ? kSidFirst : 0));
    pad_to(s.sid_list, 4, (int32_t)0);
    // slices of 32 positions; columns = largest degree in the slice
    d.nsl = (d.nv + 31) / 32;
    pad_to(s.soff, 8, (uint16_t)0);
    d.q0 = (int32_t)s.soff.size();
    int32_t cols = 0;
    s.soff.push_back(0);
    for (int32_t j = 0; j < d.nsl; ++j) {
      int32_t K = 0;
      for (int32_t q = 32 * j; q < std::min(d.nv, 32 * j + 32); ++q) K = std::max(K, deg[ord[q]]);
      cols += K;
      if (cols > 0xffff) return "block has too many incidence entries";
      s.soff.push_back((uint16_t)cols);
    }
    pad_to(s.soff, 8, (uint16_t)0);
    d.s0 = (int32_t)s.sidx.size();  // a multiple of 32
    d.nslot = 32 * cols;
    s.sidx.resize(s.sidx.size() + d.nslot, 0);
    s.wmap.resize(s.sidx.size(), -1);
    // the entries of every position: each task at both endpoints (a self
    // loop once), the source side flagged
    ent_ptr.assign(d.nv + 1, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      ++ent_ptr[pos[u] + 1];
      if (v != u) ++ent_ptr[pos[v] + 1];
    }
    for (int32_t q = 0; q < d.nv; ++q) ent_ptr[q + 1] += ent_ptr[q];
    ents.resize(ent_ptr[d.nv]);
    col.assign(ent_ptr.begin(), ent_ptr.end() - 1);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      const int32_t e = s.edge_perm[i];
      int32_t u, v;
      task_ends(s, e, u, v);
      const int32_t pu = pos[u], pv = pos[v];
      ents[col[pu]++] = SlotEntry{pv, e, true};
      if (v != u) ents[col[pv]++] = SlotEntry{pu, e, false};
    }
    for (int32_t j = 0; j < d.nsl; ++j) place_slice(s, d, j, ent_ptr, ents);
    for (int64_t i = s.vert_ptr[b]; i < s.vert_ptr[b + 1]; ++i) deg[s.vert_list[i]] = 0;
    s.max_nv = std::max(s.max_nv, d.nv);
    s.max_nslot = std::max(s.max_nslot, d.nslot);
    s.max_nsh = std::max(s.max_nsh, d.nv - d.ni);
    s.max_nsl = std::max(s.max_nsl, d.nsl);
    if (s.sidx.size() >= (size_t)INT32_MAX || next >= INT32_MAX / 2) return "schedule too large";
  }
  s.n_run = align4(next);
  next = s.n_run;
  for (int64_t v = 0; v < s.nd; ++v)
    if (s.rec_of[v] < 0) s.rec_of[v] = (int32_t)next++;  // untouched vertices
  s.n_rec = align4(next);  // keeps every plane of a state buffer 16-byte aligned
  s.vrec.assign(s.n_rec, -1);
  for (int64_t v = 0; v < s.nd; ++v) s.vrec[s.rec_of[v]] = (int32_t)v;
  // the fold's work list: every copy in record order (block runs in order)
  s.fold_rec.clear();
  s.fold_sid.clear();
  for (int64_t b = 0; b < s.k; ++b) {
    const FluxDesc& d = s.fdesc[b];
    for (int32_t q = d.ni; q < d.nv; ++q) {
      s.fold_rec.push_back(d.rec_lo + q);
      s.fold_sid.push_back(s.sid_list[d.h0 + q - d.ni]);
    }
  }
  s.cptr.assign(n_sh + 1, 0);
  s.crec.clear();
  s.crec.reserve(s.vert_ptr.back());
  for (int64_t h = 0; h < n_sh; ++h) {
    s.crec.insert(s.crec.end(), copies[h].begin(), copies[h].end());
    s.cptr[h + 1] = (int32_t)s.crec.size();
  }
  for (int64_t v = 0; v < s.nd; ++v)  // every copy of a shared vertex maps back to it
    if (sid[v] >= 0)
      for (int32_t c = s.cptr[sid[v]]; c < s.cptr[sid[v] + 1]; ++c) s.vrec[s.crec[c]] = (int32_t)v;
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
  s.sent.clear();
  s.wmap.clear();
  s.max_nx = s.max_ny = s.max_nxy = 0;
  std::vector<int32_t> pos(s.nd, -1), cnt;
  // one entry run of 32 * u slots per block (u from the largest block), so
  // that block b's run starts at slot 32 * u * b
  int64_t big = 0;
  for (int64_t b = 0; b < s.k; ++b) big = std::max(big, s.block_ptr[b + 1] - s.block_ptr[b]);
  s.spmv_u = (int32_t)(((big + 31) / 32 + 3) / 4 * 4);
  for (int64_t b = 0; b < s.k; ++b) {
    SpmvDesc& d = s.sdesc[b];
    d.ne = (int32_t)(s.block_ptr[b + 1] - s.block_ptr[b]);
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
    if (nxs > (int32_t)kColMask + 1 || nys > (int32_t)kColMask + 1)
      return "block touches too many vertices";
    s.max_nx = std::max(s.max_nx, nxs);
    s.max_ny = std::max(s.max_ny, nys);
    s.max_nxy = std::max(s.max_nxy, ((nxs + 3) & ~3) + ((nys + 3) & ~3));
    // entries sorted by row position (a counting sort; schedule order within
    // a row), each lane of the kernel's warp taking u consecutive ones
    cnt.assign(nys + 1, 0);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      ++cnt[pos[u] + 1];
    }
    for (int32_t q = 0; q < nys; ++q) cnt[q + 1] += cnt[q];
    d.u = s.spmv_u;
    d.i0 = (int32_t)s.sent.size();
    const size_t run = (size_t)32 * d.u;
    s.sent.resize(d.i0 + run, 0u);
    s.wmap.resize(d.i0 + run, -1);
    for (int64_t i = s.block_ptr[b]; i < s.block_ptr[b + 1]; ++i) {
      int32_t u, v;
      task_ends(s, s.edge_perm[i], u, v);
      const int32_t t = cnt[pos[u]]++;  // rank in row order
      const int32_t j = d.i0 + spmv_slot(t, d.u);
      s.sent[j] = ((uint32_t)pos[u] << kRowShift) | (uint32_t)pos[v];
      s.wmap[j] = s.edge_perm[i];
    }
    if (s.sent.size() >= (size_t)INT32_MAX) return "schedule too large";
  }
  s.w_pad = (int64_t)s.wmap.size();
  return "";
}

}  // namespace

std::string rebuild_flux_layout(HostSchedule& s) { return flux_layout(s); }

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
