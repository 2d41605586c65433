// partition.cpp -- host side of the edge partition (Section 3.2).
//
// Builds the clone-and-connect graph with contracted original edges
// (Definition 3; the "very large weight" on original edges read as
// contraction), partitions it by multilevel recursive bisection into
// k = ceil(m/C) blocks of exactly C tasks (the last block takes the rest),
// and reconstructs the edge partition (Definition 4).  The paper hands the
// vertex partition to METIS; this library fixes its own deterministic rules
// instead, so the schedule does not depend on thread count or timing:
//   coarsening   heavy-edge matching in ascending vertex order, ties to the
//                smaller neighbour, combined weight <= max(1, min(sL,W-sL)/16),
//                while n > 64 and each level shrinks by >= 10%; a level whose
//                adjacency shrank by < 15% is kept but ends the coarsening;
//   initial cut  graph growing from the last vertex of a BFS from vertex 0;
//   refinement   4 passes of positive-gain moves in (gain desc, id asc) order
//                under the balance window max(tol, |lw - sL|),
//                tol = max(1, min(sL, W-sL)/32);
//   exact size   best-gain moves off the heavy side at the finest level.
// Recursion subtrees run on separate host threads.
#include "internal.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>

namespace ep {
namespace {

constexpr int32_t kCoarsenMin = 64;
constexpr int kPasses = 4;
constexpr int32_t kParallelMin = 1 << 20;  // graphs this large split loops over host threads

// fn(lo, hi, t) over [0, n) in `parts` contiguous ranges (part t = [lo, hi)).
template <typename Fn>
void for_ranges(int64_t n, int parts, Fn fn) {
  if (parts <= 1) {
    fn((int64_t)0, n, 0);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < parts; ++t)
    pool.emplace_back([&, t]() { fn(n * t / parts, n * (t + 1) / parts, t); });
  for (auto& th : pool) th.join();
}

int loop_parts(int64_t n) {
  if (n < kParallelMin) return 1;
  return (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
}

struct Graph {
  int32_t n = 0;
  std::vector<int64_t> xadj;  // n+1
  std::vector<int32_t> adj;   // ascending per row
  std::vector<int32_t> ew;
  std::vector<int32_t> vw;
};

// ---------------------------------------------------------------- H build

// Incidence lists by counting sort, auxiliary pairs per data vertex, then one
// row per task merged through a stamp table.
void build_h(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, bool bip, Graph& H) {
  const int64_t nd = bip ? 2 * n : n;
  auto ends = [&](int64_t e, int64_t& u, int64_t& v) {
    u = bip ? n + src[e] : src[e];
    v = dst[e];
  };
  std::vector<int64_t> start(nd + 1, 0);
  for (int64_t e = 0; e < m; ++e) {
    int64_t u, v;
    ends(e, u, v);
    ++start[u + 1];
    if (v != u) ++start[v + 1];
  }
  for (int64_t v = 0; v < nd; ++v) start[v + 1] += start[v];
  std::vector<int32_t> inc(start[nd]);
  {
    std::vector<int64_t> cur(start.begin(), start.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
      int64_t u, v;
      ends(e, u, v);
      inc[cur[u]++] = (int32_t)e;
      if (v != u) inc[cur[v]++] = (int32_t)e;
    }
  }
  // row lengths of H before merging: each task has <= 2 path neighbours per endpoint
  std::vector<int64_t> rowcnt(m + 1, 0);
  for (int64_t v = 0; v < nd; ++v)
    for (int64_t i = start[v]; i + 1 < start[v + 1]; ++i) {
      ++rowcnt[inc[i] + 1];
      ++rowcnt[inc[i + 1] + 1];
    }
  for (int64_t e = 0; e < m; ++e) rowcnt[e + 1] += rowcnt[e];
  std::vector<int32_t> raw(rowcnt[m]);
  {
    std::vector<int64_t> cur(rowcnt.begin(), rowcnt.end() - 1);
    for (int64_t v = 0; v < nd; ++v)
      for (int64_t i = start[v]; i + 1 < start[v + 1]; ++i) {
        raw[cur[inc[i]]++] = inc[i + 1];
        raw[cur[inc[i + 1]]++] = inc[i];
      }
  }
  H.n = (int32_t)m;
  H.xadj.assign(m + 1, 0);
  H.adj.clear();
  H.ew.clear();
  H.adj.reserve(raw.size());
  H.ew.reserve(raw.size());
  H.vw.assign(m, 1);
  for (int64_t e = 0; e < m; ++e) {
    int32_t* b = raw.data() + rowcnt[e];
    int32_t* t = raw.data() + rowcnt[e + 1];
    std::sort(b, t);
    for (int32_t* p = b; p < t;) {
      int32_t* q = p;
      while (q < t && *q == *p) ++q;
      H.adj.push_back(*p);
      H.ew.push_back((int32_t)(q - p));
      p = q;
    }
    H.xadj[e + 1] = (int64_t)H.adj.size();
  }
}

// -------------------------------------------------------------- coarsening

// Returns the coarse vertex count; cmap[u] = coarse id, lead[c] = smaller
// member, other[c] = partner or -1.
int32_t heavy_edge_matching(const Graph& g, int32_t maxw, std::vector<int32_t>& cmap,
                            std::vector<int32_t>& lead, std::vector<int32_t>& other) {
  const int32_t n = g.n;
  cmap.assign(n, -1);
  lead.clear();
  other.clear();
  for (int32_t u = 0; u < n; ++u) {
    if (cmap[u] >= 0) continue;
    int32_t pick = -1, pw = 0;
    for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j) {
      const int32_t v = g.adj[j];
      if (cmap[v] >= 0 || v == u) continue;
      if ((int64_t)g.vw[u] + g.vw[v] > maxw) continue;
      // rows are ascending, so the first maximum is the smallest id
      if (pick < 0 || g.ew[j] > pw) {
        pick = v;
        pw = g.ew[j];
      }
    }
    const int32_t c = (int32_t)lead.size();
    cmap[u] = c;
    lead.push_back(u);
    other.push_back(pick);
    if (pick >= 0) cmap[pick] = c;
  }
  return (int32_t)lead.size();
}

// Coarse graph: the row of a coarse vertex is the union of its members' rows
// mapped to coarse ids, without the coarse vertex itself, parallel entries
// merged by summing weights, ascending.  Rows are built independently
// (ranges of coarse vertices on host threads for large graphs) and joined.
void contract(const Graph& g, const std::vector<int32_t>& cmap, const std::vector<int32_t>& lead,
              const std::vector<int32_t>& other, Graph& cg) {
  const int32_t nc = (int32_t)lead.size();
  cg.n = nc;
  cg.xadj.assign(nc + 1, 0);
  cg.vw.assign(nc, 0);
  const int parts = loop_parts(nc);
  std::vector<std::vector<int32_t>> padj(parts), pew(parts);
  for_ranges(nc, parts, [&](int64_t lo, int64_t hi, int t) {
    std::vector<std::pair<int32_t, int32_t>> row;
    auto& oa = padj[t];
    auto& ow = pew[t];
    for (int64_t c = lo; c < hi; ++c) {
      row.clear();
      const int32_t mem[2] = {lead[c], other[c]};
      int32_t w = 0;
      for (int i = 0; i < 2; ++i) {
        const int32_t x = mem[i];
        if (x < 0) continue;
        w += g.vw[x];
        for (int64_t j = g.xadj[x]; j < g.xadj[x + 1]; ++j) {
          const int32_t cv = cmap[g.adj[j]];
          if (cv != (int32_t)c) row.emplace_back(cv, g.ew[j]);
        }
      }
      cg.vw[c] = w;
      std::sort(row.begin(), row.end());
      int32_t len = 0;
      for (size_t i = 0; i < row.size();) {
        size_t j = i;
        int32_t sum = 0;
        while (j < row.size() && row[j].first == row[i].first) sum += row[j++].second;
        oa.push_back(row[i].first);
        ow.push_back(sum);
        ++len;
        i = j;
      }
      cg.xadj[c + 1] = len;
    }
  });
  for (int32_t c = 0; c < nc; ++c) cg.xadj[c + 1] += cg.xadj[c];
  cg.adj.resize(cg.xadj[nc]);
  cg.ew.resize(cg.xadj[nc]);
  for_ranges(parts, parts, [&](int64_t lo, int64_t, int t) {
    const int64_t at = cg.xadj[(int64_t)nc * lo / parts];
    std::copy(padj[t].begin(), padj[t].end(), cg.adj.begin() + at);
    std::copy(pew[t].begin(), pew[t].end(), cg.ew.begin() + at);
  });
}

// -------------------------------------------------------- initial bisection

void initial_cut(const Graph& g, int64_t sL, std::vector<uint8_t>& side) {
  const int32_t n = g.n;
  std::vector<int32_t> q;
  q.reserve(n);
  std::vector<uint8_t> seen(n, 0);
  q.push_back(0);
  seen[0] = 1;
  for (size_t h = 0; h < q.size(); ++h) {
    const int32_t u = q[h];
    for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j)
      if (!seen[g.adj[j]]) {
        seen[g.adj[j]] = 1;
        q.push_back(g.adj[j]);
      }
  }
  const int32_t root = q.back();
  std::fill(seen.begin(), seen.end(), 0);
  side.assign(n, 1);
  q.clear();
  q.push_back(root);
  seen[root] = 1;
  size_t h = 0;
  int32_t next_unseen = 0;
  int64_t lw = 0;
  while (lw < sL) {
    if (h == q.size()) {
      while (next_unseen < n && seen[next_unseen]) ++next_unseen;
      if (next_unseen == n) break;
      seen[next_unseen] = 1;
      q.push_back(next_unseen);
    }
    const int32_t u = q[h++];
    if (lw + g.vw[u] > sL) continue;
    side[u] = 0;
    lw += g.vw[u];
    for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j)
      if (!seen[g.adj[j]]) {
        seen[g.adj[j]] = 1;
        q.push_back(g.adj[j]);
      }
  }
}

// -------------------------------------------------------------- refinement

inline int64_t iabs(int64_t a) { return a < 0 ? -a : a; }

void gains_of(const Graph& g, const std::vector<uint8_t>& side, std::vector<int64_t>& gain) {
  gain.resize(g.n);
  for_ranges(g.n, loop_parts(g.n), [&](int64_t lo, int64_t hi, int) {
    for (int64_t u = lo; u < hi; ++u) {
      int64_t ext = 0, in = 0;
      for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j)
        (side[g.adj[j]] == side[u] ? in : ext) += g.ew[j];
      gain[u] = ext - in;
    }
  });
}

void flip(const Graph& g, std::vector<uint8_t>& side, std::vector<int64_t>& gain, int32_t u) {
  side[u] = (uint8_t)(1 - side[u]);
  gain[u] = -gain[u];
  for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j) {
    const int32_t x = g.adj[j];
    gain[x] += (side[x] == side[u] ? -2 : 2) * (int64_t)g.ew[j];
  }
}

void refine_level(const Graph& g, int64_t sL, int64_t W, std::vector<uint8_t>& side) {
  const int64_t tol = std::max<int64_t>(1, std::min(sL, W - sL) / 32);
  int64_t lw = 0;
  for (int32_t u = 0; u < g.n; ++u)
    if (!side[u]) lw += g.vw[u];
  std::vector<int64_t> gain;
  std::vector<int32_t> order;
  gains_of(g, side, gain);  // kept exact by flip() across passes
  for (int pass = 0; pass < kPasses; ++pass) {
    order.clear();
    for (int32_t u = 0; u < g.n; ++u)
      if (gain[u] > 0) order.push_back(u);
    std::vector<int64_t> g0(gain);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return g0[a] != g0[b] ? g0[a] > g0[b] : a < b;
    });
    int moves = 0;
    for (int32_t u : order) {
      if (gain[u] <= 0) continue;
      const int64_t nl = side[u] ? lw + g.vw[u] : lw - g.vw[u];
      if (iabs(nl - sL) > std::max(tol, iabs(lw - sL))) continue;
      flip(g, side, gain, u);
      lw = nl;
      ++moves;
    }
    if (!moves) break;
  }
}

// Exact balance at the finest level: a heap of (gain, -id) over the heavy
// side, built in linear time and updated lazily (a vertex's gain only grows
// while its neighbours leave, so older entries are recognisable as stale).
void exact_balance(const Graph& g, int64_t sL, std::vector<uint8_t>& side) {
  int64_t lw = 0;
  for (int32_t u = 0; u < g.n; ++u)
    if (!side[u]) lw += g.vw[u];
  if (lw == sL) return;
  const uint8_t heavy = lw > sL ? 0 : 1;
  std::vector<int64_t> gain;
  gains_of(g, side, gain);
  using Item = std::pair<int64_t, int32_t>;  // (gain, -id): larger is better
  std::vector<Item> heap;
  heap.reserve((size_t)g.n);
  for (int32_t u = 0; u < g.n; ++u)
    if (side[u] == heavy) heap.emplace_back(gain[u], -u);
  std::make_heap(heap.begin(), heap.end());
  while (lw != sL && !heap.empty()) {
    std::pop_heap(heap.begin(), heap.end());
    const Item top = heap.back();
    heap.pop_back();
    const int32_t u = -top.second;
    if (side[u] != heavy || top.first != gain[u]) continue;  // stale
    flip(g, side, gain, u);
    for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j) {
      const int32_t x = g.adj[j];
      if (side[x] == heavy) {
        heap.emplace_back(gain[x], -x);
        std::push_heap(heap.begin(), heap.end());
      }
    }
    lw += heavy ? 1 : -1;
  }
}

bool stopped(const std::atomic<int>* stop) {
  return stop && stop->load(std::memory_order_relaxed) != 0;
}

// Leaves `side` unfinished when `stop` is raised (the caller checks it too).
void bisect(const Graph& g0, int64_t sL, std::vector<uint8_t>& side, const std::atomic<int>* stop) {
  const int64_t W = g0.n;
  const int32_t maxw = (int32_t)std::max<int64_t>(1, std::min(sL, W - sL) / 16);
  std::vector<Graph> levels;  // coarse levels 1..L
  std::vector<std::vector<int32_t>> maps;
  const Graph* cur = &g0;
  std::vector<int32_t> cmap, lead, other;
  while (cur->n > kCoarsenMin && levels.size() < 63) {
    if (stopped(stop)) return;
    const int32_t nc = heavy_edge_matching(*cur, maxw, cmap, lead, other);
    if ((int64_t)nc * 10 > (int64_t)cur->n * 9) break;
    Graph cg;
    contract(*cur, cmap, lead, other, cg);
    const bool dense = (int64_t)cg.adj.size() * 20 > (int64_t)cur->adj.size() * 17;
    maps.push_back(cmap);
    levels.push_back(std::move(cg));
    cur = &levels.back();
    if (dense) break;  // the adjacency shrank by less than 15%: stop coarsening
  }
  initial_cut(*cur, sL, side);
  refine_level(*cur, sL, W, side);
  for (int l = (int)levels.size() - 1; l >= 0; --l) {
    if (stopped(stop)) return;
    const Graph& fine = l == 0 ? g0 : levels[l - 1];
    std::vector<uint8_t> fs(fine.n);
    for (int32_t u = 0; u < fine.n; ++u) fs[u] = side[maps[l][u]];
    side.swap(fs);
    refine_level(fine, sL, W, side);
  }
  exact_balance(g0, sL, side);
}

void split(const Graph& g, const std::vector<int32_t>& gid, const std::vector<uint8_t>& side,
           uint8_t s, Graph& sg, std::vector<int32_t>& sgid) {
  std::vector<int32_t> loc(g.n, -1);
  int32_t cnt = 0;
  for (int32_t u = 0; u < g.n; ++u)
    if (side[u] == s) loc[u] = cnt++;
  sg.n = cnt;
  sg.xadj.assign(cnt + 1, 0);
  sg.vw.assign(cnt, 1);
  sg.adj.clear();
  sg.ew.clear();
  sgid.resize(cnt);
  for (int32_t u = 0; u < g.n; ++u) {
    const int32_t lu = loc[u];
    if (lu < 0) continue;
    sgid[lu] = gid[u];
    for (int64_t j = g.xadj[u]; j < g.xadj[u + 1]; ++j) {
      const int32_t lv = loc[g.adj[j]];
      if (lv < 0) continue;
      sg.adj.push_back(lv);
      sg.ew.push_back(g.ew[j]);
    }
    sg.xadj[lu + 1] = (int64_t)sg.adj.size();
  }
}

struct Recursion {
  int32_t C;
  int32_t* part;
  std::atomic<int> spare;  // threads that may still be started
  const std::atomic<int>* stop;  // cancellation request (nullable)
};

constexpr int32_t kSpawnMin = 4096;  // do not start a thread for smaller subtrees

void recurse(Graph g, std::vector<int32_t> gid, int32_t kk, int32_t first, Recursion& R) {
  if (stopped(R.stop)) return;
  if (kk == 1) {
    for (int32_t x : gid) R.part[x] = first;
    return;
  }
  const int32_t kL = (kk + 1) / 2;
  std::vector<uint8_t> side;
  bisect(g, (int64_t)kL * R.C, side, R.stop);
  if (stopped(R.stop)) return;
  Graph gl, gr;
  std::vector<int32_t> il, ir;
  split(g, gid, side, 0, gl, il);
  split(g, gid, side, 1, gr, ir);
  g = Graph();
  gid.clear();
  gid.shrink_to_fit();
  bool spawn = false;
  if (gl.n >= kSpawnMin) {
    int s = R.spare.load();
    while (s > 0 && !(spawn = R.spare.compare_exchange_weak(s, s - 1))) {
    }
  }
  if (spawn) {
    std::thread t([&]() { recurse(std::move(gl), std::move(il), kL, first, R); });
    recurse(std::move(gr), std::move(ir), kk - kL, first + kL, R);
    t.join();
    R.spare.fetch_add(1);
  } else {
    recurse(std::move(gl), std::move(il), kL, first, R);
    recurse(std::move(gr), std::move(ir), kk - kL, first + kL, R);
  }
}

}  // namespace

bool partition_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                     uint32_t flags, int threads, int32_t* part, const std::atomic<int>* stop) {
  const int32_t k = (int32_t)((m + C - 1) / C);
  if ((flags & 2u) || k == 1) {
    for (int64_t e = 0; e < m; ++e) part[e] = (int32_t)(e / C);
    return true;
  }
  Graph H;
  build_h(src, dst, m, n, (flags & 1u) != 0, H);
  std::vector<int32_t> gid(m);
  for (int64_t e = 0; e < m; ++e) gid[e] = (int32_t)e;
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  Recursion R;
  R.C = C;
  R.part = part;
  R.spare.store(threads - 1);
  R.stop = stop;
  recurse(std::move(H), std::move(gid), k, 0, R);
  return !stopped(stop);
}

}  // namespace ep
