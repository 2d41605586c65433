// prescreen.cpp -- the checks made before partitioning (Section 4, the
// optimisation workflow): is there enough data reuse, and is the graph a
// special pattern with a known optimal schedule.
//
// Patterns with a preset (optimal under Eq. 1, see below):
//   path  -- a simple path: every block of C consecutive path edges touches
//            C + 1 vertices, the least any C edges of a path can touch, so
//            walking the path and cutting every C edges gives m + k loads.
//   star  -- every task uses one centre vertex and a leaf of its own: every
//            block loads the centre plus one leaf per task whatever the
//            schedule, so the default order is optimal.
// Low reuse: when the mean degree of the touched data vertices is at most 2
// (every data object is used by about two tasks or fewer), the reorder is
// skipped and the default order is kept.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace ep {

namespace {

struct Ends {
  int64_t u, v;  // data vertices of a task; u == v for a self loop
};

Ends ends(const int32_t* src, const int32_t* dst, int64_t e, int64_t n, bool bip) {
  if (bip) return {n + src[e], dst[e]};
  return {src[e], dst[e]};
}

}  // namespace

PrescreenResult prescreen(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, bool bip) {
  PrescreenResult r;
  const int64_t nd = bip ? 2 * n : n;
  std::vector<int64_t> deg(nd, 0);
  bool loops = false;
  for (int64_t e = 0; e < m; ++e) {
    const Ends t = ends(src, dst, e, n, bip);
    ++deg[t.u];
    if (t.v != t.u)
      ++deg[t.v];
    else
      loops = true;
  }
  int64_t ones = 0, first_end = -1, centre = -1;
  for (int64_t v = 0; v < nd; ++v) {
    if (deg[v] == 0) continue;
    ++r.touched;
    r.degree_sum += deg[v];
    r.max_degree = std::max(r.max_degree, deg[v]);
    if (deg[v] == 1) {
      ++ones;
      if (first_end < 0) first_end = v;
    }
    if (deg[v] == m && centre < 0) centre = v;
  }
  // path: no loops, degrees <= 2, two ends, m + 1 vertices, one component
  if (!loops && r.max_degree <= 2 && ones == 2 && r.touched == m + 1) {
    std::vector<int64_t> xadj(nd + 1, 0);
    for (int64_t v = 0; v < nd; ++v) xadj[v + 1] = xadj[v] + deg[v];
    std::vector<int64_t> fill(xadj.begin(), xadj.end() - 1);
    std::vector<int32_t> inc(2 * m);
    for (int64_t e = 0; e < m; ++e) {
      const Ends t = ends(src, dst, e, n, bip);
      inc[fill[t.u]++] = (int32_t)e;
      inc[fill[t.v]++] = (int32_t)e;
    }
    std::vector<uint8_t> used(m, 0);
    r.order.reserve(m);
    int64_t v = first_end;
    for (;;) {
      int32_t next = -1;
      for (int64_t j = xadj[v]; j < xadj[v + 1]; ++j)
        if (!used[inc[j]]) {
          next = inc[j];
          break;
        }
      if (next < 0) break;
      used[next] = 1;
      r.order.push_back(next);
      const Ends t = ends(src, dst, next, n, bip);
      v = t.u == v ? t.v : t.u;
    }
    if ((int64_t)r.order.size() == m) {
      r.origin = kOriginPath;
      return r;
    }
    r.order.clear();
  }
  // star: one centre in every task, every other touched vertex a leaf
  if (!loops && m >= 2 && centre >= 0 && r.touched == m + 1 && ones == m) {
    r.origin = kOriginStar;
    return r;
  }
  r.origin = r.degree_sum <= 2 * r.touched ? kOriginLowReuse : kOriginPartition;
  return r;
}

}  // namespace ep
