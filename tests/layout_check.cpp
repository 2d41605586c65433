// Host-only check of the kernel layouts the library builds (test code).
//
// Flux: invariants of the replica layout and the sliced-ELL slots, then one
// explicit step emulated in FP64 the way the kernels compute it (pull form
// over every kernel block's slots, interior vertices in place, shared
// vertices through their accumulator applied to every copy) against the
// plain edge-list step; also with a shard halo declared.
// SpMV: the warp kernel's algorithm emulated lane by lane (each lane's chunk
// of the row-ranked entries read the way the kernel reads them, runs of equal
// rows, the segmented scan over the 32 lanes, every row total stored once)
// against the plain edge-list product.
// Prints "total fails N"; exit status 1 on any failure.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "internal.h"

using namespace ep;

static int fails = 0;
#define CHECK(c, ...)                                          \
  do {                                                         \
    if (!(c)) {                                                \
      if (fails < 20) {                                        \
        printf("FAIL %s:%d: ", __FILE__, __LINE__);            \
        printf(__VA_ARGS__);                                   \
        printf("\n");                                          \
      }                                                        \
      ++fails;                                                 \
    }                                                          \
  } while (0)

// mesh-like random graph: each task joins a vertex to one of the next 40
// ids, with self loops and repeated pairs mixed in
static void local_graph(int n, int m, std::mt19937& rng, std::vector<int32_t>& s, std::vector<int32_t>& d) {
  s.clear();
  d.clear();
  for (int i = 0; i < m; ++i) {
    const int u = (int)(rng() % n);
    s.push_back(u);
    d.push_back((u + 1 + (int)(rng() % 40)) % n);
  }
  for (int i = 0; i < m / 50; ++i) s[i] = d[i];
  for (int i = m / 50; i < m / 25; ++i) {
    s[i] = s[i + m / 25];
    d[i] = d[i + m / 25];
  }
}

static bool build(HostSchedule& h, int n, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
                  int C, bool dflt, bool bip) {
  const int64_t m = (int64_t)src.size();
  h.m = m;
  h.n = n;
  h.nd = bip ? 2 * (int64_t)n : n;
  h.C = C;
  h.flags = (bip ? 1u : 0u) | (dflt ? 2u : 0u);
  h.k = (m + C - 1) / C;
  h.src = src;
  h.dst = dst;
  h.part.resize(m);
  if (dflt) {
    for (int64_t e = 0; e < m; ++e) h.part[e] = (int32_t)(e / C);
  } else if (!partition_edges(src.data(), dst.data(), m, n, C, h.flags & 1u, 4, h.part.data())) {
    printf("partition stopped\n");
    return false;
  }
  const std::string err = build_schedule(h, 4);
  if (!err.empty()) {
    printf("build error %s\n", err.c_str());
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ flux

static void check_flux(const HostSchedule& h, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
                       int n, const char* what) {
  const int64_t m = (int64_t)src.size(), K = (int64_t)h.fdesc.size();
  CHECK(h.n_rec % 4 == 0, "%s: n_rec", what);
  CHECK((int64_t)h.vrec.size() == h.n_rec, "%s: vrec size", what);
  std::vector<int> slot_count(m, 0), src_count(m, 0);
  for (int64_t b = 0; b < K; ++b) {
    const FluxDesc& d = h.fdesc[b];
    CHECK(d.rec_lo % 4 == 0 && d.s0 % 32 == 0 && d.nslot % 32 == 0 && d.h0 % 4 == 0 && d.q0 % 8 == 0,
          "%s: alignment of block %lld", what, (long long)b);
    CHECK(d.rec_lo + d.nv <= h.n_run, "%s: record run", what);
    CHECK(d.nsl == (d.nv + 31) / 32, "%s: slices", what);
    CHECK(32 * h.soff[d.q0 + d.nsl] == d.nslot, "%s: slots against offsets", what);
    CHECK(d.nv <= h.max_nv && d.nslot <= h.max_nslot && d.nv - d.ni <= h.max_nsh && d.nsl <= h.max_nsl,
          "%s: maxima", what);
    for (int32_t q = 0; q < d.nv; ++q) {
      const int32_t v = h.vrec[d.rec_lo + q];
      CHECK(v >= 0 && v < n, "%s: vertex of a position", what);
      if (q < d.ni) {
        CHECK(h.rec_of[v] == d.rec_lo + q, "%s: interior record", what);
      } else {
        const int32_t raw = h.sid_list[d.h0 + q - d.ni], sid = raw & kSidMask;
        CHECK(sid >= 0 && sid < h.n_sh, "%s: shared id range", what);
        CHECK((raw < 0) == (h.crec[h.cptr[sid]] == d.rec_lo + q), "%s: first-copy flag", what);
        CHECK(h.vrec[h.crec[h.cptr[sid]]] == v, "%s: first copy of the same vertex", what);
      }
    }
    for (int32_t j = 0; j < d.nsl; ++j)
      for (int32_t col = 0; col < h.soff[d.q0 + j + 1] - h.soff[d.q0 + j]; ++col)
        for (int l = 0; l < 32; ++l) {
          const int64_t sl = d.s0 + 32 * (int64_t)(h.soff[d.q0 + j] + col) + l;
          const uint16_t e = h.sidx[sl];
          const int p = 32 * j + l;
          if (h.wmap[sl] < 0) {  // unused: weight 0, any position of the block
            CHECK((e & kSlotSrc) == 0 && (int)e < std::max(1, std::min(d.nv, 32)), "%s: unused slot", what);
            continue;
          }
          CHECK(p < d.nv, "%s: slot lane past the block", what);
          CHECK((e & kSlotPos) < d.nv, "%s: slot position range", what);
          const int32_t t = h.wmap[sl];
          CHECK(t >= 0 && t < m, "%s: slot task", what);
          if (t < 0 || t >= m) continue;
          slot_count[t]++;
          const int32_t vp = h.vrec[d.rec_lo + p], vo = h.vrec[d.rec_lo + (e & kSlotPos)];
          if (e & kSlotSrc) {
            src_count[t]++;
            CHECK(h.gslot[t] == sl, "%s: source slot of task", what);
            CHECK(vp == src[t] && vo == dst[t], "%s: source slot endpoints", what);
          } else {
            CHECK(vp == dst[t] && vo == src[t], "%s: destination slot endpoints", what);
          }
        }
  }
  for (int64_t t = 0; t < m; ++t) {
    CHECK(src_count[t] == 1, "%s: one source slot per task", what);
    CHECK(slot_count[t] == (src[t] == dst[t] ? 1 : 2), "%s: slots per task", what);
  }
  for (int v = 0; v < n; ++v) CHECK(h.vrec[h.rec_of[v]] == v, "%s: rec_of / vrec", what);
  for (int32_t v : h.halo) {  // a touched halo vertex is shared
    const int32_t r = h.rec_of[v];
    if (r >= h.n_run) continue;  // untouched here
    bool shared = false;
    for (int64_t sh = 0; sh < h.n_sh && !shared; ++sh) shared = h.vrec[h.crec[h.cptr[sh]]] == v;
    CHECK(shared, "%s: halo vertex %d not shared", what, v);
  }

  // one explicit step, D = 3, FP64
  const int D = 3;
  const double tau = 0.01;
  std::mt19937 rng(7);
  std::normal_distribution<double> nd(0, 1);
  std::vector<double> x((size_t)n * D), w(m), ref((size_t)n * D, 0.0);
  for (auto& v : x) v = nd(rng);
  for (auto& v : w) v = 0.5 + (rng() % 1000) / 1000.0;
  for (int64_t t = 0; t < m; ++t) {
    const int u = src[t], v = dst[t];
    double dd[D], q = 0;
    for (int c = 0; c < D; ++c) {
      dd[c] = x[v * D + c] - x[u * D + c];
      q += dd[c] * dd[c];
    }
    for (int c = 0; c < D; ++c) {
      ref[u * D + c] += w[t] * dd[c] / (1 + q);
      ref[v * D + c] -= w[t] * dd[c] / (1 + q);
    }
  }
  std::vector<double> xl((size_t)h.n_rec * D, 0.0), xo, acc((size_t)h.n_sh * D, 0.0), wl(h.w_pad, 0.0);
  for (int64_t r = 0; r < h.n_rec; ++r)
    if (h.vrec[r] >= 0)
      for (int c = 0; c < D; ++c) xl[r * D + c] = x[h.vrec[r] * D + c];
  for (int64_t sl = 0; sl < h.w_pad; ++sl)
    if (h.wmap[sl] >= 0) wl[sl] = w[h.wmap[sl]];
  xo = xl;
  for (int64_t b = 0; b < K; ++b) {
    const FluxDesc& d = h.fdesc[b];
    for (int32_t j = 0; j < d.nsl; ++j)
      for (int l = 0; l < 32; ++l) {
        const int p = 32 * j + l;
        if (p >= d.nv) continue;
        double a[D] = {0, 0, 0};
        for (int col = 0; col < h.soff[d.q0 + j + 1] - h.soff[d.q0 + j]; ++col) {
          const int64_t sl = d.s0 + 32 * (int64_t)(h.soff[d.q0 + j] + col) + l;
          const int o = h.sidx[sl] & kSlotPos;
          double dd[D], q = 0;
          for (int c = 0; c < D; ++c) {
            dd[c] = xl[(d.rec_lo + o) * D + c] - xl[(d.rec_lo + p) * D + c];
            q += dd[c] * dd[c];
          }
          for (int c = 0; c < D; ++c) a[c] += wl[sl] * dd[c] / (1 + q);
        }
        if (p < d.ni) {
          for (int c = 0; c < D; ++c) xo[(d.rec_lo + p) * D + c] = xl[(d.rec_lo + p) * D + c] + tau * a[c];
        } else {
          const int sid = h.sid_list[d.h0 + p - d.ni] & kSidMask;
          for (int c = 0; c < D; ++c) acc[sid * D + c] += a[c];
        }
      }
  }
  for (int64_t sh = 0; sh < h.n_sh; ++sh)
    for (int32_t c = h.cptr[sh]; c < h.cptr[sh + 1]; ++c)
      for (int k = 0; k < D; ++k) xo[h.crec[c] * D + k] = xl[h.crec[h.cptr[sh]] * D + k] + tau * acc[sh * D + k];
  double err2 = 0, nrm = 0;
  for (int v = 0; v < n; ++v)
    for (int c = 0; c < D; ++c) {
      const double want = x[v * D + c] + tau * ref[v * D + c], got = xo[h.rec_of[v] * D + c];
      err2 += (got - want) * (got - want);
      nrm += want * want;
    }
  const double rel = std::sqrt(err2 / nrm);
  CHECK(rel < 1e-13, "%s: emulated step, relative error %.3e", what, rel);
  printf("flux %s: kernel blocks %lld, shared %lld, slots %zu, rel %.2e\n", what, (long long)K,
         (long long)h.n_sh, h.sidx.size(), rel);
}

static void run_flux(int n, const std::vector<int32_t>& s, const std::vector<int32_t>& d, int C, bool dflt,
                     bool halo) {
  HostSchedule h;
  if (!build(h, n, s, d, C, dflt, false)) {
    ++fails;
    return;
  }
  char what[96];
  snprintf(what, sizeof what, "n=%d m=%zu C=%d %s", n, s.size(), C, dflt ? "default" : "partitioned");
  check_flux(h, s, d, n, what);
  if (!halo) return;
  std::mt19937 rng(11);
  h.halo.clear();
  for (int v = 0; v < n; ++v)
    if (rng() % 10 == 0) h.halo.push_back(v);
  h.halo.push_back(h.halo.empty() ? 0 : h.halo[0]);  // a duplicate
  const std::string err = rebuild_flux_layout(h);
  CHECK(err.empty(), "halo rebuild: %s", err.c_str());
  snprintf(what, sizeof what, "n=%d m=%zu C=%d %s halo", n, s.size(), C, dflt ? "default" : "partitioned");
  check_flux(h, s, d, n, what);
}

// ------------------------------------------------------------------ SpMV

struct Run {
  int cur = -1, hrow = -1;
  double acc = 0, hsum = 0;
  bool whole = true;
};

static void check_spmv(const HostSchedule& h, const std::vector<int32_t>& rows, const std::vector<int32_t>& cols,
                       int n, const char* what) {
  const int64_t m = (int64_t)rows.size();
  std::mt19937 rng(5);
  std::uniform_real_distribution<double> ud(-1, 1);
  std::vector<double> x(n), w(m), ref(n, 0.0);
  for (auto& v : x) v = ud(rng);
  for (auto& v : w) v = ud(rng);
  for (int64_t t = 0; t < m; ++t) ref[rows[t]] += w[t] * x[cols[t]];
  std::vector<double> xl(n), wl(h.w_pad, 0.0), yl(n, 0.0);
  for (int j = 0; j < n; ++j) xl[h.xrec_of[j]] = x[j];
  for (int64_t sl = 0; sl < h.w_pad; ++sl)
    if (h.wmap[sl] >= 0) wl[sl] = w[h.wmap[sl]];
  std::vector<int> stored_rec(n, 0);
  for (int64_t b = 0; b < h.k; ++b) {
    const SpmvDesc& d = h.sdesc[b];
    CHECK(d.i0 == 32 * d.u * b, "%s: entry run of block %lld", what, (long long)b);
    CHECK(d.u % 4 == 0 && 32 * d.u >= d.ne, "%s: chunk size", what);
    const int nx = d.n_xo + d.n_xf, ny = d.n_yi + d.n_yob + d.n_yf, own = d.n_yi + d.n_yob;
    std::vector<double> xs(nx), ys(ny, 0.0);
    std::vector<int> stores(ny, 0);
    for (int c = 0; c < nx; ++c) xs[c] = xl[c < d.n_xo ? d.x_lo + c : h.xlist[d.fx0 + c - d.n_xo]];
    Run run[32];
    auto take = [&](Run& r, uint32_t e, double v) {
      const int row = (int)(e >> kRowShift);
      if (row != r.cur) {
        if (r.cur >= 0) {
          if (r.whole) {
            r.hrow = r.cur;
            r.hsum = r.acc;
            r.whole = false;
          } else {
            ys[r.cur] = r.acc;
            ++stores[r.cur];
          }
        }
        r.cur = row;
        r.acc = v;
      } else {
        r.acc += v;
      }
    };
    for (int l = 0; l < 32; ++l) {
      const int nj = std::min(std::max(d.ne - l * d.u, 0), d.u);
      for (int c = 0; 4 * c < nj; ++c)  // chunk c of lane l: slots i0 + (32 c + l) * 4 + q
        for (int q = 0; q < 4 && 4 * c + q < nj; ++q) {
          const int64_t slot = d.i0 + (int64_t)(32 * c + l) * 4 + q;
          const uint32_t e = h.sent[slot];
          CHECK((int)(e & kColMask) < nx && (int)(e >> kRowShift) < ny, "%s: entry range", what);
          take(run[l], e, wl[slot] * xs[e & kColMask]);
        }
    }
    // the join, as the warp does it
    int rt[32], rh[32], F[32];
    bool cont[32];
    double S[32];
    for (int l = 0; l < 32; ++l) {
      rt[l] = run[l].cur;
      rh[l] = run[l].whole ? run[l].cur : run[l].hrow;
    }
    for (int l = 0; l < 32; ++l) {
      cont[l] = l > 0 && rh[l] >= 0 && rh[l] == rt[l - 1];
      S[l] = run[l].acc;
      F[l] = !(run[l].whole && cont[l]);
    }
    for (int o = 1; o < 32; o <<= 1) {
      double S2[32];
      int F2[32];
      for (int l = 0; l < 32; ++l) {
        S2[l] = S[l];
        F2[l] = F[l];
        if (l >= o && !F[l]) {
          S2[l] = S[l] + S[l - o];
          F2[l] = F[l - o];
        }
      }
      std::copy(S2, S2 + 32, S);
      std::copy(F2, F2 + 32, F);
    }
    for (int l = 0; l < 32; ++l) {
      const double S_prev = l > 0 ? S[l - 1] : S[l];
      const bool cont_next = l < 31 ? cont[l + 1] : cont[l];
      if (!run[l].whole) {
        ys[rh[l]] = run[l].hsum + (cont[l] ? S_prev : 0.0);
        ++stores[rh[l]];
      }
      if (rt[l] >= 0 && !(l < 31 && cont_next)) {
        ys[rt[l]] = S[l];
        ++stores[rt[l]];
      }
    }
    for (int p = 0; p < ny; ++p) {
      CHECK(stores[p] == 1, "%s: block %lld row position %d stored %d times", what, (long long)b, p, stores[p]);
      int32_t r;
      if (p < d.n_yi) {
        r = d.yi_lo + p;
        yl[r] = ys[p];
        ++stored_rec[r];
      } else {
        r = p < own ? d.yb_lo + (p - d.n_yi) : h.ylist[d.fy0 + (p - own)];
        CHECK(r >= h.ny_int, "%s: shared row record below the zeroed range", what);
        yl[r] += ys[p];
      }
    }
  }
  for (int i = 0; i < n; ++i) CHECK(stored_rec[i] <= 1, "%s: single-block row stored twice", what);
  double err2 = 0, nrm = 0;
  for (int i = 0; i < n; ++i) {
    const double got = yl[h.yrec_of[i]];
    err2 += (got - ref[i]) * (got - ref[i]);
    nrm += ref[i] * ref[i];
  }
  const double rel = std::sqrt(err2 / std::max(nrm, 1e-300));
  CHECK(rel < 1e-13, "%s: emulated SpMV, relative error %.3e", what, rel);
  printf("spmv %s: blocks %lld, u %d, rel %.2e\n", what, (long long)h.k, h.spmv_u, rel);
}

// power-law-ish bipartite graph: rows and columns drawn with a skew, duplicates kept
static void skewed_graph(int n, int m, std::mt19937& rng, std::vector<int32_t>& r, std::vector<int32_t>& c) {
  r.clear();
  c.clear();
  std::uniform_real_distribution<double> u01(0, 1);
  for (int i = 0; i < m; ++i) {
    r.push_back((int32_t)(n * std::pow(u01(rng), 3.0)) % n);
    c.push_back((int32_t)(n * std::pow(u01(rng), 2.0)) % n);
  }
}

static void run_spmv(int n, const std::vector<int32_t>& r, const std::vector<int32_t>& c, int C, bool dflt) {
  HostSchedule h;
  if (!build(h, n, r, c, C, dflt, true)) {
    ++fails;
    return;
  }
  char what[96];
  snprintf(what, sizeof what, "n=%d m=%zu C=%d %s", n, r.size(), C, dflt ? "default" : "partitioned");
  check_spmv(h, r, c, n, what);
}

int main() {
  std::mt19937 rng(3);
  std::vector<int32_t> s, d;
  local_graph(3000, 9000, rng, s, d);
  for (int C : {1, 7, 64, 256, 1000, 9000})
    for (bool dflt : {false, true}) run_flux(3000, s, d, C, dflt, C == 256 || C == 64);
  local_graph(2000, 3000, rng, s, d);  // with isolated vertices
  for (auto& v : s) v %= 1500;
  for (auto& v : d) v %= 1500;
  run_flux(2000, s, d, 100, false, true);
  skewed_graph(4096, 40000, rng, s, d);
  for (int C : {1, 37, 256, 512, 2048})
    for (bool dflt : {false, true}) run_spmv(4096, s, d, C, dflt);
  printf("total fails %d\n", fails);
  return fails != 0;
}
