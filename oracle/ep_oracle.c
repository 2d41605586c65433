/*
 * ep_oracle.c -- plain serial CPU oracle for the edge-partition schedule.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only tests/, the package smoke check and the bench's CPU-baseline
 * leg do.  It shares no code with the CUDA library.
 *
 * What it computes (paper: "A Graph-based Model for GPU Caching Problems"):
 *   - the data-affinity graph D=(V,E): data objects are vertices, tasks are
 *     edges (Section 3.1, Definition 1); for SpMV the bipartite graph with one
 *     vertex per x_j and per y_i (Section 5.2);
 *   - the clone-and-connect transform D -> D' (Section 3.2, Definition 3) with
 *     clones joined in index order, and the "very large" weight on original
 *     edges read as contracting every original edge: the result H has one
 *     vertex per task and one unit-weight edge per auxiliary edge;
 *   - a balanced vertex partition of H (the paper uses METIS; the rules below
 *     replace it with a fixed deterministic multilevel recursive bisection);
 *   - the reconstruction of the edge partition (Definition 4);
 *   - per-block distinct-vertex lists, the cpack first-touch relabelling
 *     (Section 4.1) and the vertex-cut cost C = sum_v (p_v - 1) (Eq. 1).
 *
 * Partition rules (fixed here because the paper leaves them to METIS):
 *   k = ceil(m / C) blocks.  RB(S, k'): if k' = 1 the set S is one block;
 *   otherwise the left part gets kL = ceil(k'/2) blocks and exactly kL*C
 *   vertices of H, the right part the rest; blocks are numbered left to right.
 *   Bisection of the induced graph (vertex ids ascending by task id):
 *     coarsen  while n > 64: heavy-edge matching visiting u ascending; u takes
 *              the unmatched neighbour of largest edge weight (ties: smaller
 *              id) whose combined vertex weight is <= maxw = max(1, min(sL,
 *              W-sL)/16); coarse ids in order of the smaller member; stop (and
 *              drop the level) when it shrinks the graph by less than 10%;
 *              stop after a level whose adjacency (entries, both directions)
 *              shrank by less than 15% (dense coarse graphs of power-law
 *              inputs);
 *     initial  graph growing: start at the last vertex dequeued by a BFS from
 *              vertex 0 (neighbours ascending); BFS from there adding each
 *              dequeued vertex to the left while it fits (a vertex that does
 *              not fit stays right and is not expanded); when the queue runs
 *              dry, restart at the smallest unvisited vertex;
 *     refine   at every level, up to 4 passes: candidates are the vertices of
 *              positive gain (external minus internal edge weight), ordered by
 *              (gain desc, id asc) at the start of the pass; each is moved if
 *              its current gain is still positive and the move leaves
 *              |lw - sL| <= max(tol, current |lw - sL|), tol = max(1,
 *              min(sL, W-sL)/32); a vertex moves at most once per pass;
 *     fix      at the finest level, while lw != sL move the vertex of the
 *              heavy side with the largest gain (ties: smaller id) across.
 *   Inside a block edges keep ascending task id.  Vertex lists scan the block's
 *   edges in order, endpoint u then v, keeping first appearances.  cpack gives
 *   new ids in order of first appearance over blocks 0..k-1; untouched
 *   vertices follow in ascending old id.
 *
 * Parity: the worked example of Fig. 1 (9 vs 7 loads), Theorem 1 on every
 * produced partition and Theorem 2 against brute-force optima pin what the
 * paper fixes.  The exact tie-break output of the heuristic beyond those cases
 * is a rule of this project, not of the paper.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_COARSEN_MIN 64
#define ORC_NPASS 4

typedef struct {
  int32_t n;
  int64_t *xadj; /* n+1 */
  int32_t *adj;  /* neighbours, ascending per vertex */
  int32_t *ew;   /* edge weights */
  int32_t *vw;   /* vertex weights */
} graph_t;

static void graph_free(graph_t *g) {
  free(g->xadj);
  free(g->adj);
  free(g->ew);
  free(g->vw);
  memset(g, 0, sizeof(*g));
}

typedef struct {
  int32_t a, b;
} pair_t;

static int cmp_pair(const void *p, const void *q) {
  const pair_t *x = (const pair_t *)p, *y = (const pair_t *)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  return 0;
}

/* Endpoints of task e as data-vertex ids.  Bipartite (SpMV): x_j -> j and
 * y_i -> n + i, where the task is A[i][j] with src = i (row), dst = j (col). */
static void endpoints(const int32_t *src, const int32_t *dst, int64_t e, int64_t n, int bip,
                      int64_t *u, int64_t *v) {
  if (bip) {
    *u = n + (int64_t)src[e];
    *v = (int64_t)dst[e];
  } else {
    *u = src[e];
    *v = dst[e];
  }
}

/* Clone-and-connect with contracted original edges: H has one vertex per task;
 * for every data vertex, its incident tasks in ascending id are joined by a
 * path of unit-weight auxiliary edges.  Parallel auxiliary edges are merged
 * with summed weight.  Returns 0, or -1 when out of memory. */
static int build_h(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int bip,
                   graph_t *H) {
  int64_t nd = bip ? 2 * n : n;
  int64_t *deg = calloc((size_t)nd + 1, sizeof(int64_t));
  int64_t *pos = malloc(((size_t)nd + 1) * sizeof(int64_t));
  int32_t *inc = malloc((size_t)(2 * m + 1) * sizeof(int32_t));
  if (!deg || !pos || !inc) return -1;
  for (int64_t e = 0; e < m; e++) {
    int64_t u, v;
    endpoints(src, dst, e, n, bip, &u, &v);
    deg[u]++;
    if (v != u) deg[v]++;
  }
  pos[0] = 0;
  for (int64_t v = 0; v < nd; v++) pos[v + 1] = pos[v] + deg[v];
  memcpy(deg, pos, (size_t)nd * sizeof(int64_t)); /* deg is now a write cursor */
  for (int64_t e = 0; e < m; e++) {
    int64_t u, v;
    endpoints(src, dst, e, n, bip, &u, &v);
    inc[deg[u]++] = (int32_t)e;
    if (v != u) inc[deg[v]++] = (int32_t)e;
  }
  /* auxiliary edges, both directions */
  int64_t np = 0;
  for (int64_t v = 0; v < nd; v++) {
    int64_t d = pos[v + 1] - pos[v];
    if (d > 1) np += 2 * (d - 1);
  }
  pair_t *pr = malloc((size_t)(np + 1) * sizeof(pair_t));
  if (!pr) return -1;
  int64_t q = 0;
  for (int64_t v = 0; v < nd; v++) {
    for (int64_t i = pos[v]; i + 1 < pos[v + 1]; i++) {
      pr[q].a = inc[i];
      pr[q].b = inc[i + 1];
      q++;
      pr[q].a = inc[i + 1];
      pr[q].b = inc[i];
      q++;
    }
  }
  qsort(pr, (size_t)np, sizeof(pair_t), cmp_pair);
  H->n = (int32_t)m;
  H->xadj = calloc((size_t)m + 1, sizeof(int64_t));
  H->adj = malloc((size_t)(np + 1) * sizeof(int32_t));
  H->ew = malloc((size_t)(np + 1) * sizeof(int32_t));
  H->vw = malloc((size_t)(m + 1) * sizeof(int32_t));
  if (!H->xadj || !H->adj || !H->ew || !H->vw) return -1;
  for (int64_t e = 0; e < m; e++) H->vw[e] = 1;
  int64_t nnz = 0;
  for (int64_t i = 0; i < np;) {
    int64_t j = i;
    while (j < np && pr[j].a == pr[i].a && pr[j].b == pr[i].b) j++;
    H->adj[nnz] = pr[i].b;
    H->ew[nnz] = (int32_t)(j - i);
    H->xadj[pr[i].a + 1]++;
    nnz++;
    i = j;
  }
  for (int64_t e = 0; e < m; e++) H->xadj[e + 1] += H->xadj[e];
  free(pr);
  free(inc);
  free(pos);
  free(deg);
  return 0;
}

/* ---------------------------------------------------------------- coarsening */

/* Heavy-edge matching.  cmap[u] = coarse id; returns the number of coarse
 * vertices.  mate[u] = partner (u itself when single). */
static int32_t match_heavy(const graph_t *g, int32_t maxw, int32_t *cmap, int32_t *mate) {
  for (int32_t u = 0; u < g->n; u++) mate[u] = -1;
  int32_t nc = 0;
  for (int32_t u = 0; u < g->n; u++) {
    if (mate[u] >= 0) continue;
    int32_t best = -1, bw = -1;
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t v = g->adj[j];
      if (v == u || mate[v] >= 0) continue;
      if ((int64_t)g->vw[u] + g->vw[v] > maxw) continue;
      if (g->ew[j] > bw || (g->ew[j] == bw && v < best)) {
        best = v;
        bw = g->ew[j];
      }
    }
    if (best >= 0) {
      mate[u] = best;
      mate[best] = u;
      cmap[u] = nc;
      cmap[best] = nc;
    } else {
      mate[u] = u;
      cmap[u] = nc;
    }
    nc++;
  }
  return nc;
}

static int build_coarse(const graph_t *g, const int32_t *cmap, const int32_t *mate, int32_t nc,
                        graph_t *cg) {
  cg->n = nc;
  cg->xadj = calloc((size_t)nc + 1, sizeof(int64_t));
  cg->vw = malloc((size_t)(nc + 1) * sizeof(int32_t));
  cg->adj = malloc((size_t)(g->xadj[g->n] + 1) * sizeof(int32_t));
  cg->ew = malloc((size_t)(g->xadj[g->n] + 1) * sizeof(int32_t));
  pair_t *tmp = malloc((size_t)(g->xadj[g->n] + 1) * sizeof(pair_t));
  if (!cg->xadj || !cg->vw || !cg->adj || !cg->ew || !tmp) return -1;
  int64_t nnz = 0;
  for (int32_t u = 0; u < g->n; u++) {
    if (mate[u] < u) continue; /* only the smaller member (leader) emits */
    int32_t c = cmap[u];
    int32_t mem[2] = {u, mate[u]};
    int nm = mate[u] == u ? 1 : 2;
    int32_t w = 0;
    int64_t t = 0;
    for (int i = 0; i < nm; i++) {
      int32_t x = mem[i];
      w += g->vw[x];
      for (int64_t j = g->xadj[x]; j < g->xadj[x + 1]; j++) {
        int32_t cv = cmap[g->adj[j]];
        if (cv == c) continue;
        tmp[t].a = cv;
        tmp[t].b = g->ew[j];
        t++;
      }
    }
    cg->vw[c] = w;
    /* sort by neighbour id, merge duplicates by summing weights */
    qsort(tmp, (size_t)t, sizeof(pair_t), cmp_pair);
    for (int64_t i = 0; i < t;) {
      int64_t j = i;
      int32_t s = 0;
      while (j < t && tmp[j].a == tmp[i].a) s += tmp[j++].b;
      cg->adj[nnz] = tmp[i].a;
      cg->ew[nnz] = s;
      nnz++;
      i = j;
    }
    cg->xadj[c + 1] = nnz;
  }
  free(tmp);
  return 0;
}

/* ------------------------------------------------------- initial bisection */

static void grow_bisection(const graph_t *g, int64_t sL, uint8_t *side) {
  int32_t n = g->n;
  int32_t *queue = malloc((size_t)n * sizeof(int32_t));
  uint8_t *seen = calloc((size_t)n, 1);
  /* start vertex: last vertex dequeued by a BFS from vertex 0 */
  int32_t head = 0, tail = 0, last = 0;
  queue[tail++] = 0;
  seen[0] = 1;
  while (head < tail) {
    int32_t u = queue[head++];
    last = u;
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t v = g->adj[j];
      if (!seen[v]) {
        seen[v] = 1;
        queue[tail++] = v;
      }
    }
  }
  memset(seen, 0, (size_t)n);
  for (int32_t u = 0; u < n; u++) side[u] = 1;
  int64_t lw = 0;
  int32_t scan = 0;
  head = tail = 0;
  queue[tail++] = last;
  seen[last] = 1;
  while (lw < sL) {
    if (head == tail) {
      while (scan < n && seen[scan]) scan++;
      if (scan == n) break;
      queue[tail++] = scan;
      seen[scan] = 1;
    }
    int32_t u = queue[head++];
    if (lw + g->vw[u] > sL) continue; /* does not fit: stays right */
    side[u] = 0;
    lw += g->vw[u];
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t v = g->adj[j];
      if (!seen[v]) {
        seen[v] = 1;
        queue[tail++] = v;
      }
    }
  }
  free(seen);
  free(queue);
}

/* ------------------------------------------------------------- refinement */

static int64_t abs64(int64_t a) { return a < 0 ? -a : a; }

static void compute_gains(const graph_t *g, const uint8_t *side, int64_t *gain) {
  for (int32_t u = 0; u < g->n; u++) {
    int64_t s = 0;
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++)
      s += side[g->adj[j]] != side[u] ? g->ew[j] : -(int64_t)g->ew[j];
    gain[u] = s;
  }
}

static void apply_move(const graph_t *g, uint8_t *side, int64_t *gain, int32_t u) {
  side[u] ^= 1;
  gain[u] = -gain[u];
  for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
    int32_t x = g->adj[j];
    if (side[x] == side[u])
      gain[x] -= 2 * (int64_t)g->ew[j];
    else
      gain[x] += 2 * (int64_t)g->ew[j];
  }
}

typedef struct {
  int64_t gain;
  int32_t id;
} cand_t;

/* order: gain descending, id ascending */
static int cmp_cand(const void *p, const void *q) {
  const cand_t *x = (const cand_t *)p, *y = (const cand_t *)q;
  if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

static void refine(const graph_t *g, int64_t sL, int64_t W, uint8_t *side) {
  int32_t n = g->n;
  int64_t tol = (sL < W - sL ? sL : W - sL) / 32;
  if (tol < 1) tol = 1;
  int64_t *gain = malloc((size_t)(n + 1) * sizeof(int64_t));
  cand_t *cand = malloc((size_t)(n + 1) * sizeof(cand_t));
  int64_t lw = 0;
  for (int32_t u = 0; u < n; u++)
    if (side[u] == 0) lw += g->vw[u];
  for (int pass = 0; pass < ORC_NPASS; pass++) {
    compute_gains(g, side, gain);
    int32_t nc = 0;
    for (int32_t u = 0; u < n; u++)
      if (gain[u] > 0) {
        cand[nc].gain = gain[u];
        cand[nc].id = u;
        nc++;
      }
    qsort(cand, (size_t)nc, sizeof(cand_t), cmp_cand);
    int32_t moved = 0;
    for (int32_t i = 0; i < nc; i++) {
      int32_t u = cand[i].id;
      if (gain[u] <= 0) continue;
      int64_t nl = side[u] == 0 ? lw - g->vw[u] : lw + g->vw[u];
      int64_t lim = abs64(lw - sL) > tol ? abs64(lw - sL) : tol;
      if (abs64(nl - sL) > lim) continue;
      apply_move(g, side, gain, u);
      lw = nl;
      moved++;
    }
    if (moved == 0) break;
  }
  free(cand);
  free(gain);
}

/* binary max-heap on (gain desc, id asc) with lazy deletion */
typedef struct {
  cand_t *a;
  int64_t n;
} heap_t;

static int heap_less(const cand_t *x, const cand_t *y) { /* x before y? */
  if (x->gain != y->gain) return x->gain > y->gain;
  return x->id < y->id;
}

static void heap_push(heap_t *h, int64_t gain, int32_t id) {
  int64_t i = h->n++;
  h->a[i].gain = gain;
  h->a[i].id = id;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!heap_less(&h->a[i], &h->a[p])) break;
    cand_t t = h->a[i];
    h->a[i] = h->a[p];
    h->a[p] = t;
    i = p;
  }
}

static cand_t heap_pop(heap_t *h) {
  cand_t top = h->a[0];
  h->a[0] = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, b = i;
    if (l < h->n && heap_less(&h->a[l], &h->a[b])) b = l;
    if (r < h->n && heap_less(&h->a[r], &h->a[b])) b = r;
    if (b == i) break;
    cand_t t = h->a[i];
    h->a[i] = h->a[b];
    h->a[b] = t;
    i = b;
  }
  return top;
}

/* Finest level (unit vertex weights): move best-gain vertices off the heavy
 * side until the left side holds exactly sL vertices. */
static void exact_fix(const graph_t *g, int64_t sL, uint8_t *side) {
  int32_t n = g->n;
  int64_t lw = 0;
  for (int32_t u = 0; u < n; u++)
    if (side[u] == 0) lw += g->vw[u];
  if (lw == sL) return;
  uint8_t heavy = lw > sL ? 0 : 1;
  int64_t *gain = malloc((size_t)(n + 1) * sizeof(int64_t));
  compute_gains(g, side, gain);
  /* each move pushes at most deg entries; bound the heap by n + 2*nnz */
  heap_t h;
  h.n = 0;
  h.a = malloc((size_t)(n + 2 * g->xadj[n] + 1) * sizeof(cand_t));
  for (int32_t u = 0; u < n; u++)
    if (side[u] == heavy) heap_push(&h, gain[u], u);
  while (lw != sL && h.n > 0) {
    cand_t c = heap_pop(&h);
    if (side[c.id] != heavy || c.gain != gain[c.id]) continue; /* stale */
    int32_t u = c.id;
    apply_move(g, side, gain, u);
    lw += heavy == 0 ? -1 : 1;
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t x = g->adj[j];
      if (side[x] == heavy) heap_push(&h, gain[x], x);
    }
  }
  free(h.a);
  free(gain);
}

/* --------------------------------------------------------------- bisection */

#define ORC_MAXLEV 64

static void bisect(const graph_t *g0, int64_t sL, uint8_t *side0) {
  int64_t W = g0->n; /* unit weights at the finest level */
  graph_t lev[ORC_MAXLEV];
  int32_t *cmaps[ORC_MAXLEV];
  int L = 0;
  lev[0] = *g0;
  int64_t mw = sL < W - sL ? sL : W - sL;
  int32_t maxw = (int32_t)(mw / 16 > 1 ? mw / 16 : 1);
  while (L + 1 < ORC_MAXLEV && lev[L].n > ORC_COARSEN_MIN) {
    const graph_t *g = &lev[L];
    int32_t *cmap = malloc((size_t)g->n * sizeof(int32_t));
    int32_t *mate = malloc((size_t)g->n * sizeof(int32_t));
    int32_t nc = match_heavy(g, maxw, cmap, mate);
    if ((int64_t)nc * 10 > (int64_t)g->n * 9) {
      free(cmap);
      free(mate);
      break;
    }
    graph_t cg;
    build_coarse(g, cmap, mate, nc, &cg);
    free(mate);
    cmaps[L] = cmap;
    lev[++L] = cg;
    /* a level whose adjacency shrank by less than 15% ends the coarsening */
    if (cg.xadj[cg.n] * 20 > g->xadj[g->n] * 17) break;
  }
  uint8_t *side = malloc((size_t)lev[L].n);
  grow_bisection(&lev[L], sL, side);
  refine(&lev[L], sL, W, side);
  for (int l = L - 1; l >= 0; l--) {
    uint8_t *fs = malloc((size_t)lev[l].n);
    for (int32_t u = 0; u < lev[l].n; u++) fs[u] = side[cmaps[l][u]];
    free(side);
    side = fs;
    refine(&lev[l], sL, W, side);
    free(cmaps[l]);
    graph_free(&lev[l + 1]);
  }
  exact_fix(&lev[0], sL, side);
  memcpy(side0, side, (size_t)g0->n);
  free(side);
}

/* induced subgraph of the vertices with side[u] == s; ids keep their order */
static void induced(const graph_t *g, const uint8_t *side, uint8_t s, const int32_t *gid,
                    graph_t *sg, int32_t **sgid) {
  int32_t *loc = malloc((size_t)g->n * sizeof(int32_t));
  int32_t cnt = 0;
  for (int32_t u = 0; u < g->n; u++) loc[u] = side[u] == s ? cnt++ : -1;
  sg->n = cnt;
  sg->xadj = calloc((size_t)cnt + 1, sizeof(int64_t));
  sg->vw = malloc((size_t)(cnt + 1) * sizeof(int32_t));
  *sgid = malloc((size_t)(cnt + 1) * sizeof(int32_t));
  int64_t nnz = 0;
  for (int32_t u = 0; u < g->n; u++)
    if (loc[u] >= 0)
      for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++)
        if (loc[g->adj[j]] >= 0) nnz++;
  sg->adj = malloc((size_t)(nnz + 1) * sizeof(int32_t));
  sg->ew = malloc((size_t)(nnz + 1) * sizeof(int32_t));
  nnz = 0;
  for (int32_t u = 0; u < g->n; u++) {
    if (loc[u] < 0) continue;
    int32_t lu = loc[u];
    sg->vw[lu] = g->vw[u];
    (*sgid)[lu] = gid[u];
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t lv = loc[g->adj[j]];
      if (lv < 0) continue;
      sg->adj[nnz] = lv;
      sg->ew[nnz] = g->ew[j];
      nnz++;
    }
    sg->xadj[lu + 1] = nnz;
  }
  free(loc);
}

static void rb(graph_t *g, int32_t *gid, int32_t kk, int32_t C, int32_t first, int32_t *part) {
  if (kk == 1) {
    for (int32_t u = 0; u < g->n; u++) part[gid[u]] = first;
    return;
  }
  int32_t kL = (kk + 1) / 2;
  int64_t sL = (int64_t)kL * C;
  uint8_t *side = malloc((size_t)g->n);
  bisect(g, sL, side);
  graph_t gl, gr;
  int32_t *gidl, *gidr;
  induced(g, side, 0, gid, &gl, &gidl);
  induced(g, side, 1, gid, &gr, &gidr);
  free(side);
  rb(&gl, gidl, kL, C, first, part);
  graph_free(&gl);
  free(gidl);
  rb(&gr, gidr, kk - kL, C, first + kL, part);
  graph_free(&gr);
  free(gidr);
}

/* ===================================================================== API */

static int check_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n) {
  if (m <= 0 || n <= 0 || m >= INT32_MAX) return -1;
  for (int64_t e = 0; e < m; e++)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
  return 0;
}

/* Number of H adjacency entries (both directions), or -1 on bad input. */
int64_t orc_h_nnz(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t bip) {
  if (check_edges(src, dst, m, n)) return -1;
  graph_t H;
  if (build_h(src, dst, m, n, bip, &H)) return -1;
  int64_t nnz = H.xadj[m];
  graph_free(&H);
  return nnz;
}

/* H as CSR: xadj[m+1], adj[nnz], ew[nnz]. */
int32_t orc_h_graph(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t bip,
                    int64_t *xadj, int32_t *adj, int32_t *ew) {
  if (check_edges(src, dst, m, n)) return -1;
  graph_t H;
  if (build_h(src, dst, m, n, bip, &H)) return -1;
  memcpy(xadj, H.xadj, (size_t)(m + 1) * sizeof(int64_t));
  memcpy(adj, H.adj, (size_t)H.xadj[m] * sizeof(int32_t));
  memcpy(ew, H.ew, (size_t)H.xadj[m] * sizeof(int32_t));
  graph_free(&H);
  return 0;
}

/* One bisection of a unit-vertex-weight graph given as CSR (ascending
 * adjacency): side[u] = 0 (left, exactly sL vertices) or 1. */
int32_t orc_bisect(const int64_t *xadj, const int32_t *adj, const int32_t *ew, int32_t n,
                   int64_t sL, uint8_t *side) {
  if (n <= 0 || sL <= 0 || sL >= n) return -1;
  graph_t g;
  g.n = n;
  g.xadj = (int64_t *)xadj;
  g.adj = (int32_t *)adj;
  g.ew = (int32_t *)ew;
  g.vw = malloc((size_t)n * sizeof(int32_t));
  for (int32_t u = 0; u < n; u++) g.vw[u] = 1;
  bisect(&g, sL, side);
  free(g.vw);
  return 0;
}

/* Pre-screen before partitioning (Section 4, the optimisation workflow):
 * out[0] = touched data vertices, out[1] = sum of their degrees (a self loop
 * counts once), out[2] = max degree, out[3] = outcome: 2 path (one simple
 * path: walk it from its smaller-id end), 3 star (one centre in every task,
 * every other vertex a leaf), 4 low reuse (mean degree <= 2), 0 partition.
 * The paper gives neither thresholds nor presets; these are the readings
 * used here.  order[m] (may be NULL) receives the walk for a path. */
int32_t orc_prescreen(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, uint32_t flags,
                      int64_t *out, int32_t *order) {
  if (check_edges(src, dst, m, n)) return -1;
  int bip = (int)(flags & 1u);
  int64_t nd = bip ? 2 * n : n;
  int64_t *deg = calloc((size_t)nd, sizeof(int64_t));
  int32_t *slot0 = malloc((size_t)nd * sizeof(int32_t)); /* first two incident tasks */
  int32_t *slot1 = malloc((size_t)nd * sizeof(int32_t));
  int loops = 0;
  for (int64_t e = 0; e < m; e++) {
    int64_t u, v;
    endpoints(src, dst, e, n, bip, &u, &v);
    int64_t ends[2] = {u, v};
    int cnt = (u == v) ? 1 : 2;
    if (u == v) loops = 1;
    for (int i = 0; i < cnt; i++) {
      int64_t x = ends[i];
      if (deg[x] == 0) slot0[x] = (int32_t)e;
      if (deg[x] == 1) slot1[x] = (int32_t)e;
      deg[x]++;
    }
  }
  int64_t touched = 0, sum = 0, maxd = 0, ones = 0, end0 = -1, centre = -1;
  for (int64_t x = 0; x < nd; x++) {
    if (deg[x] == 0) continue;
    touched++;
    sum += deg[x];
    if (deg[x] > maxd) maxd = deg[x];
    if (deg[x] == 1) {
      ones++;
      if (end0 < 0) end0 = x;
    }
    if (deg[x] == m && centre < 0) centre = x;
  }
  int64_t outcome = 0;
  if (!loops && maxd <= 2 && ones == 2 && touched == m + 1) {
    /* walk: leave each vertex by the incident task not arrived on */
    int64_t x = end0, steps = 0;
    int32_t prev = -1;
    while (steps < m) {
      int32_t e = -1;
      if (slot0[x] != prev)
        e = slot0[x];
      else if (deg[x] == 2 && slot1[x] != prev)
        e = slot1[x];
      if (e < 0) break;
      if (order) order[steps] = e;
      steps++;
      int64_t u, v;
      endpoints(src, dst, e, n, bip, &u, &v);
      x = (u == x) ? v : u;
      prev = e;
    }
    if (steps == m) outcome = 2;
  }
  if (outcome == 0 && !loops && m >= 2 && centre >= 0 && touched == m + 1 && ones == m)
    outcome = 3;
  if (outcome == 0 && sum <= 2 * touched) outcome = 4;
  out[0] = touched;
  out[1] = sum;
  out[2] = maxd;
  out[3] = outcome;
  free(deg);
  free(slot0);
  free(slot1);
  return 0;
}

/* Edge partition: part[e] in [0, k), k = ceil(m / C).  flags bit 0 =
 * bipartite, bit 1 = default order (C consecutive tasks per block), bit 2 =
 * pre-screen first (orc_prescreen): a path is cut every C tasks along its
 * walk, a star or a low-reuse graph keeps the default order. */
int32_t orc_partition(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t C,
                      uint32_t flags, int32_t *part) {
  if (C <= 0 || check_edges(src, dst, m, n)) return -1;
  int32_t k = (int32_t)((m + C - 1) / C);
  if ((flags & 4u) && !(flags & 2u)) {
    int64_t info[4];
    int32_t *order = malloc((size_t)m * sizeof(int32_t));
    orc_prescreen(src, dst, m, n, flags, info, order);
    if (info[3] == 2)
      for (int64_t i = 0; i < m; i++) part[order[i]] = (int32_t)(i / C);
    free(order);
    if (info[3] == 2) return 0;
    if (info[3] == 3 || info[3] == 4) flags |= 2u;
  }
  if ((flags & 2u) || k == 1) {
    for (int64_t e = 0; e < m; e++) part[e] = (int32_t)(e / C);
    return 0;
  }
  graph_t H;
  if (build_h(src, dst, m, n, (int)(flags & 1u), &H)) return -2;
  int32_t *gid = malloc((size_t)m * sizeof(int32_t));
  for (int64_t e = 0; e < m; e++) gid[e] = (int32_t)e;
  rb(&H, gid, k, C, 0, part);
  free(gid);
  graph_free(&H);
  return 0;
}

/* Schedule from a partition.  Outputs (caller-sized):
 *   block_ptr[k+1], edge_perm[m]      tasks grouped by block, ascending id
 *   vert_ptr[k+1], vert_list[<= 2m]   distinct vertices per block, first touch
 *   relabel[nd]                       cpack new id of every data vertex
 *   stats[0] = loads (sum of |V_b|), stats[1] = vertex cut sum (p_v - 1),
 *   stats[2] = touched vertices
 * nd = n, or 2n when bipartite. */
int32_t orc_schedule(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                     uint32_t flags, const int32_t *part, int32_t k, int64_t *block_ptr,
                     int32_t *edge_perm, int64_t *vert_ptr, int32_t *vert_list, int32_t *relabel,
                     int64_t *stats) {
  int bip = (int)(flags & 1u);
  int64_t nd = bip ? 2 * n : n;
  if (check_edges(src, dst, m, n) || k <= 0) return -1;
  for (int64_t e = 0; e < m; e++)
    if (part[e] < 0 || part[e] >= k) return -1;
  memset(block_ptr, 0, (size_t)(k + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m; e++) block_ptr[part[e] + 1]++;
  for (int32_t b = 0; b < k; b++) block_ptr[b + 1] += block_ptr[b];
  int64_t *cur = malloc((size_t)(k + 1) * sizeof(int64_t));
  memcpy(cur, block_ptr, (size_t)k * sizeof(int64_t));
  for (int64_t e = 0; e < m; e++) edge_perm[cur[part[e]]++] = (int32_t)e;
  free(cur);
  /* vertex lists: last block that listed v */
  int32_t *mark = malloc((size_t)nd * sizeof(int32_t));
  for (int64_t v = 0; v < nd; v++) mark[v] = -1;
  int64_t loads = 0;
  vert_ptr[0] = 0;
  for (int32_t b = 0; b < k; b++) {
    for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; i++) {
      int64_t u, v;
      endpoints(src, dst, edge_perm[i], n, bip, &u, &v);
      if (mark[u] != b) {
        mark[u] = b;
        vert_list[loads++] = (int32_t)u;
      }
      if (mark[v] != b) {
        mark[v] = b;
        vert_list[loads++] = (int32_t)v;
      }
    }
    vert_ptr[b + 1] = loads;
  }
  /* cpack: first appearance over blocks in order */
  for (int64_t v = 0; v < nd; v++) relabel[v] = -1;
  int32_t next = 0;
  for (int64_t i = 0; i < loads; i++)
    if (relabel[vert_list[i]] < 0) relabel[vert_list[i]] = next++;
  int64_t touched = next;
  for (int64_t v = 0; v < nd; v++)
    if (relabel[v] < 0) relabel[v] = next++;
  free(mark);
  stats[0] = loads;
  stats[1] = loads - touched;
  stats[2] = touched;
  return 0;
}
