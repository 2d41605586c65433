/*
 * cpu_fair.c -- a multi-threaded FP64 CPU implementation of the explicit
 * flux steps, for the bench's CPU context line ("what all host cores do").
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by the CPU-baseline
 * leg of bench.py and by its own test against the NumPy oracle.  It is not the
 * oracle (which stays the plain serial definition) and shares no code with the
 * CUDA library.
 *
 * One step computes, for every data vertex v, out_v = sum over the tasks
 * e = (u, v') touching v of +f_e (v is the source u) or -f_e (v is the
 * target v'), with f_e = w_e d / (1 + |d|^2), d = x_{v'} - x_u (the edge
 * interaction of Section 1's cfd example), then x <- x + tau * out.  Vertices
 * are split over OpenMP threads and each thread sums its vertices' tasks from
 * a vertex-to-task list built once (so no two threads write the same vertex).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  int64_t n, m;
  int32_t D;
  int64_t *off;  /* n + 1 */
  int32_t *task; /* 2m (self loops once) */
} fair_t;

/* Vertex-to-task lists; returns an opaque handle or NULL. */
void *fair_build(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t D) {
  if (D < 1 || D > 8 || m <= 0 || n <= 0) return NULL;
  fair_t *f = calloc(1, sizeof(fair_t));
  if (!f) return NULL;
  f->n = n;
  f->m = m;
  f->D = D;
  f->off = calloc((size_t)n + 1, sizeof(int64_t));
  f->task = malloc((size_t)(2 * m) * sizeof(int32_t));
  if (!f->off || !f->task) {
    free(f->off);
    free(f->task);
    free(f);
    return NULL;
  }
  for (int64_t e = 0; e < m; e++) {
    f->off[src[e] + 1]++;
    if (dst[e] != src[e]) f->off[dst[e] + 1]++;
  }
  for (int64_t v = 0; v < n; v++) f->off[v + 1] += f->off[v];
  int64_t *fill = malloc((size_t)n * sizeof(int64_t));
  if (!fill) {
    free(f->off);
    free(f->task);
    free(f);
    return NULL;
  }
  for (int64_t v = 0; v < n; v++) fill[v] = f->off[v];
  for (int64_t e = 0; e < m; e++) {
    f->task[fill[src[e]]++] = (int32_t)e;
    if (dst[e] != src[e]) f->task[fill[dst[e]]++] = (int32_t)e;
  }
  free(fill);
  return f;
}

void fair_free(void *h) {
  fair_t *f = h;
  if (!f) return;
  free(f->off);
  free(f->task);
  free(f);
}

/* `steps` explicit steps on x[D][n] (in place) using `threads` threads
 * (<= 0: the OpenMP default); out[D][n] is scratch that ends holding
 * flux(x_{T-1}).  Returns the number of threads used. */
int fair_steps(void *h, const int32_t *src, const int32_t *dst, const double *w, double *x,
               double *out, int32_t steps, double tau, int32_t threads) {
  fair_t *f = h;
  const int64_t n = f->n;
  const int D = f->D;
  int used = 1;
  for (int t = 0; t < steps; t++) {
#pragma omp parallel num_threads(threads > 0 ? threads : omp_get_max_threads())
    {
#pragma omp single
      used = omp_get_num_threads();
#pragma omp for schedule(static)
      for (int64_t v = 0; v < n; v++) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = f->off[v]; j < f->off[v + 1]; j++) {
          const int32_t e = f->task[j];
          const int64_t a = src[e], b = dst[e];
          double d[8], s = 0.0;
          for (int c = 0; c < D; c++) {
            d[c] = x[c * n + b] - x[c * n + a];
            s += d[c] * d[c];
          }
          const double g = w[e] / (1.0 + s) * (a == v ? 1.0 : -1.0);
          for (int c = 0; c < D; c++) acc[c] += g * d[c];
        }
        for (int c = 0; c < D; c++) out[c * n + v] = acc[c];
      }
#pragma omp for schedule(static)
      for (int64_t i = 0; i < (int64_t)D * n; i++) x[i] += tau * out[i];
    }
  }
  return used;
}
