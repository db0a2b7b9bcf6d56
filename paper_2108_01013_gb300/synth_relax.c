/*
 * Seeded synthetic packings for the benchmark and the tests: random
 * sequential insertion (largest first) into a periodic box, random placement
 * of whatever could not be inserted, then Jacobi overlap-removal sweeps.
 *
 * This file holds none of the suspension model's arithmetic: it only places
 * spheres so that they barely overlap.  Both the CUDA path and the oracle
 * read the arrays it produces.  Deterministic for a given seed on any
 * machine and thread count: every random draw comes from a counter-based
 * splitmix64 stream, and every sweep accumulates each particle's
 * displacement in a fixed neighbour order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* splitmix64 (Steele, Lea, Flood 2014) evaluated at counter k of stream seed */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double urand(uint64_t seed, uint64_t k) {
  uint64_t z = mix64(seed * 0x9E3779B97F4A7C15ULL + (k + 1) * 0xD1B54A32D192ED03ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct grid {
  int nc[3];
  double cs[3];
  int64_t ncell;
  int64_t *head;   /* cell -> first particle, -1 terminated */
  int64_t *next;
} grid;

static int64_t cell_of(const grid *g, const double L[3], double x, double y, double z) {
  int c[3];
  double p[3] = {x, y, z};
  for (int d = 0; d < 3; ++d) {
    int k = (int)floor(p[d] / g->cs[d]);
    if (k < 0) k = 0;
    if (k >= g->nc[d]) k = g->nc[d] - 1;
    c[d] = k;
  }
  (void)L;
  return ((int64_t)c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
}

static void grid_init(grid *g, const double L[3], double cmin, int64_t n) {
  for (int d = 0; d < 3; ++d) {
    g->nc[d] = (int)floor(L[d] / cmin);
    if (g->nc[d] < 3) g->nc[d] = 3;
    g->cs[d] = L[d] / g->nc[d];
  }
  g->ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
  g->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)g->ncell);
  g->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t c = 0; c < g->ncell; ++c) g->head[c] = -1;
}

static void grid_free(grid *g) { free(g->head); free(g->next); }

static double wrapd(double v, double L) {
  v = fmod(v, L);
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

static double pdist2(const double L[3], const double *pi, const double *pj) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double dd = pj[d] - pi[d];
    dd -= L[d] * rint(dd / L[d]);
    s += dd * dd;
  }
  return s;
}

/* Visit the 27 cells around cell (cx,cy,cz), periodic, each once even when
 * the grid has exactly 3 cells along an axis. */
#define FOR_NEIGHBOUR_CELLS(g, cx, cy, cz, ...)                                 \
  for (int oz = -1; oz <= 1; ++oz)                                               \
    for (int oy = -1; oy <= 1; ++oy)                                             \
      for (int ox = -1; ox <= 1; ++ox) {                                         \
        int qx = ((cx) + ox + (g)->nc[0]) % (g)->nc[0];                          \
        int qy = ((cy) + oy + (g)->nc[1]) % (g)->nc[1];                          \
        int qz = ((cz) + oz + (g)->nc[2]) % (g)->nc[2];                          \
        int64_t qc = ((int64_t)qz * (g)->nc[1] + qy) * (g)->nc[0] + qx;          \
        __VA_ARGS__                                                              \
      }

/*
 * Place n spheres of radii a (already ordered largest first by the caller)
 * in the box L.  x is SoA (3,n) output.  Returns the number placed without
 * overlap by insertion.
 */
int64_t synth_insert(int64_t n, const double *a, const double L[3], uint64_t seed,
                     int tries, double *x) {
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) amax = a[i] > amax ? a[i] : amax;
  grid g;
  grid_init(&g, L, 2.0 * amax, n);
  int64_t placed = 0;
  uint64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    int ok = 0;
    double p[3];
    for (int t = 0; t < tries && !ok; ++t) {
      p[0] = urand(seed, k++) * L[0];
      p[1] = urand(seed, k++) * L[1];
      p[2] = urand(seed, k++) * L[2];
      for (int d = 0; d < 3; ++d) if (p[d] >= L[d]) p[d] = 0.0;
      int64_t c = cell_of(&g, L, p[0], p[1], p[2]);
      int cx = (int)(c % g.nc[0]), cy = (int)((c / g.nc[0]) % g.nc[1]), cz = (int)(c / ((int64_t)g.nc[0] * g.nc[1]));
      ok = 1;
      FOR_NEIGHBOUR_CELLS(&g, cx, cy, cz, {
        for (int64_t j = g.head[qc]; j >= 0 && ok; j = g.next[j]) {
          double pj[3] = {x[j], x[n + j], x[2 * n + j]};
          double s = a[i] + a[j];
          if (pdist2(L, p, pj) < s * s) ok = 0;
        }
      })
    }
    if (!ok) {
      p[0] = urand(seed, k++) * L[0];
      p[1] = urand(seed, k++) * L[1];
      p[2] = urand(seed, k++) * L[2];
      for (int d = 0; d < 3; ++d) if (p[d] >= L[d]) p[d] = 0.0;
    } else {
      ++placed;
    }
    x[i] = p[0]; x[n + i] = p[1]; x[2 * n + i] = p[2];
    int64_t c = cell_of(&g, L, p[0], p[1], p[2]);
    g.next[i] = g.head[c];
    g.head[c] = i;
  }
  grid_free(&g);
  return placed;
}

/*
 * Jacobi overlap removal: every sweep moves each particle away from each
 * overlapping neighbour by a share of the overlap (the smaller particle
 * moves more), all moves computed from the same positions.  Stops when the
 * largest overlap is below tol or after max_iter sweeps.  Returns the number
 * of sweeps; *max_overlap receives the final largest overlap.
 */
int synth_relax(int64_t n, double *x, const double *a, const double L[3], int max_iter,
                double tol, double step, double *max_overlap) {
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) amax = a[i] > amax ? a[i] : amax;
  grid g;
  grid_init(&g, L, 2.0 * amax, n);
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g.ncell + 1));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double *disp = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double mo = 0.0;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    /* bucket particles by cell, in index order within a cell */
    memset(start, 0, sizeof(int64_t) * (size_t)(g.ncell + 1));
    for (int64_t i = 0; i < n; ++i) {
      cell[i] = cell_of(&g, L, x[i], x[n + i], x[2 * n + i]);
      start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < g.ncell; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < g.ncell; ++c) g.head[c] = start[c];
    for (int64_t i = 0; i < n; ++i) order[g.head[cell[i]]++] = i;
    mo = 0.0;
#pragma omp parallel for schedule(static) reduction(max : mo)
    for (int64_t i = 0; i < n; ++i) {
      double pi[3] = {x[i], x[n + i], x[2 * n + i]};
      double di[3] = {0.0, 0.0, 0.0};
      int64_t c = cell[i];
      int cx = (int)(c % g.nc[0]), cy = (int)((c / g.nc[0]) % g.nc[1]), cz = (int)(c / ((int64_t)g.nc[0] * g.nc[1]));
      FOR_NEIGHBOUR_CELLS(&g, cx, cy, cz, {
        for (int64_t q = start[qc]; q < start[qc + 1]; ++q) {
          int64_t j = order[q];
          if (j == i) continue;
          double r[3];
          for (int d = 0; d < 3; ++d) {
            r[d] = x[d * n + j] - pi[d];
            r[d] -= L[d] * rint(r[d] / L[d]);
          }
          double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
          double s = a[i] + a[j];
          if (r2 >= s * s) continue;
          double rr = sqrt(r2);
          double o = s - rr;
          if (o > mo) mo = o;
          double w = a[j] * a[j] * a[j] / (a[i] * a[i] * a[i] + a[j] * a[j] * a[j]);
          if (rr > 1e-12) {
            for (int d = 0; d < 3; ++d) di[d] -= step * w * o * r[d] / rr;
          } else {
            di[0] -= step * w * o;
          }
        }
      })
      disp[i] = di[0]; disp[n + i] = di[1]; disp[2 * n + i] = di[2];
    }
    if (mo < tol) break;
    for (int64_t i = 0; i < n; ++i)
      for (int d = 0; d < 3; ++d) x[d * n + i] = wrapd(x[d * n + i] + disp[d * n + i], L[d]);
  }
  *max_overlap = mo;
  free(cell); free(start); free(order); free(disp);
  grid_free(&g);
  return it;
}
