/*
 * kdt_oracle_fourier.c -- plain CPU reference for the paper's own split
 * estimator (TEST INFRASTRUCTURE, see kdt_oracle.h).
 *
 * Sec. 3.1, Lemma 1: on (0,1), away from a and b,
 *     1(a < x < b) = sum_{j >= 0} c_j(x) g_j(a, b)
 * with c_0 = 1, c_{2j-1}(x) = cos((2j-1)x), c_{2j}(x) = sin((2j-1)x) and
 *     g_0(a,b)      = 1 - (1(a>0) + 1(b<1)) / 2
 *     g_{2j-1}(a,b) = 2/(pi(2j-1)) (1(b<1) sin((2j-1)b) - 1(a>0) sin((2j-1)a))
 *     g_{2j}(a,b)   = 2/(pi(2j-1)) (1(a>0) cos((2j-1)a) - 1(b<1) cos((2j-1)b)),
 * truncated after j = 2J (the (2J)th partial sum 1_J).
 *
 * Sec. 3.2: the count of points in a box is approximated by
 * sum_j C_j g_j(a, b) with the additive statistics C_j = sum_i c_j(x_i),
 * which subsets compute separately and add (the map-reduce pattern); the
 * split m of a cell along its key coordinate t solves Eq. (kd:eq:b),
 *     1_J(X, a, b_{-t}(m)) = 1_J(X, a_{-t}(m), b),
 * i.e. the approximate counts on the two sides of m are equal.
 *
 * Readings (the paper leaves them open):
 *   - the statistics of a cell are summed over the cell's own points, so the
 *     factors of the other coordinates are exactly 1 and only the key
 *     coordinate's indicator is expanded (per-cell 1-D moments);
 *   - the root of Eq. (kd:eq:b) is found by bisection in double precision
 *     on (a_t, b_t), 60 halvings, keeping the half where
 *     F(m) = 1_J(a_t, m) - 1_J(m, b_t) changes sign (F < 0 moves the lower
 *     end up); the split is the midpoint of the last interval, rounded to
 *     float (m32), and a point goes left when its coordinate is <= m32;
 *   - a cell's bounds on a coordinate are the float splits of its ancestors
 *     on that coordinate ((0,1) at the root); keys cycle x, y, z, ... (Sec. 1);
 *   - every coordinate must lie in the open interval (0,1) (Sec. 2: the data
 *     are scaled there); an empty cell gets the sentinel split (+inf, -1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kdt_oracle.h"

static const double kPi = 3.14159265358979323846;

double kdto_fourier_c(int32_t j, double x) {
  if (j == 0) return 1.0;
  const double k = (double)(2 * ((j + 1) / 2) - 1); /* the odd harmonic 2j'-1 of term j */
  return (j & 1) ? cos(k * x) : sin(k * x);
}

double kdto_fourier_g(int32_t j, double a, double b) {
  const double ia = a > 0.0 ? 1.0 : 0.0, ib = b < 1.0 ? 1.0 : 0.0;
  if (j == 0) return 1.0 - 0.5 * (ia + ib);
  const double k = (double)(2 * ((j + 1) / 2) - 1);
  const double q = 2.0 / (kPi * k);
  if (j & 1) return q * (ib * sin(k * b) - ia * sin(k * a));
  return q * (ia * cos(k * a) - ib * cos(k * b));
}

int kdto_fourier_moments(const double *x, int64_t cnt, int32_t J, double *out) {
  if (J < 1 || J > KDTO_FOURIER_MAX_J || cnt < 0 || (cnt > 0 && !x) || !out) return KDTO_ERR_INVALID_ARG;
  for (int32_t j = 0; j <= 2 * J; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < cnt; ++i) s += kdto_fourier_c(j, x[i]);
    out[j] = s;
  }
  return KDTO_OK;
}

/* F(m) of the reading above, from the moments C_0..C_2J. */
static double fourier_f(const double *C, int32_t J, double a, double b, double m) {
  double f = 0.0;
  for (int32_t j = 0; j <= 2 * J; ++j) f += C[j] * (kdto_fourier_g(j, a, m) - kdto_fourier_g(j, m, b));
  return f;
}

int kdto_fourier_split(const double *x, int64_t cnt, double a, double b, int32_t J, double *out_m) {
  if (!out_m || !(a >= 0.0 && a < b && b <= 1.0)) return KDTO_ERR_INVALID_ARG;
  if (J < 1 || J > KDTO_FOURIER_MAX_J) return KDTO_ERR_INVALID_ARG;
  double *C = malloc((size_t)(2 * J + 1) * sizeof *C);
  if (!C) return KDTO_ERR_OOM;
  const int st = kdto_fourier_moments(x, cnt, J, C);
  if (st != KDTO_OK) { free(C); return st; }
  double lo = a, hi = b;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (fourier_f(C, J, a, b, mid) < 0.0) lo = mid;
    else hi = mid;
  }
  *out_m = 0.5 * (lo + hi);
  free(C);
  return KDTO_OK;
}

typedef struct {
  int64_t begin, count;
} fcell;

int kdto_fourier_build(const float *points, int64_t n, int32_t d, int32_t depth, int32_t J,
                       uint32_t *out_perm, float *out_split_vals, int8_t *out_split_dims,
                       int64_t *out_node_offsets) {
  if (n < 0 || n > (int64_t)0xffffffffLL || d < 1 || d > 64 || depth < 1 || depth > KDTO_MAX_LEVELS ||
      J < 1 || J > KDTO_FOURIER_MAX_J || (n > 0 && (!points || !out_perm)) || !out_split_vals ||
      !out_split_dims || !out_node_offsets)
    return KDTO_ERR_INVALID_ARG;
  for (int64_t j = 0; j < (int64_t)d * n; ++j) {
    if (isnan(points[j])) return KDTO_ERR_NAN_INPUT;
    if (!(points[j] > 0.0f && points[j] < 1.0f)) return KDTO_ERR_INVALID_ARG;
  }
  int st = KDTO_OK;
  int64_t *order = malloc((size_t)(n > 0 ? n : 1) * sizeof *order);
  int64_t *scratch = malloc((size_t)(n > 0 ? n : 1) * sizeof *scratch);
  double *xs = malloc((size_t)(n > 0 ? n : 1) * sizeof *xs);
  fcell *cells = malloc(sizeof *cells);
  if (!order || !scratch || !xs || !cells) { st = KDTO_ERR_OOM; goto done; }
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  cells[0].begin = 0;
  cells[0].count = n;

  for (int32_t level = 0; level < depth; ++level) {
    const int64_t ncell = (int64_t)1 << level;
    const int32_t t = level % d;
    fcell *next = malloc((size_t)(2 * ncell) * sizeof *next);
    if (!next) { st = KDTO_ERR_OOM; goto done; }
    for (int64_t k = 0; k < ncell; ++k) {
      const fcell *c = &cells[k];
      const int64_t heap = ncell - 1 + k;
      fcell *lc = &next[2 * k], *rc = &next[2 * k + 1];
      if (c->count == 0) {
        out_split_dims[heap] = -1;
        out_split_vals[heap] = INFINITY;
        *lc = *c;
        *rc = *c;
        continue;
      }
      /* bounds on coordinate t: the float splits of the ancestors on t */
      double a = 0.0, b = 1.0;
      for (int64_t h = heap; h > 0;) {
        const int64_t par = (h - 1) / 2;
        int32_t plevel = 0;
        while (((int64_t)1 << (plevel + 1)) - 1 <= par) ++plevel;
        if (plevel % d == t) {
          const double v = (double)out_split_vals[par];
          if (h == 2 * par + 1) { if (v < b) b = v; }
          else if (v > a) a = v;
        }
        h = par;
      }
      int64_t *idx = order + c->begin;
      for (int64_t i = 0; i < c->count; ++i) xs[i] = (double)points[(int64_t)t * n + idx[i]];
      double m;
      st = kdto_fourier_split(xs, c->count, a, b, J, &m);
      if (st != KDTO_OK) { free(next); goto done; }
      const float m32 = (float)m;
      int64_t nl = 0, nr = 0;
      for (int64_t i = 0; i < c->count; ++i)
        if (points[(int64_t)t * n + idx[i]] <= m32) idx[nl++] = idx[i];
        else scratch[nr++] = idx[i];
      memcpy(idx + nl, scratch, (size_t)nr * sizeof *idx);
      out_split_dims[heap] = (int8_t)t;
      out_split_vals[heap] = m32;
      lc->begin = c->begin;
      lc->count = nl;
      rc->begin = c->begin + nl;
      rc->count = nr;
    }
    free(cells);
    cells = next;
  }
  {
    const int64_t nleaf = (int64_t)1 << depth;
    for (int64_t k = 0; k < nleaf; ++k) out_node_offsets[k] = cells[k].begin;
    out_node_offsets[nleaf] = n;
    for (int64_t i = 0; i < n; ++i) out_perm[i] = (uint32_t)order[i];
  }
done:
  free(order);
  free(scratch);
  free(xs);
  free(cells);
  return st;
}
