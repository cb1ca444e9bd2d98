/*
 * kdt_oracle.c -- plain, slow, single-threaded CPU reference build.
 *
 * TEST INFRASTRUCTURE: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. It is written for
 * a reader checking it against the paper, not for speed: every cell sorts
 * copies of its keys, the combine sorts its (median, subset) pairs, and the
 * partition copies through a scratch array.
 *
 * Paper: A. Chakravorty, W. S. Cleveland, P. J. Wolfe, "Scalable k-d trees
 * for distributed data" (arXiv 2201.08288).
 *
 * Readings of the paper that this file fixes (each is listed with its reason
 * in the design notes of the repository):
 *   R1  per-subset statistic: the lower median, 0-based rank (w-1)/2 of the
 *       subset's keys in the cell (Sec. 2 defines "the median" of a cell
 *       without fixing even counts);
 *   R2  combine: sort the non-empty (median, subset) pairs by key, ties by
 *       subset id; the split is the key of the first pair whose cumulative
 *       point count c satisfies 2c >= W, W the cell size (the project's rule;
 *       the paper's per-subset summaries are additive moments, Sec. 3.2);
 *   R3  ties go left: key <= split is the left child, key > split the right
 *       (Sec. 2 uses open cells and discards boundary points; here every
 *       point is kept);
 *   R4  order: keys are compared through the order-preserving uint32 map
 *       below, so -0.0 < +0.0; the partition is stable;
 *   R5  an empty cell (depth mode) records dim -1, value +inf;
 *   R6  levels are 0-based: depth D gives levels 0..D-1 and 2^D leaves;
 *   R7  widest spread = the range (double)max - (double)min of the cell's
 *       points per coordinate (0 when max and min are the same key); the
 *       lowest coordinate wins ties (Sec. 1, widest-dispersion rule);
 *   R2u (combine = KDTO_COMBINE_UNWEIGHTED) every non-empty subset counts
 *       once: the split is the lower median, rank (m-1)/2 in (key, subset)
 *       order, of the m subset medians (the plain median of medians);
 *   R8  leaf mode: a cell is terminal when it holds <= leaf_size points, or
 *       when its last s splits each left the right child empty, s = d for
 *       cyclic keys and s = 1 for widest spread (its point set can no longer
 *       change). Terminal cells record dim -1, value +inf and pass all their
 *       points to the left child. L is the first level whose cells are all
 *       terminal.
 */
#include "kdt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- order-preserving key (Sec. 1: keys are compared as reals) ---------- */

uint32_t kdto_key(float x) {
  uint32_t u;
  memcpy(&u, &x, sizeof u);
  if (u & 0x80000000u) return ~u;      /* negative: reverse the order      */
  return u | 0x80000000u;              /* non-negative: above every negative */
}

float kdto_key_value(uint32_t key) {
  uint32_t u = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
  float x;
  memcpy(&x, &u, sizeof x);
  return x;
}

/* ---- subset membership (Sec. 3.2: a partition of I into R subsets) ------ */

static int32_t subset_of(const kdto_params *p, int64_t i) {
  switch (p->subset_mode) {
  case KDTO_SUBSET_MOD:
    return (int32_t)(i % p->r);
  case KDTO_SUBSET_CONTIGUOUS:
    return (int32_t)(((uint64_t)i * (uint64_t)p->r) / (uint64_t)p->n);
  default:
    return p->sid8 ? (int32_t)p->sid8[i] : (int32_t)p->sid16[i];
  }
}

static int validate(const float *points, const kdto_params *p) {
  if (!p) return KDTO_ERR_INVALID_ARG;
  if (p->n < 0 || p->n > (int64_t)0xffffffffLL) return KDTO_ERR_INVALID_ARG;
  if (p->d < 1 || p->d > 64) return KDTO_ERR_INVALID_ARG;
  if (p->r < 1 || p->r > 65536) return KDTO_ERR_INVALID_ARG;
  if (p->key_rule != KDTO_KEY_CYCLIC && p->key_rule != KDTO_KEY_WIDEST_SPREAD)
    return KDTO_ERR_INVALID_ARG;
  if (p->combine != KDTO_COMBINE_WEIGHTED && p->combine != KDTO_COMBINE_UNWEIGHTED)
    return KDTO_ERR_INVALID_ARG;
  if (p->depth < 0 || p->depth > KDTO_MAX_LEVELS) return KDTO_ERR_INVALID_ARG;
  if (p->depth == 0) {
    if (p->leaf_size < 1) return KDTO_ERR_INVALID_ARG;
    if (p->max_levels < 0 || p->max_levels > KDTO_MAX_LEVELS) return KDTO_ERR_INVALID_ARG;
  }
  if (p->n > 0 && !points) return KDTO_ERR_INVALID_ARG;
  if (p->subset_mode == KDTO_SUBSET_EXPLICIT) {
    if (p->n > 0 && ((p->sid8 == NULL) == (p->sid16 == NULL))) return KDTO_ERR_INVALID_ARG;
    for (int64_t i = 0; i < p->n; ++i)
      if (subset_of(p, i) >= p->r) return KDTO_ERR_INVALID_ARG;
  } else if (p->subset_mode != KDTO_SUBSET_MOD && p->subset_mode != KDTO_SUBSET_CONTIGUOUS) {
    return KDTO_ERR_INVALID_ARG;
  }
  for (int64_t j = 0; j < (int64_t)p->d * p->n; ++j)
    if (isnan(points[j])) return KDTO_ERR_NAN_INPUT;
  return KDTO_OK;
}

/* ---- one cell's split ---------------------------------------------------- */

typedef struct { int32_t sid; uint32_t key; } sid_key;
typedef struct { uint32_t key; int32_t sid; int64_t w; } med_pair;

static int cmp_sid_key(const void *a, const void *b) {
  const sid_key *x = a, *y = b;
  if (x->sid != y->sid) return x->sid < y->sid ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return 0;
}

static int cmp_med_pair(const void *a, const void *b) {
  const med_pair *x = a, *y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->sid != y->sid) return x->sid < y->sid ? -1 : 1;
  return 0;
}

/* Key coordinate of a cell: cyclic x, y, z, ... by level, or widest range (R7). */
static int32_t key_dim(const float *pts, const kdto_params *p, const int64_t *idx,
                       int64_t cnt, int32_t level) {
  if (p->key_rule == KDTO_KEY_CYCLIC) return level % p->d;
  int32_t best = 0;
  double best_range = -1.0;
  for (int32_t l = 0; l < p->d; ++l) {
    uint32_t lo = 0xffffffffu, hi = 0;
    for (int64_t i = 0; i < cnt; ++i) {
      uint32_t k = kdto_key(pts[(int64_t)l * p->n + idx[i]]);
      if (k < lo) lo = k;
      if (k > hi) hi = k;
    }
    double range = (lo == hi) ? 0.0
                              : (double)kdto_key_value(hi) - (double)kdto_key_value(lo);
    if (range > best_range) { best_range = range; best = l; }
  }
  return best;
}

/*
 * Split key of a non-empty cell along coordinate t:
 *   1. per subset s, the lower median of the keys of the cell's points in s (R1);
 *   2. the count-weighted lower median of those medians (R2).
 */
static int split_key(const float *pts, const kdto_params *p, const int64_t *idx,
                     int64_t cnt, int32_t t, uint32_t *out_key) {
  sid_key *sk = malloc((size_t)cnt * sizeof *sk);
  med_pair *mp = malloc((size_t)cnt * sizeof *mp);
  if (!sk || !mp) { free(sk); free(mp); return KDTO_ERR_OOM; }
  for (int64_t i = 0; i < cnt; ++i) {
    sk[i].sid = subset_of(p, idx[i]);
    sk[i].key = kdto_key(pts[(int64_t)t * p->n + idx[i]]);
  }
  qsort(sk, (size_t)cnt, sizeof *sk, cmp_sid_key);

  /* step 1: runs of equal subset id; the run is sorted by key */
  int64_t npairs = 0;
  for (int64_t b = 0; b < cnt;) {
    int64_t e = b;
    while (e < cnt && sk[e].sid == sk[b].sid) ++e;
    int64_t w = e - b;
    mp[npairs].key = sk[b + (w - 1) / 2].key;
    mp[npairs].sid = sk[b].sid;
    mp[npairs].w = w;
    ++npairs;
    b = e;
  }

  /* step 2: first pair in (key, sid) order whose cumulative count reaches
   * half (R2), or the pair at rank (npairs-1)/2 when every subset counts once (R2u) */
  qsort(mp, (size_t)npairs, sizeof *mp, cmp_med_pair);
  uint32_t chosen = mp[npairs - 1].key;
  if (p->combine == KDTO_COMBINE_UNWEIGHTED) {
    chosen = mp[(npairs - 1) / 2].key;
  } else {
    int64_t cum = 0;
    for (int64_t j = 0; j < npairs; ++j) {
      cum += mp[j].w;
      if (2 * cum >= cnt) { chosen = mp[j].key; break; }
    }
  }
  *out_key = chosen;
  free(sk);
  free(mp);
  return KDTO_OK;
}

int kdto_split_cell(const float *points, const kdto_params *p, const int64_t *idx,
                    int64_t cnt, int32_t level, int32_t *out_dim, uint32_t *out_key,
                    float *out_val, int64_t *out_left) {
  int st = validate(points, p);
  if (st != KDTO_OK) return st;
  if (cnt < 0 || (cnt > 0 && !idx)) return KDTO_ERR_INVALID_ARG;
  for (int64_t i = 0; i < cnt; ++i)
    if (idx[i] < 0 || idx[i] >= p->n) return KDTO_ERR_INVALID_ARG;
  if (cnt == 0) {
    *out_dim = -1;
    *out_key = kdto_key(INFINITY);
    *out_val = INFINITY;
    *out_left = 0;
    return KDTO_OK;
  }
  int32_t t = key_dim(points, p, idx, cnt, level);
  uint32_t m;
  st = split_key(points, p, idx, cnt, t, &m);
  if (st != KDTO_OK) return st;
  int64_t left = 0;
  for (int64_t i = 0; i < cnt; ++i)
    if (kdto_key(points[(int64_t)t * p->n + idx[i]]) <= m) ++left;
  *out_dim = t;
  *out_key = m;
  *out_val = kdto_key_value(m);
  *out_left = left;
  return KDTO_OK;
}

/* ---- the level-by-level build ------------------------------------------ */

typedef struct {
  int64_t begin, count;
  int32_t stall; /* consecutive splits on this path that left the right child empty */
} cell;

int kdto_build(const float *points, const kdto_params *p, uint32_t *out_perm,
               float *out_split_vals, int8_t *out_split_dims,
               int64_t *out_node_offsets, int32_t *out_levels) {
  int st = validate(points, p);
  if (st != KDTO_OK) return st;
  if ((p->n > 0 && !out_perm) || !out_node_offsets || !out_levels)
    return KDTO_ERR_INVALID_ARG;

  const int64_t n = p->n;
  const int leaf_mode = (p->depth == 0);
  const int32_t stall_limit = (p->key_rule == KDTO_KEY_CYCLIC) ? p->d : 1;

  int64_t *order = malloc((size_t)(n > 0 ? n : 1) * sizeof *order);
  int64_t *scratch = malloc((size_t)(n > 0 ? n : 1) * sizeof *scratch);
  cell *cells = malloc(sizeof *cells);
  if (!order || !scratch || !cells) { st = KDTO_ERR_OOM; goto done; }
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  cells[0].begin = 0;
  cells[0].count = n;
  cells[0].stall = 0;

  int32_t level = 0;
  for (;;) {
    const int64_t ncell = (int64_t)1 << level;
    /* is every cell of this level terminal? */
    int all_terminal = 1;
    for (int64_t k = 0; k < ncell; ++k) {
      const cell *c = &cells[k];
      int term = leaf_mode ? (c->count <= p->leaf_size || c->stall >= stall_limit)
                           : (c->count == 0);
      if (!term) { all_terminal = 0; break; }
    }
    if (leaf_mode ? all_terminal : (level == p->depth)) break;
    if (leaf_mode && level == p->max_levels) { st = KDTO_ERR_LEVEL_CAP; goto done; }

    cell *next = malloc((size_t)(2 * ncell) * sizeof *next);
    if (!next) { st = KDTO_ERR_OOM; goto done; }
    for (int64_t k = 0; k < ncell; ++k) {
      const cell *c = &cells[k];
      const int64_t heap = ncell - 1 + k;
      int term = leaf_mode ? (c->count <= p->leaf_size || c->stall >= stall_limit)
                           : (c->count == 0);
      cell *lc = &next[2 * k], *rc = &next[2 * k + 1];
      if (term) {
        /* R5/R8: sentinel split, every point stays in the left child */
        out_split_dims[heap] = -1;
        out_split_vals[heap] = INFINITY;
        *lc = *c;
        rc->begin = c->begin + c->count;
        rc->count = 0;
        rc->stall = c->stall;
        continue;
      }
      int64_t *idx = order + c->begin;
      int32_t t = key_dim(points, p, idx, c->count, level);
      uint32_t m;
      st = split_key(points, p, idx, c->count, t, &m);
      if (st != KDTO_OK) { free(next); goto done; }
      /* R3/R4: stable partition, key <= m to the left */
      int64_t nl = 0, nr = 0;
      for (int64_t i = 0; i < c->count; ++i)
        if (kdto_key(points[(int64_t)t * n + idx[i]]) <= m) idx[nl++] = idx[i];
        else scratch[nr++] = idx[i];
      memcpy(idx + nl, scratch, (size_t)nr * sizeof *idx);
      out_split_dims[heap] = (int8_t)t;
      out_split_vals[heap] = kdto_key_value(m);
      int32_t stall = (nr == 0) ? c->stall + 1 : 0;
      lc->begin = c->begin;
      lc->count = nl;
      lc->stall = stall;
      rc->begin = c->begin + nl;
      rc->count = nr;
      rc->stall = stall;
    }
    free(cells);
    cells = next;
    ++level;
  }

  {
    const int64_t nleaf = (int64_t)1 << level;
    for (int64_t k = 0; k < nleaf; ++k) out_node_offsets[k] = cells[k].begin;
    out_node_offsets[nleaf] = n;
    for (int64_t i = 0; i < n; ++i) out_perm[i] = (uint32_t)order[i];
    *out_levels = level;
  }

done:
  free(order);
  free(scratch);
  free(cells);
  return st;
}
