/*
 * kdt_oracle.h -- plain, slow, single-threaded CPU reference for the
 * level-by-level k-d tree build with subset-median splits.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA library; the status numbers below
 * are restated here on purpose so that neither side includes the other.
 *
 * What it computes (paper: "Scalable k-d trees for distributed data"):
 *   - the canonical k-d tree of depth D: level l splits each of its 2^l cells
 *     at a median of the key coordinate, giving 2^D - 1 split statistics in
 *     level order (Sec. 1, Fig. 1; Sec. 2, last paragraph);
 *   - keys cycle x, y, z, ... (Sec. 1) or, per cell, the coordinate of
 *     widest dispersion (Sec. 1, the Friedman rule), read as the range;
 *   - the data index set is partitioned into R subsets (Sec. 3.2, the
 *     additivity remark; App. C.2) and each subset contributes a summary that
 *     is combined per cell. Here the per-subset summary is the lower median
 *     and the combination is the count-weighted lower median of those
 *     medians (the project's rule; the paper combines additive moments).
 *
 * Status codes (same numbering as the product's public header).
 */
#ifndef KDT_ORACLE_H
#define KDT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  KDTO_OK = 0,
  KDTO_ERR_INVALID_ARG = 1,
  KDTO_ERR_NAN_INPUT = 2,
  KDTO_ERR_OOM = 3,
  KDTO_ERR_LEVEL_CAP = 7
};

enum { KDTO_KEY_CYCLIC = 0, KDTO_KEY_WIDEST_SPREAD = 1 };
enum { KDTO_SUBSET_MOD = 0, KDTO_SUBSET_CONTIGUOUS = 1, KDTO_SUBSET_EXPLICIT = 2 };

/* Largest depth / level count the oracle accepts (outputs hold 2^L + 1 offsets). */
#define KDTO_MAX_LEVELS 30

typedef struct {
  int64_t n;               /* number of points, 0 <= n <= 2^32 - 1               */
  int32_t d;               /* dimensions, 1..64                                   */
  int32_t subset_mode;     /* KDTO_SUBSET_*                                       */
  int32_t r;               /* number of subsets, 1..65536                         */
  const uint8_t *sid8;     /* explicit mode: one of sid8 / sid16 (host, length n) */
  const uint16_t *sid16;
  int32_t depth;           /* > 0: fixed depth; 0: leaf mode                      */
  int32_t leaf_size;       /* leaf mode: cells with count <= leaf_size terminate  */
  int32_t max_levels;      /* leaf mode: cap on the number of split levels        */
  int32_t key_rule;        /* KDTO_KEY_*                                          */
  int32_t combine;         /* KDTO_COMBINE_*                                      */
} kdto_params;

/* How a cell's split is formed from its subsets' lower medians (R2 / R2u). */
enum { KDTO_COMBINE_WEIGHTED = 0, KDTO_COMBINE_UNWEIGHTED = 1 };

/* Order-preserving float -> uint32 key and its inverse. */
uint32_t kdto_key(float x);
float kdto_key_value(uint32_t key);

/*
 * Full build. points: host SoA, points[j*n + i] = coordinate j of point i.
 * Outputs (host, caller-allocated): out_perm[n]; out_split_vals and
 * out_split_dims[2^L - 1] in level order (children of node h are 2h+1, 2h+2);
 * out_node_offsets[2^L + 1] (CSR of the 2^L leaves over out_perm);
 * *out_levels = L. Capacity: L <= depth (depth mode) or <= max_levels.
 */
int kdto_build(const float *points, const kdto_params *p, uint32_t *out_perm,
               float *out_split_vals, int8_t *out_split_dims,
               int64_t *out_node_offsets, int32_t *out_levels);

/*
 * The split of one cell: idx[0..cnt) are the original indices of the cell's
 * points (any order). level is the cell's 0-based level (selects the cyclic
 * key). Writes the key dimension, the split key and its float value, and the
 * number of points with key <= split (the left child's size). For cnt == 0
 * writes dim -1, the key of +inf, value +inf, left 0.
 */
int kdto_split_cell(const float *points, const kdto_params *p, const int64_t *idx,
                    int64_t cnt, int32_t level, int32_t *out_dim,
                    uint32_t *out_key, float *out_val, int64_t *out_left);

/* ---- the paper's Fourier-moment estimator (kdt_oracle_fourier.c) ------- */

/* Largest number of harmonics J (terms c_0 .. c_2J) the oracle accepts. */
#define KDTO_FOURIER_MAX_J 4096

/* Basis term c_j(x) and coefficient g_j(a, b) of Lemma 1 (Sec. 3.1). */
double kdto_fourier_c(int32_t j, double x);
double kdto_fourier_g(int32_t j, double a, double b);
/* out[j] = sum_i c_j(x[i]) for j = 0..2J: the additive statistics of Sec. 3.2. */
int kdto_fourier_moments(const double *x, int64_t cnt, int32_t J, double *out);
/*
 * Root of Eq. (kd:eq:b) on (a, b) for the values x[0..cnt) of the cell's key
 * coordinate: bisection of F(m) = 1_J(a, m) - 1_J(m, b) (60 halvings, double),
 * *out_m the midpoint of the last interval. Requires 0 <= a < b <= 1.
 */
int kdto_fourier_split(const double *x, int64_t cnt, double a, double b, int32_t J, double *out_m);
/*
 * Depth-D tree with cyclic keys whose splits are the estimator's roots
 * rounded to float; points with coordinate <= split go left (stable).
 * Every coordinate must lie in (0,1). Outputs as for kdto_build with L = depth.
 */
int kdto_fourier_build(const float *points, int64_t n, int32_t d, int32_t depth, int32_t J,
                       uint32_t *out_perm, float *out_split_vals, int8_t *out_split_dims,
                       int64_t *out_node_offsets);

#ifdef __cplusplus
}
#endif
#endif
