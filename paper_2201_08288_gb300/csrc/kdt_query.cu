// kdt_query.cu -- queries on a built tree: boxes (range counts and lists) and
// k nearest neighbours.
//
// The paper motivates the k-d tree by the searches it speeds up (Sec. 1): a
// query visits only the cells its region can reach. A node h at level l < L
// with dim t >= 0 sends keys <= its split key to the left child and the
// others to the right (the build's rule, in the total order of the key
// transform, -0 below +0); a node with dim -1 (an empty or terminal cell)
// has all of its points in its leftmost leaf. Leaf k holds
// perm[offs[k] .. offs[k+1]).
//
// One thread per query, depth-first with an explicit stack of at most L + 1
// nodes.
//   Box: a point is inside when lo_j <= x_j <= hi_j for every coordinate j,
//   compared as keys; the left child is visited when key(lo_t) <= split key,
//   the right when key(hi_t) > split key.
//   Nearest: squared distances in double, summed over j = 0..d-1 in order
//   with no fused multiply-add, so that the value is a fixed function of the
//   inputs; ties go to the smaller original index. The nearer child is
//   visited first; the farther one is skipped when the squared distance to
//   the split plane exceeds the current k-th distance (a lower bound on
//   every point beyond the plane, because rounding to nearest is monotone).
#include <algorithm>

#include "kdt.h"
#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int kQueryThreads = 128;

struct TreeView {
  const float* x;  // [d][n]
  int64_t n;
  int32_t d, L;
  const uint32_t* perm;
  const float* vals;
  const int8_t* dims;
  const int64_t* offs;
};

// Leaf range of node h at level l: the leaves below it.
__device__ __forceinline__ void node_leaves(const TreeView& tv, uint32_t h, int l, uint32_t* k0, uint32_t* k1) {
  const uint32_t k = h - ((1u << l) - 1u);
  *k0 = k << (tv.L - l);
  *k1 = (k + 1u) << (tv.L - l);
}

__global__ void __launch_bounds__(kQueryThreads) k_query_box(TreeView tv, const float* lo, const float* hi,
                                                             int32_t nq, uint32_t* count, uint32_t* list,
                                                             uint32_t cap) {
  const int32_t qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  const int d = tv.d;
  uint32_t stack_h[KDT_MAX_LEVELS + 2];
  int8_t stack_l[KDT_MAX_LEVELS + 2];
  int sp = 0;
  stack_h[sp] = 0;
  stack_l[sp++] = 0;
  uint32_t found = 0;
  while (sp > 0) {
    const uint32_t h = stack_h[--sp];
    const int l = stack_l[sp];
    if (l < tv.L) {
      const int t = tv.dims[h];
      if (t < 0) {  // every point of the node is in its leftmost leaf
        stack_h[sp] = 2u * h + 1u;
        stack_l[sp++] = (int8_t)(l + 1);
        continue;
      }
      const uint32_t m = ord_key(tv.vals[h]);
      if (ord_key(hi[(int64_t)t * nq + qi]) > m) {
        stack_h[sp] = 2u * h + 2u;
        stack_l[sp++] = (int8_t)(l + 1);
      }
      if (ord_key(lo[(int64_t)t * nq + qi]) <= m) {
        stack_h[sp] = 2u * h + 1u;
        stack_l[sp++] = (int8_t)(l + 1);
      }
      continue;
    }
    uint32_t k0, k1;
    node_leaves(tv, h, l, &k0, &k1);
    for (int64_t p = tv.offs[k0]; p < tv.offs[k1]; ++p) {
      const uint32_t i = tv.perm[p];
      bool in = true;
      for (int j = 0; j < d && in; ++j) {
        const uint32_t kx = ord_key(tv.x[(int64_t)j * tv.n + i]);
        in = ord_key(lo[(int64_t)j * nq + qi]) <= kx && kx <= ord_key(hi[(int64_t)j * nq + qi]);
      }
      if (in) {
        if (list && found < cap) list[(size_t)qi * cap + found] = i;
        ++found;
      }
    }
  }
  count[qi] = found;
}

// (distance, index) order: smaller distance first, then smaller index.
__device__ __forceinline__ bool nearer(double a, uint32_t ia, double b, uint32_t ib) {
  return a < b || (a == b && ia < ib);
}

template <int K>
__global__ void __launch_bounds__(kQueryThreads) k_query_knn(TreeView tv, const float* qs, int32_t nq, int32_t k,
                                                             uint32_t* out_idx, double* out_d2) {
  const int32_t qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  const int d = tv.d;
  double bd[K];
  uint32_t bi[K];
  for (int j = 0; j < K; ++j) {
    bd[j] = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    bi[j] = 0xffffffffu;
  }
  int nbest = 0;
  uint32_t stack_h[KDT_MAX_LEVELS + 2];
  int8_t stack_l[KDT_MAX_LEVELS + 2];
  double stack_b[KDT_MAX_LEVELS + 2];  // lower bound of the node's squared distance
  int sp = 0;
  stack_h[sp] = 0;
  stack_l[sp] = 0;
  stack_b[sp++] = 0.0;
  while (sp > 0) {
    --sp;
    const uint32_t h = stack_h[sp];
    const int l = stack_l[sp];
    const double bound = stack_b[sp];
    if (nbest == k && bound > bd[k - 1]) continue;
    if (l < tv.L) {
      const int t = tv.dims[h];
      if (t < 0) {
        stack_h[sp] = 2u * h + 1u;
        stack_l[sp] = (int8_t)(l + 1);
        stack_b[sp++] = bound;
        continue;
      }
      const float mv = tv.vals[h];
      const float qv = qs[(int64_t)t * nq + qi];
      const double diff = __dsub_rn((double)qv, (double)mv);
      const double plane = __dmul_rn(diff, diff);
      const bool q_left = ord_key(qv) <= ord_key(mv);
      const uint32_t near = q_left ? 2u * h + 1u : 2u * h + 2u, far = q_left ? 2u * h + 2u : 2u * h + 1u;
      stack_h[sp] = far;  // pushed first, visited last
      stack_l[sp] = (int8_t)(l + 1);
      stack_b[sp++] = fmax(bound, plane);
      stack_h[sp] = near;
      stack_l[sp] = (int8_t)(l + 1);
      stack_b[sp++] = bound;
      continue;
    }
    uint32_t k0, k1;
    node_leaves(tv, h, l, &k0, &k1);
    for (int64_t p = tv.offs[k0]; p < tv.offs[k1]; ++p) {
      const uint32_t i = tv.perm[p];
      double d2 = 0.0;
      for (int j = 0; j < d; ++j) {
        const double df = __dsub_rn((double)tv.x[(int64_t)j * tv.n + i], (double)qs[(int64_t)j * nq + qi]);
        d2 = __dadd_rn(d2, __dmul_rn(df, df));
      }
      if (nbest == k && !nearer(d2, i, bd[k - 1], bi[k - 1])) continue;
      // insert into the sorted list (registers: K is a compile-time bound)
      int pos = nbest < k ? nbest : k - 1;
      if (nbest < k) ++nbest;
#pragma unroll
      for (int j = K - 1; j > 0; --j)
        if (j <= pos && j < k) {
          if (nearer(d2, i, bd[j - 1], bi[j - 1])) {
            bd[j] = bd[j - 1];
            bi[j] = bi[j - 1];
            pos = j - 1;
          }
        }
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j == pos) {
          bd[j] = d2;
          bi[j] = i;
        }
    }
  }
  for (int j = 0; j < K; ++j)
    if (j < k) {
      out_idx[(size_t)qi * k + j] = bi[j];
      out_d2[(size_t)qi * k + j] = bd[j];
    }
}

kdt_status check_tree(const float* points, int64_t n, int32_t d, const uint32_t* perm, const float* vals,
                      const int8_t* dims, const int64_t* offs, int32_t L) {
  if (n < 0 || n > (int64_t)0xffffffffLL || d < 1 || d > KDT_MAX_DIMS || L < 0 || L > KDT_MAX_LEVELS)
    return KDT_ERR_INVALID_ARG;
  if (!offs || (n > 0 && (!points || !perm)) || (L > 0 && (!vals || !dims))) return KDT_ERR_INVALID_ARG;
  return KDT_OK;
}

}  // namespace

}  // namespace kdt

using namespace kdt;

extern "C" {

kdt_status kdt_query_box(const float* points, int64_t n, int32_t d, const uint32_t* perm, const float* split_vals,
                         const int8_t* split_dims, const int64_t* node_offsets, int32_t levels, const float* lo,
                         const float* hi, int32_t nq, uint32_t* out_count, uint32_t* out_list, uint32_t list_cap,
                         void* stream) {
  const kdt_status v = check_tree(points, n, d, perm, split_vals, split_dims, node_offsets, levels);
  if (v != KDT_OK) return v;
  if (nq < 0 || (nq > 0 && (!lo || !hi || !out_count)) || (out_list && list_cap == 0)) return KDT_ERR_INVALID_ARG;
  if (capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the query waits on its stream
  if (nq == 0) return KDT_OK;
  const TreeView tv{points, n, d, levels, perm, split_vals, split_dims, node_offsets};
  cudaStream_t st = (cudaStream_t)stream;
  {
    TraceScope ts(K_QUERY, st, (uint64_t)nq);
    k_query_box<<<(nq + kQueryThreads - 1) / kQueryThreads, kQueryThreads, 0, st>>>(tv, lo, hi, nq, out_count,
                                                                                    out_list, list_cap);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return KDT_ERR_CUDA;
  }
  return KDT_OK;
}

kdt_status kdt_query_knn(const float* points, int64_t n, int32_t d, const uint32_t* perm, const float* split_vals,
                         const int8_t* split_dims, const int64_t* node_offsets, int32_t levels, const float* queries,
                         int32_t nq, int32_t k, uint32_t* out_idx, double* out_dist2, void* stream) {
  const kdt_status v = check_tree(points, n, d, perm, split_vals, split_dims, node_offsets, levels);
  if (v != KDT_OK) return v;
  if (nq < 0 || k < 1 || k > KDT_KNN_MAX_K || (nq > 0 && (!queries || !out_idx || !out_dist2)))
    return KDT_ERR_INVALID_ARG;
  if (capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the query waits on its stream
  if (nq == 0) return KDT_OK;
  const TreeView tv{points, n, d, levels, perm, split_vals, split_dims, node_offsets};
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t grid = (nq + kQueryThreads - 1) / kQueryThreads;
  {
    TraceScope ts(K_QUERY, st, (uint64_t)nq);
    if (k <= 8)
      k_query_knn<8><<<grid, kQueryThreads, 0, st>>>(tv, queries, nq, k, out_idx, out_dist2);
    else
      k_query_knn<KDT_KNN_MAX_K><<<grid, kQueryThreads, 0, st>>>(tv, queries, nq, k, out_idx, out_dist2);  // k <= 32
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return KDT_ERR_CUDA;
  }
  return KDT_OK;
}

}  // extern "C"
