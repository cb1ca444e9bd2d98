// kdt_api.cu -- C ABI entry points and the host-side level driver.
//
// One build = a loop over levels of the multi-CTA pipeline for cells larger
// than the subtree capacity; every cell that fits in shared memory is handed
// to the persistent subtree kernel, which finishes all of its remaining
// levels; terminal cells are recorded on the way and turned into offsets and
// sentinels by the finalize kernel.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kdt.h"
#include "kdt_engine.h"
#include "kdt_launch.h"
#include "kdt_trace.h"

namespace kdt {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Workspace of a one-tree build: the engine's shared tables, then the tree.
struct PlainPlan {
  StepPlan step;
  TreePlan tree;
  size_t tree_off = 0;
  size_t total = 0;
};

PlainPlan plan_plain(const kdt_params& p) {
  PlainPlan pp;
  pp.tree = plan_tree(p);
  StepNeeds needs;
  needs.add(p, pp.tree);
  pp.step = plan_step(needs);
  pp.tree_off = align_up(pp.step.bytes);
  pp.total = pp.tree_off + pp.tree.bytes;
  return pp;
}

kdt_status build_device(const float* points, const kdt_params& p, uint8_t* ws, const PlainPlan& pp,
                        uint32_t* out_perm, float* out_vals, int8_t* out_dims, int64_t* out_offs,
                        int32_t* out_levels, cudaStream_t st) {
  Engine e(pp.step, ws, st);
  kdt_status s = e.reset();
  if (s != KDT_OK) return s;
  s = e.admit(0, points, p, pp.tree, ws + pp.tree_off, out_perm, out_vals, out_dims, out_offs);
  if (s != KDT_OK) return s;
  s = e.run_to_completion();
  if (s != KDT_OK) return s;
  std::vector<kdt_status> status;
  std::vector<int32_t> levels;
  s = e.finalize({0u}, &status, &levels);
  if (s != KDT_OK) return s;
  if (status[0] != KDT_OK) return status[0];
  if (out_levels) *out_levels = p.depth > 0 ? p.depth : levels[0];
  return KDT_OK;
}

}  // namespace

// Build with a caller-provided workspace that is never NULL; used by entry
// points that own their workspace memory. Allocates nothing.
kdt_status build_in_workspace(const float* points, const kdt_params* p, void* workspace, size_t workspace_bytes,
                              uint32_t* out_perm, float* out_split_vals, int8_t* out_split_dims,
                              int64_t* out_node_offsets, int32_t* out_levels, cudaStream_t st) {
  const kdt_status v = validate_params(p);
  if (v != KDT_OK) return v;
  if ((p->n > 0 && (!points || !out_perm)) || !out_node_offsets || !workspace) return KDT_ERR_INVALID_ARG;
  const int L_cap = p->depth > 0 ? p->depth : p->max_levels;
  if (L_cap > 0 && (!out_split_vals || !out_split_dims)) return KDT_ERR_INVALID_ARG;
  const PlainPlan pp = plan_plain(*p);
  if (workspace_bytes < pp.total) return KDT_ERR_CAPACITY;
  if ((uintptr_t)workspace % kAlign) return KDT_ERR_INVALID_ARG;
  return build_device(points, *p, (uint8_t*)workspace, pp, out_perm, out_split_vals, out_split_dims,
                      out_node_offsets, out_levels, st);
}

}  // namespace kdt

using namespace kdt;

extern "C" {

kdt_status kdt_workspace_size(const kdt_params* p, size_t* bytes) {
  const kdt_status v = validate_params(p);
  if (v != KDT_OK) return v;
  if (!bytes) return KDT_ERR_INVALID_ARG;
  *bytes = plan_plain(*p).total;
  return KDT_OK;
}

kdt_status kdt_build(const float* points, const kdt_params* p, void* workspace, size_t workspace_bytes,
                     uint32_t* out_perm, float* out_split_vals, int8_t* out_split_dims,
                     int64_t* out_node_offsets, int32_t* out_levels, void* stream) {
  const kdt_status v = validate_params(p);
  if (v != KDT_OK) return v;
  if (capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the build waits on its stream
  if ((p->n > 0 && (!points || !out_perm)) || !out_node_offsets) return KDT_ERR_INVALID_ARG;
  const int L_cap = p->depth > 0 ? p->depth : p->max_levels;
  if (L_cap > 0 && (!out_split_vals || !out_split_dims)) return KDT_ERR_INVALID_ARG;
  const PlainPlan pp = plan_plain(*p);
  cudaStream_t st = (cudaStream_t)stream;
  void* owned = nullptr;
  if (!workspace) {
    if (kdt::dev_malloc(&owned, pp.total) != cudaSuccess) {
      (void)cudaGetLastError();
      return KDT_ERR_OOM;
    }
    workspace = owned;
  } else if (workspace_bytes < pp.total) {
    return KDT_ERR_CAPACITY;
  } else if ((uintptr_t)workspace % kAlign) {
    return KDT_ERR_INVALID_ARG;
  }
  kdt_status s = build_device(points, *p, (uint8_t*)workspace, pp, out_perm, out_split_vals,
                              out_split_dims, out_node_offsets, out_levels, st);
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  return s;
}

kdt_status kdt_workspace_size_host(const kdt_params* p, size_t* bytes) {
  const kdt_status v = validate_params(p);
  if (v != KDT_OK) return v;
  if (!bytes) return KDT_ERR_INVALID_ARG;
  const PlainPlan pp = plan_plain(*p);
  const uint64_t n = (uint64_t)p->n;
  const uint64_t leaves = (uint64_t)1 << pp.tree.L_cap;
  size_t extra = align_up((size_t)p->d * n * 4) + align_up(n * (size_t)pp.tree.sid_bytes) +
                 align_up(n * 4) + align_up(leaves * 4) + align_up(leaves) + align_up((leaves + 1) * 8);
  *bytes = pp.total + extra;
  return KDT_OK;
}

kdt_status kdt_build_host(const float* points_host, const kdt_params* p, void* workspace,
                          size_t workspace_bytes, uint32_t* out_perm_host, float* out_split_vals_host,
                          int8_t* out_split_dims_host, int64_t* out_node_offsets_host, int32_t* out_levels,
                          void* stream) {
  const kdt_status v = validate_params(p);
  if (v != KDT_OK) return v;
  if (capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the build waits on its stream
  if ((p->n > 0 && (!points_host || !out_perm_host)) || !out_node_offsets_host) return KDT_ERR_INVALID_ARG;
  size_t need = 0;
  kdt_workspace_size_host(p, &need);
  const PlainPlan pp = plan_plain(*p);
  cudaStream_t st = (cudaStream_t)stream;
  void* owned = nullptr;
  if (!workspace) {
    if (kdt::dev_malloc(&owned, need) != cudaSuccess) {
      (void)cudaGetLastError();
      return KDT_ERR_OOM;
    }
    workspace = owned;
  } else if (workspace_bytes < need) {
    return KDT_ERR_CAPACITY;
  } else if ((uintptr_t)workspace % kAlign) {
    return KDT_ERR_INVALID_ARG;
  }
  uint8_t* ws = (uint8_t*)workspace;
  const uint64_t n = (uint64_t)p->n;
  const uint64_t leaves = (uint64_t)1 << pp.tree.L_cap;
  size_t off = pp.total;
  float* d_pts = (float*)(ws + off);
  off += align_up((size_t)p->d * n * 4);
  void* d_sid = ws + off;
  off += align_up(n * (size_t)pp.tree.sid_bytes);
  uint32_t* d_perm = (uint32_t*)(ws + off);
  off += align_up(n * 4);
  float* d_vals = (float*)(ws + off);
  off += align_up(leaves * 4);
  int8_t* d_dims = (int8_t*)(ws + off);
  off += align_up(leaves);
  int64_t* d_offs = (int64_t*)(ws + off);

  kdt_status s = KDT_OK;
  kdt_params pd = *p;
  int32_t levels = 0;
  do {
    if (n && cudaMemcpyAsync(d_pts, points_host, (size_t)p->d * n * 4, cudaMemcpyHostToDevice, st) !=
                 cudaSuccess) {
      s = KDT_ERR_CUDA;
      break;
    }
    if (pp.tree.sid_bytes) {
      const void* hs = p->subset_id16 ? (const void*)p->subset_id16 : (const void*)p->subset_id8;
      if (n && cudaMemcpyAsync(d_sid, hs, n * (size_t)pp.tree.sid_bytes, cudaMemcpyHostToDevice, st) !=
                   cudaSuccess) {
        s = KDT_ERR_CUDA;
        break;
      }
      pd.subset_id8 = p->subset_id8 ? (const uint8_t*)d_sid : nullptr;
      pd.subset_id16 = p->subset_id16 ? (const uint16_t*)d_sid : nullptr;
    }
    s = build_device(d_pts, pd, ws, pp, d_perm, d_vals, d_dims, d_offs, &levels, st);
    if (s != KDT_OK) break;
    const uint64_t nl = (uint64_t)1 << levels;
    if ((n && cudaMemcpyAsync(out_perm_host, d_perm, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        (nl > 1 && out_split_vals_host &&
         cudaMemcpyAsync(out_split_vals_host, d_vals, (nl - 1) * 4, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess) ||
        (nl > 1 && out_split_dims_host &&
         cudaMemcpyAsync(out_split_dims_host, d_dims, nl - 1, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaMemcpyAsync(out_node_offsets_host, d_offs, (nl + 1) * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      s = KDT_ERR_CUDA;
      break;
    }
    if (out_levels) *out_levels = levels;
  } while (0);
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  return s;
}

int32_t kdt_subtree_capacity(int32_t d) {
  if (d < 1 || d > KDT_MAX_DIMS) return 0;
  return subtree_capacity(d);
}

const char* kdt_status_str(kdt_status s) {
  switch (s) {
    case KDT_OK: return "ok";
    case KDT_ERR_INVALID_ARG: return "invalid argument";
    case KDT_ERR_NAN_INPUT: return "NaN in the input points";
    case KDT_ERR_OOM: return "out of memory";
    case KDT_ERR_CUDA: return "CUDA runtime error";
    case KDT_ERR_CAPACITY: return "buffer or workspace too small";
    case KDT_ERR_TIMEOUT: return "bounded device wait gave up";
    case KDT_ERR_LEVEL_CAP: return "leaf mode needs more than max_levels levels";
    case KDT_ERR_BUSY: return "server busy";
    case KDT_ERR_NOT_FOUND: return "unknown ticket";
    case KDT_ERR_CANCELLED: return "request cancelled";
  }
  return "unknown status";
}

}  // extern "C"
