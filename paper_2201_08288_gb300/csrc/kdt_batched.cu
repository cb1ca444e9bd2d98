// kdt_batched.cu -- many independent trees built together.
//
// Every tree is admitted into its own slot of one engine at tick 0; each tick
// then splits the big cells of all trees in the same kernels (a tile or a
// segment knows its tree) and finishes every cell that became small in one
// persistent subtree launch. Results per tree are identical to kdt_build's:
// no reduction crosses trees.
#include <cstdlib>
#include <algorithm>
#include <vector>

#include "kdt.h"
#include "kdt_engine.h"
#include "kdt_trace.h"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct BatchPlan {
  kdt::StepPlan step;
  std::vector<kdt::TreePlan> trees;
  std::vector<size_t> tree_off;
  size_t total = 0;
};

kdt_status plan_batch(const kdt_tree_desc* trees, int32_t num, BatchPlan* bp) {
  if (!trees || num < 1) return KDT_ERR_INVALID_ARG;
  kdt::StepNeeds needs;
  bp->trees.resize(num);
  for (int32_t i = 0; i < num; ++i) {
    const kdt_status v = kdt::validate_params(&trees[i].params);
    if (v != KDT_OK) return v;
    if (trees[i].params.fourier_j != 0) return KDT_ERR_INVALID_ARG;  // plain builds only
    bp->trees[i] = kdt::plan_tree(trees[i].params);
    needs.add(trees[i].params, bp->trees[i]);
  }
  bp->step = kdt::plan_step(needs);
  size_t off = align_up(bp->step.bytes);
  bp->tree_off.resize(num);
  for (int32_t i = 0; i < num; ++i) {
    bp->tree_off[i] = off;
    off += align_up(bp->trees[i].bytes);
  }
  bp->total = off;
  return KDT_OK;
}

}  // namespace

extern "C" {

kdt_status kdt_workspace_size_batched(const kdt_tree_desc* trees, int32_t num_trees, size_t* bytes) {
  if (!bytes) return KDT_ERR_INVALID_ARG;
  BatchPlan bp;
  const kdt_status s = plan_batch(trees, num_trees, &bp);
  if (s != KDT_OK) return s;
  *bytes = bp.total;
  return KDT_OK;
}

kdt_status kdt_build_batched(const kdt_tree_desc* trees, int32_t num_trees, void* workspace,
                             size_t workspace_bytes, int32_t* out_levels, kdt_status* out_status, void* stream) {
  BatchPlan bp;
  kdt_status s = plan_batch(trees, num_trees, &bp);
  if (s != KDT_OK) return s;
  if (kdt::capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the build waits on its stream
  for (int32_t i = 0; i < num_trees; ++i) {
    const kdt_tree_desc& t = trees[i];
    const int L_cap = t.params.depth > 0 ? t.params.depth : t.params.max_levels;
    if ((t.params.n > 0 && (!t.points || !t.out_perm)) || !t.out_node_offsets ||
        (L_cap > 0 && (!t.out_split_vals || !t.out_split_dims)))
      return KDT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* owned = nullptr;
  if (!workspace) {
    if (kdt::dev_malloc(&owned, bp.total) != cudaSuccess) {
      (void)cudaGetLastError();
      return KDT_ERR_OOM;
    }
    workspace = owned;
  } else if (workspace_bytes < bp.total) {
    return KDT_ERR_CAPACITY;
  } else if ((uintptr_t)workspace % kAlign) {
    return KDT_ERR_INVALID_ARG;
  }
  uint8_t* ws = (uint8_t*)workspace;
  kdt::Engine e(bp.step, ws, st);
  std::vector<uint32_t> slots(num_trees);
  std::vector<kdt_status> status;
  std::vector<int32_t> levels;
  do {
    if ((s = e.reset()) != KDT_OK) break;
    for (int32_t i = 0; i < num_trees && s == KDT_OK; ++i) {
      slots[i] = (uint32_t)i;
      s = e.admit((uint32_t)i, trees[i].points, trees[i].params, bp.trees[i], ws + bp.tree_off[i],
                  trees[i].out_perm, trees[i].out_split_vals, trees[i].out_split_dims,
                  trees[i].out_node_offsets);
    }
    if (s != KDT_OK) break;
    // all level steps after the roots' in one graph launch (KDT_BATCH_GRAPH=0:
    // every step launched and sized by the host, a debugging aid)
    static const bool use_graph = [] {
      const char* v = std::getenv("KDT_BATCH_GRAPH");
      return !(v && v[0] == '0');
    }();
    if ((s = use_graph ? e.run_graph() : e.run_to_completion()) != KDT_OK) break;
    s = e.finalize(slots, &status, &levels);
  } while (0);
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  if (s != KDT_OK) return s;
  kdt_status first = KDT_OK;
  for (int32_t i = 0; i < num_trees; ++i) {
    if (out_status) out_status[i] = status[i];
    if (out_levels) out_levels[i] = trees[i].params.depth > 0 ? trees[i].params.depth : levels[i];
    if (first == KDT_OK) first = status[i];
  }
  return first;
}

}  // extern "C"
