// kdt_engine.h -- host-side driver shared by the plain, batched and served
// builds.
//
// The engine owns the tables of one "forest": up to max_trees trees, each in
// its own slot, whose cells are split together. One tick is one level step of
// the multi-CTA pipeline over every big cell of every tree in flight (each
// tree at its own level), followed by the subtree kernel over every cell that
// became small during the tick. A tree's cells never mix with another tree's
// data; trees join (admit) and leave (finalize) between ticks.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "kdt.h"
#include "kdt_launch.h"

namespace kdt {

kdt_status validate_params(const kdt_params* p);
// The parameters a build runs with: a Fourier-estimator build ignores the
// subsets (one subset, no ids), since its statistics are sums.
kdt_params effective_params(const kdt_params& p);

// Memory of one tree (offsets relative to the tree's base, 256-byte aligned).
struct TreePlan {
  int L_cap = 0;
  int small_max = 0;
  int sid_bytes = 0;
  bool sub_wide = false;   // small cells run in the subtree kernel's wide shape
  bool presorted = false;  // root split by the pipeline, reordered by subset first
  bool leafsort = false;   // subsets not in index order: leaves are sorted at the end
  uint64_t n = 0;
  uint64_t term_cap = 0;
  uint64_t huge_cap = 0;  // terminal cells larger than one CTA's leaf sort
  uint64_t maxB = 0;      // big cells at one level
  uint64_t cap_small = 0; // small cells over the whole build
  size_t xbuf[2] = {0, 0}, pbuf[2] = {0, 0}, sbuf[2] = {0, 0}, terms = 0, root_off = 0, root_cur = 0,
         huge = 0, words = 0;
  size_t bytes = 0;
};
// no_subtree: every cell stays in the multi-CTA pipeline (a sharded build's
// trees, whose splits are exchanged level by level).
TreePlan plan_tree(const kdt_params& p, bool no_subtree = false);

// Capacities of the shared tables, accumulated over the trees they must serve
// at the same time.
struct StepNeeds {
  uint64_t points = 0, maxB = 0, cap_small = 0, nseg = 0;
  uint32_t max_trees = 0, slice_cells = 32;
  bool widest = false;
  bool fourier = false;  // a tree splits by the Fourier-moment estimator
  int max_d = 1, min_d = 1 << 30;  // min_d == max_d: every tree has the same d
  int max_r = 1;                   // the largest subset count: segments per cell
  void add(const kdt_params& p, const TreePlan& tp);
};

struct StepPlan {
  StepNeeds needs;
  // grid_step: the grid scale of the level step's kernels (two per SM);
  // sms: the device's SMs (the subtree kernel's grid is sms x its shape's CTAs)
  uint32_t maxB = 0, cap_small = 0, max_tiles = 0, nseg_cap = 0, bigseg_cap = 0, grid_step = 0, sms = 0, off_cap = 0;
  size_t trees = 0, words = 0, slot_words = 0, slots_list = 0, big[2] = {0, 0}, small = 0, tile_base = 0,
         seg_base = 0, tiles = 0, tile_left = 0, tile_loff = 0, tile_mm = 0, child_mm = 0, kdim = 0,
         mkey = 0, lcount = 0, seg_w = 0, seg_key = 0, seg_med = 0, bigseg = 0, midseg = 0, slices = 0,
         off[2] = {0, 0}, obase[2] = {0, 0}, crow = 0;
  size_t bytes = 0;
};
StepPlan plan_step(const StepNeeds& needs);

class Engine {
 public:
  Engine(const StepPlan& plan, uint8_t* base, cudaStream_t st);

  // Clear every counter (call once before the first admit).
  kdt_status reset();
  // Make the forest's trees 0..shards-1 the shards of one tree (see
  // StepDev::shards); the tables are device memory of the caller.
  void set_sharding(uint32_t shards, uint32_t span, uint32_t* idx, uint32_t* wcount, uint32_t* mm_tmp) {
    s_.shards = shards;
    s_.shard_span = span;
    s_.shard_idx = idx;
    s_.wcount = wcount;
    s_.mm_tmp = mm_tmp;
  }
  // Put a tree into `slot`. tree_base holds TreePlan::bytes of device memory.
  kdt_status admit(uint32_t slot, const float* points, const kdt_params& p, const TreePlan& tp, uint8_t* tree_base,
                   uint32_t* out_perm, float* out_vals, int8_t* out_dims, int64_t* out_offs);
  // One tick (see above). Synchronises the stream once.
  kdt_status tick();
  // True while some cell of some tree still waits for a tick.
  bool busy() const { return big_count_ > 0 || small_count_ > 0 || small_count_w_ > 0; }
  // Slots (among `slots`) whose trees have no cell left.
  kdt_status done_slots(const std::vector<uint32_t>& slots, std::vector<uint32_t>* done);
  // Offsets and sentinels of finished trees, then their status and L.
  kdt_status finalize(const std::vector<uint32_t>& slots, std::vector<kdt_status>* status,
                      std::vector<int32_t>* levels);
  // Run ticks until nothing is left in flight.
  kdt_status run_to_completion();
  // The same with one graph launch: the first tick (new roots) from the
  // host, then every later tick inside a CUDA graph whose conditional while
  // node repeats a pair of recorded ticks until no cell is left.
  kdt_status run_graph();
  // Iterations (pairs of ticks) of the last run_graph.
  uint32_t graph_iters() const { return graph_iters_; }

 private:
  StepPlan plan_;
  uint8_t* base_;
  cudaStream_t st_;
  TreeDev* trees_ = nullptr;      // device [max_trees]
  uint32_t* words_ = nullptr;     // device engine words
  uint32_t* slot_words_ = nullptr;  // device [4][max_trees]: term_count, status, levels, live
  uint32_t* slots_list_ = nullptr;  // device [max_trees]
  Cell* big_[2] = {nullptr, nullptr};
  uint32_t* off_[2] = {nullptr, nullptr};
  uint32_t* obase_[2] = {nullptr, nullptr};
  Cell* small_ = nullptr;
  LCell* slices_ = nullptr;
  StepDev s_{};
  int cur_ = 0;
  uint32_t big_count_ = 0, small_count_ = 0, small_count_w_ = 0;  // small: front (narrow), back (wide)
  uint64_t big_points_ = 0, small_points_ = 0;
  bool root_dims_ = false;
  bool debug_ = false;
  uint32_t graph_iters_ = 0;
  // Record a tick over cell list p into the stream's capture (counts on the device).
  kdt_status record_tick(int p);
  // The subtree kernel over the small-cell queue: the narrow shape over its
  // front, the wide one over its back (host counts, or the device's).
  void launch_small(bool from_device);
  std::vector<Cell> pending_big_, pending_small_, pending_small_w_;
  std::vector<TreeHost> host_;       // per slot: leaf-sort view of a presorted tree
  std::vector<uint8_t> leafsort_;    // per slot
  std::vector<uint8_t> wide_;        // per slot: the tree's small cells use the wide shape
};

}  // namespace kdt
