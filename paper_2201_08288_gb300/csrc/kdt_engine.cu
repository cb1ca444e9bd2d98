// kdt_engine.cu -- the forest engine (see kdt_engine.h).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "kdt_engine.h"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Engine words.
// W_NC0, W_NC1, W_ITERS (adjacent): the cell counts of the two lists and the
// iteration count of a graph-driven run
enum Word {
  W_NTILES = 0, W_BIGSEG, W_HEAD, W_NEXTBIG, W_BIGPTS, W_OFFUSED, W_MIDSEG,
  W_SMALL, W_SMALLW, W_SMALLTOT, W_SMALLPTS,  // adjacent: written together by a tick
  W_NC0, W_NC1, W_ITERS, W_COUNT
};
// a graph-driven run's iterations (two level steps each) before it gives up
constexpr uint32_t kGraphIterMax = KDT_MAX_LEVELS + 4;
// Per-slot words: [which][max_trees].
enum SlotWord { S_TERM = 0, S_STATUS, S_LEVELS, S_LIVE, S_COUNT };

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return sms;
}

kdt_status map_status(int32_t st) {
  switch (st) {
    case ST_OK: return KDT_OK;
    case ST_INVALID_ARG: return KDT_ERR_INVALID_ARG;
    case ST_NAN_INPUT: return KDT_ERR_NAN_INPUT;
    case ST_LEVEL_CAP: return KDT_ERR_LEVEL_CAP;
    case ST_CAPACITY: return KDT_ERR_CAPACITY;
    case ST_TIMEOUT: return KDT_ERR_TIMEOUT;
    default: return KDT_ERR_CUDA;
  }
}

#define ENGINE_TRY(expr)         \
  do {                           \
    if ((expr) != cudaSuccess) { \
      (void)cudaGetLastError();  \
      return KDT_ERR_CUDA;       \
    }                            \
  } while (0)

}  // namespace

kdt_status validate_params(const kdt_params* p) {
  if (!p) return KDT_ERR_INVALID_ARG;
  if (p->n < 0 || p->n > (int64_t)0xffffffffLL) return KDT_ERR_INVALID_ARG;
  if (p->d < 1 || p->d > KDT_MAX_DIMS) return KDT_ERR_INVALID_ARG;
  if (p->r < 1 || p->r > KDT_MAX_SUBSETS) return KDT_ERR_INVALID_ARG;
  if (p->key_rule != KDT_KEY_CYCLIC && p->key_rule != KDT_KEY_WIDEST_SPREAD) return KDT_ERR_INVALID_ARG;
  if (p->subset_mode != KDT_SUBSET_MOD && p->subset_mode != KDT_SUBSET_CONTIGUOUS &&
      p->subset_mode != KDT_SUBSET_EXPLICIT)
    return KDT_ERR_INVALID_ARG;
  if (p->subset_mode == KDT_SUBSET_EXPLICIT && p->n > 0 &&
      ((p->subset_id8 == nullptr) == (p->subset_id16 == nullptr)))
    return KDT_ERR_INVALID_ARG;
  if (p->depth < 0 || p->depth > KDT_MAX_LEVELS) return KDT_ERR_INVALID_ARG;
  if (p->depth == 0) {
    if (p->leaf_size < 1) return KDT_ERR_INVALID_ARG;
    if (p->max_levels < 0 || p->max_levels > KDT_MAX_LEVELS) return KDT_ERR_INVALID_ARG;
  }
  if (p->fourier_j < 0 || p->fourier_j > KDT_FOURIER_MAX_J) return KDT_ERR_INVALID_ARG;
  if (p->combine_rule != KDT_COMBINE_WEIGHTED && p->combine_rule != KDT_COMBINE_UNWEIGHTED)
    return KDT_ERR_INVALID_ARG;
  if (p->fourier_j > 0 && (p->key_rule != KDT_KEY_CYCLIC || p->depth == 0)) return KDT_ERR_INVALID_ARG;
  return KDT_OK;
}

kdt_params effective_params(const kdt_params& p) {
  kdt_params e = p;
  if (p.fourier_j > 0) {  // the estimator's sums do not depend on the subsets
    e.r = 1;
    e.subset_mode = KDT_SUBSET_MOD;
    e.subset_id8 = nullptr;
    e.subset_id16 = nullptr;
  }
  return e;
}

TreePlan plan_tree(const kdt_params& p0, bool no_subtree) {
  const kdt_params p = effective_params(p0);
  TreePlan t;
  const uint64_t n = (uint64_t)p.n;
  t.n = n;
  t.L_cap = p.depth > 0 ? p.depth : p.max_levels;
  // the estimator's splits come from the multi-CTA steps only (no subtree
  // kernel); its cells keep index order (no presort), so no leaf sort either
  const bool fourier = p.fourier_j > 0;
  t.small_max = (fourier || no_subtree) ? 0 : subtree_capacity(p.d);
  t.sub_wide = &subtree_shape(p.d) == &kSubWide;
  t.sid_bytes = p.subset_mode == KDT_SUBSET_EXPLICIT ? (p.subset_id16 ? 2 : 1) : 0;
  const bool root_terminal = p.depth > 0 ? (n == 0) : (n <= (uint64_t)p.leaf_size);
  t.leafsort = !root_terminal && p.subset_mode != KDT_SUBSET_CONTIGUOUS && !fourier;
  // a small root is put in subset order by the subtree kernel itself, which
  // counts at most kSubtreeHistWords subsets
  t.presorted = t.leafsort && (n > (uint64_t)t.small_max || !subtree_sorts_root(p.r));
  t.huge_cap = t.leafsort ? n / (uint64_t)(kLeafBlockMax + 1) + 1 : 0;
  const uint64_t leaves = (uint64_t)1 << t.L_cap;
  t.maxB = std::min<uint64_t>(n / (uint64_t)(t.small_max + 1) + 1, leaves);
  t.cap_small = std::min<uint64_t>(n, leaves) + 1;
  t.term_cap = leaves + 1;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += align_up(b);
    return o;
  };
  for (int b = 0; b < 2; ++b) {
    t.xbuf[b] = take((size_t)p.d * n * 4);
    t.pbuf[b] = take(n * 4);
    t.sbuf[b] = take(n * (size_t)t.sid_bytes);
  }
  t.terms = take(t.term_cap * sizeof(TermRec));
  t.root_off = take(((size_t)p.r + 1) * 4);
  t.root_cur = take((size_t)p.r * 4);
  t.huge = take(t.huge_cap * 4);
  t.words = take(16);
  t.bytes = off;
  return t;
}

void StepNeeds::add(const kdt_params& p0, const TreePlan& tp) {
  const kdt_params p = effective_params(p0);
  fourier = fourier || p.fourier_j > 0;
  points += tp.n;
  maxB += tp.maxB;
  cap_small += tp.cap_small;
  nseg += tp.maxB * (uint64_t)p.r;
  max_trees += 1;
  slice_cells = std::max<uint32_t>(slice_cells, (uint32_t)tp.small_max);
  widest = widest || p.key_rule == KDT_KEY_WIDEST_SPREAD;
  max_d = std::max(max_d, (int)p.d);
  max_r = std::max(max_r, (int)p.r);
  min_d = std::min(min_d, (int)p.d);
}

StepPlan plan_step(const StepNeeds& needs) {
  StepPlan s;
  s.needs = needs;
  const uint64_t clamp = 0xffffffffull;
  s.maxB = (uint32_t)std::min<uint64_t>(needs.maxB, clamp);
  s.cap_small = (uint32_t)std::min<uint64_t>(needs.cap_small, clamp);
  s.max_tiles = (uint32_t)std::min<uint64_t>(needs.points / kTile + needs.maxB + 1, clamp);
  s.nseg_cap = (uint32_t)std::min<uint64_t>(needs.nseg, clamp);
  s.off_cap = (uint32_t)std::min<uint64_t>(needs.nseg + needs.maxB, clamp);
  s.bigseg_cap = (uint32_t)std::min<uint64_t>(needs.points / (kSelWarpMin + 1) + 1, clamp);
  const int sms = device_sms();
  s.sms = (uint32_t)(sms > 0 ? sms : 148);
  s.grid_step = s.sms * 2u;
  const uint32_t grid_sub_max = s.sms * (uint32_t)std::max(kSubNarrow.ctas, kSubWide.ctas);
  const uint32_t mt = std::max<uint32_t>(needs.max_trees, 1);
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += align_up(b);
    return o;
  };
  s.trees = take((size_t)mt * sizeof(TreeDev));
  s.words = take(W_COUNT * 4);
  s.slot_words = take((size_t)S_COUNT * mt * 4);
  s.slots_list = take((size_t)mt * 2 * 4);
  s.big[0] = take((size_t)s.maxB * sizeof(Cell));
  s.big[1] = take((size_t)s.maxB * sizeof(Cell));
  s.small = take((size_t)s.cap_small * sizeof(Cell));
  s.tile_base = take(((size_t)s.maxB + 1) * 4);
  s.seg_base = take(((size_t)s.maxB + 1) * 4);
  s.tiles = take((size_t)s.max_tiles * sizeof(uint2));
  s.tile_left = take((size_t)s.max_tiles * 4);
  s.tile_loff = take((size_t)s.max_tiles * 4);
  s.tile_mm = take(needs.widest || needs.fourier ? (size_t)s.max_tiles * 2 * kMaxDims * 2 * 4 : 0);
  s.child_mm = take(needs.widest ? (size_t)s.maxB * 2 * kMaxDims * 2 * 4 : 0);
  s.kdim = take((size_t)s.maxB * 4);
  s.mkey = take((size_t)s.maxB * 4);
  s.lcount = take((size_t)s.maxB * 4);
  s.seg_w = take((size_t)s.nseg_cap * 4);
  s.seg_key = take((size_t)s.nseg_cap * 8);
  s.seg_med = take((size_t)s.nseg_cap * 4);
  s.bigseg = take((size_t)s.bigseg_cap * 4);
  s.midseg = take((size_t)s.nseg_cap * 4);
  s.slices = take((size_t)grid_sub_max * 2 * needs.slice_cells * sizeof(LCell));
  for (int b = 0; b < 2; ++b) {
    s.off[b] = take((size_t)s.off_cap * 4);
    s.obase[b] = take((size_t)s.maxB * 4);
  }
  s.crow = take((size_t)s.maxB * 2 * sizeof(uint2));
  s.bytes = off;
  return s;
}

Engine::Engine(const StepPlan& plan, uint8_t* base, cudaStream_t st) : plan_(plan), base_(base), st_(st) {
  const char* dbg = std::getenv("KDT_DEBUG");
  debug_ = dbg && *dbg && *dbg != '0';
  trees_ = (TreeDev*)(base + plan.trees);
  words_ = (uint32_t*)(base + plan.words);
  slot_words_ = (uint32_t*)(base + plan.slot_words);
  slots_list_ = (uint32_t*)(base + plan.slots_list);
  big_[0] = (Cell*)(base + plan.big[0]);
  big_[1] = (Cell*)(base + plan.big[1]);
  small_ = (Cell*)(base + plan.small);
  slices_ = (LCell*)(base + plan.slices);
  s_.tile_base = (uint32_t*)(base + plan.tile_base);
  s_.seg_base = (uint32_t*)(base + plan.seg_base);
  s_.tiles = (uint2*)(base + plan.tiles);
  s_.ntiles_total = words_ + W_NTILES;
  s_.kdim = (uint32_t*)(base + plan.kdim);
  s_.mkey = (uint32_t*)(base + plan.mkey);
  s_.lcount = (uint32_t*)(base + plan.lcount);
  s_.tile_mm = (uint32_t*)(base + plan.tile_mm);
  s_.child_mm = (uint32_t*)(base + plan.child_mm);
  s_.seg_w = (uint32_t*)(base + plan.seg_w);
  s_.seg_key = (const uint32_t**)(base + plan.seg_key);
  s_.seg_med = (uint32_t*)(base + plan.seg_med);
  s_.bigseg = (uint32_t*)(base + plan.bigseg);
  s_.bigseg_count = words_ + W_BIGSEG;
  s_.midseg = (uint32_t*)(base + plan.midseg);
  s_.midseg_count = words_ + W_MIDSEG;
  s_.tile_left = (uint32_t*)(base + plan.tile_left);
  s_.tile_loff = (uint32_t*)(base + plan.tile_loff);
  s_.next_big_count = words_ + W_NEXTBIG;
  s_.small = small_;
  s_.small_count = words_ + W_SMALL;
  s_.small_count_w = words_ + W_SMALLW;
  s_.small_total = words_ + W_SMALLTOT;
  s_.small_cap = plan.cap_small;
  s_.next_big_cap = plan.maxB;
  s_.next_big_points = words_ + W_BIGPTS;
  s_.small_points = words_ + W_SMALLPTS;
  for (int b = 0; b < 2; ++b) {
    off_[b] = (uint32_t*)(base + plan.off[b]);
    obase_[b] = (uint32_t*)(base + plan.obase[b]);
  }
  s_.off_used = words_ + W_OFFUSED;
  s_.off_cap = plan.off_cap;
  s_.bigseg_cap = plan.bigseg_cap;
  s_.midseg_cap = plan.nseg_cap;
  s_.crow = (uint2*)(base + plan.crow);
  const uint32_t mt = std::max<uint32_t>(plan.needs.max_trees, 1);
  host_.assign(mt, TreeHost{});
  leafsort_.assign(mt, 0);
  wide_.assign(mt, 0);
}

kdt_status Engine::reset() {
  ENGINE_TRY(prepare_subtree_kernel());
  ENGINE_TRY(prepare_scatter_kernel());
  ENGINE_TRY(prepare_step_kernels());
  const uint32_t mt = std::max<uint32_t>(plan_.needs.max_trees, 1);
  ENGINE_TRY(cudaMemsetAsync(words_, 0, W_COUNT * 4, st_));
  ENGINE_TRY(cudaMemsetAsync(slot_words_, 0, (size_t)S_COUNT * mt * 4, st_));
  cur_ = 0;
  big_count_ = small_count_ = small_count_w_ = 0;
  big_points_ = small_points_ = 0;
  root_dims_ = false;
  pending_big_.clear();
  pending_small_.clear();
  pending_small_w_.clear();
  return KDT_OK;
}

kdt_status Engine::admit(uint32_t slot, const float* points, const kdt_params& p0, const TreePlan& tp,
                         uint8_t* tb, uint32_t* out_perm, float* out_vals, int8_t* out_dims, int64_t* out_offs) {
  const kdt_params p = effective_params(p0);
  const uint32_t mt = std::max<uint32_t>(plan_.needs.max_trees, 1);
  if (slot >= mt) return KDT_ERR_CAPACITY;
  TreeDev h{};
  h.n = p.n;
  h.d = p.d;
  h.r = p.r;
  h.subset_mode = p.subset_mode;
  h.key_rule = p.key_rule;
  h.depth = p.depth;
  h.leaf_size = p.leaf_size;
  h.max_levels = p.max_levels;
  h.fourier_j = p.fourier_j;
  h.combine_rule = p.combine_rule;
  h.sub_wide = tp.sub_wide ? 1 : 0;
  h.stall_limit = p.key_rule == KDT_KEY_CYCLIC ? p.d : 1;
  h.sid_bytes = tp.sid_bytes;
  h.small_max = tp.small_max;
  h.presorted = tp.presorted ? 1 : 0;
  h.x_in = points;
  h.sid_in = p.subset_id16 ? (const void*)p.subset_id16 : (const void*)p.subset_id8;
  for (int b = 0; b < 2; ++b) {
    h.xbuf[b] = (float*)(tb + tp.xbuf[b]);
    h.pbuf[b] = (uint32_t*)(tb + tp.pbuf[b]);
    h.sbuf[b] = (void*)(tb + tp.sbuf[b]);
  }
  h.root_off = (uint32_t*)(tb + tp.root_off);
  h.root_cur = (uint32_t*)(tb + tp.root_cur);
  h.huge = (uint32_t*)(tb + tp.huge);
  h.huge_count = (uint32_t*)(tb + tp.words);
  h.huge_cap = (uint32_t)std::min<uint64_t>(tp.huge_cap, 0xffffffffull);
  h.out_perm = out_perm;
  h.out_vals = out_vals;
  h.out_dims = out_dims;
  h.out_offs = out_offs;
  h.terms = (TermRec*)(tb + tp.terms);
  h.term_cap = (uint32_t)std::min<uint64_t>(tp.term_cap, 0xffffffffull);
  h.term_count = slot_words_ + (size_t)S_TERM * mt + slot;
  h.status = (int32_t*)(slot_words_ + (size_t)S_STATUS * mt + slot);
  h.levels = (int32_t*)(slot_words_ + (size_t)S_LEVELS * mt + slot);
  h.live = (int32_t*)(slot_words_ + (size_t)S_LIVE * mt + slot);
  ENGINE_TRY(cudaMemcpyAsync(trees_ + slot, &h, sizeof(h), cudaMemcpyHostToDevice, st_));
  for (int w = 0; w < S_COUNT; ++w)
    ENGINE_TRY(cudaMemsetAsync(slot_words_ + (size_t)w * mt + slot, 0, 4, st_));
  ENGINE_TRY(cudaMemsetAsync(h.huge_count, 0, 4, st_));
  leafsort_[slot] = tp.leafsort ? 1 : 0;
  wide_[slot] = tp.sub_wide ? 1 : 0;
  // after the build the tree's working buffers are free: the global leaf-sort
  // passes use pbuf[0] as their second buffer and xbuf[0] for tile tables
  host_[slot] = TreeHost{(uint64_t)p.n, out_perm, h.pbuf[0], (void*)h.xbuf[0], (size_t)p.d * p.n * 4};

  const uint64_t n = (uint64_t)p.n;
  const Cell root{0u, (uint32_t)n, 0u, (int32_t)slot, 0, 0, -1};
  const bool root_terminal = p.depth > 0 ? (n == 0) : (n <= (uint64_t)p.leaf_size);
  if (root_terminal) {
    const TermRec tr{0u, (uint32_t)n, 0u, 0};
    const uint32_t one = 1;
    ENGINE_TRY(cudaMemcpyAsync(h.terms, &tr, sizeof(tr), cudaMemcpyHostToDevice, st_));
    ENGINE_TRY(cudaMemcpyAsync(h.term_count, &one, 4, cudaMemcpyHostToDevice, st_));
    launch_iota(out_perm, (uint32_t)n, st_);
    ENGINE_TRY(cudaGetLastError());
    return KDT_OK;
  }
  const int32_t one = 1;
  ENGINE_TRY(cudaMemcpyAsync(h.live, &one, 4, cudaMemcpyHostToDevice, st_));
  if (n <= (uint64_t)tp.small_max && !tp.presorted) {
    (tp.sub_wide ? pending_small_w_ : pending_small_).push_back(root);
  } else {
    pending_big_.push_back(root);
    if (p.key_rule == KDT_KEY_WIDEST_SPREAD) root_dims_ = true;
  }
  return KDT_OK;
}

kdt_status Engine::tick() {
  // new roots join the lists of this tick
  const bool has_roots = !pending_big_.empty();
  if (!pending_big_.empty()) {
    if (big_count_ + pending_big_.size() > plan_.maxB) return KDT_ERR_CAPACITY;
    ENGINE_TRY(cudaMemcpyAsync(big_[cur_] + big_count_, pending_big_.data(), pending_big_.size() * sizeof(Cell),
                               cudaMemcpyHostToDevice, st_));
    for (const Cell& c : pending_big_) big_points_ += c.count;
    big_count_ += (uint32_t)pending_big_.size();
    pending_big_.clear();
  }
  if (!pending_small_.empty() || !pending_small_w_.empty()) {
    if ((uint64_t)small_count_ + small_count_w_ + pending_small_.size() + pending_small_w_.size() > plan_.cap_small)
      return KDT_ERR_CAPACITY;
    if (!pending_small_.empty())
      ENGINE_TRY(cudaMemcpyAsync(small_ + small_count_, pending_small_.data(), pending_small_.size() * sizeof(Cell),
                                 cudaMemcpyHostToDevice, st_));
    if (!pending_small_w_.empty()) {
      // the back of the queue runs downwards: entry j at small[cap - 1 - j]
      std::reverse(pending_small_w_.begin(), pending_small_w_.end());
      const size_t m = pending_small_w_.size();
      ENGINE_TRY(cudaMemcpyAsync(small_ + plan_.cap_small - small_count_w_ - m, pending_small_w_.data(),
                                 m * sizeof(Cell), cudaMemcpyHostToDevice, st_));
    }
    for (const Cell& c : pending_small_) small_points_ += c.count;
    for (const Cell& c : pending_small_w_) small_points_ += c.count;
    small_count_ += (uint32_t)pending_small_.size();
    small_count_w_ += (uint32_t)pending_small_w_.size();
    pending_small_.clear();
    pending_small_w_.clear();
  }
  const uint32_t sw[4] = {small_count_, small_count_w_, small_count_ + small_count_w_, (uint32_t)small_points_};
  ENGINE_TRY(cudaMemcpyAsync(words_ + W_SMALL, sw, sizeof(sw), cudaMemcpyHostToDevice, st_));

  if (big_count_ > 0) {
    ENGINE_TRY(cudaMemsetAsync(words_ + W_NEXTBIG, 0, 4, st_));
    ENGINE_TRY(cudaMemsetAsync(words_ + W_BIGPTS, 0, 4, st_));
    ENGINE_TRY(cudaMemsetAsync(words_ + W_OFFUSED, 0, 4, st_));
    s_.cells = big_[cur_];
    s_.ncells = big_count_;
    s_.next_big = big_[cur_ ^ 1];
    s_.off_cur = off_[cur_];
    s_.obase_cur = obase_[cur_];
    s_.off_next = off_[cur_ ^ 1];
    s_.obase_next = obase_[cur_ ^ 1];
    const uint64_t nseg_bound = std::min<uint64_t>((uint64_t)big_count_ * (uint64_t)plan_.needs.max_r, plan_.nseg_cap);
    // tiles of this step: at most one per kTile points plus one per cell (a
    // tight launch size; the plan's max_tiles is the capacity of a full forest)
    // (the point counter is one device word: trust it only while it cannot wrap)
    const uint32_t tiles_bound =
        plan_.needs.points > 0xffffffffull
            ? plan_.max_tiles
            : (uint32_t)std::min<uint64_t>(big_points_ / (uint64_t)kTile + (uint64_t)big_count_ + 1,
                                           (uint64_t)plan_.max_tiles);
    const SelectTuning tune = current_tuning();
    s_.tiny_max = tune.tiny_max;
    s_.bitonic_max = tune.bitonic_max;
    s_.warp_max = tune.warp_max;
    launch_big_step(trees_, s_, tiles_bound, (uint32_t)nseg_bound, plan_.bigseg_cap, has_roots, root_dims_,
                    plan_.needs.widest, plan_.needs.max_d,
                    plan_.needs.min_d == plan_.needs.max_d ? plan_.needs.max_d : 0, tune, big_points_,
                    plan_.grid_step, st_, plan_.needs.fourier);
    ENGINE_TRY(cudaGetLastError());
    root_dims_ = false;
    uint32_t w[W_COUNT];
    ENGINE_TRY(cudaMemcpyAsync(w, words_, sizeof(w), cudaMemcpyDeviceToHost, st_));
    ENGINE_TRY(cudaStreamSynchronize(st_));
    if (debug_) {  // KDT_DEBUG=1: per-tick counts and raw tree statuses on stderr
      const uint32_t mt = std::max<uint32_t>(plan_.needs.max_trees, 1);
      std::vector<int32_t> stv(mt);
      ENGINE_TRY(cudaMemcpy(stv.data(), slot_words_ + (size_t)S_STATUS * mt, (size_t)mt * 4, cudaMemcpyDeviceToHost));
      std::fprintf(stderr, "kdt tick: big %u -> %u, small %u + %u\n", big_count_, w[W_NEXTBIG], w[W_SMALL],
                   w[W_SMALLW]);
      for (uint32_t k = 0; k < mt; ++k)
        if (stv[k]) std::fprintf(stderr, "kdt tick: slot %u status %d\n", k, stv[k]);
    }
    big_count_ = std::min(w[W_NEXTBIG], plan_.maxB);
    small_count_ = std::min(w[W_SMALL], plan_.cap_small);
    small_count_w_ = std::min(w[W_SMALLW], plan_.cap_small - small_count_);
    big_points_ = w[W_BIGPTS];
    small_points_ = w[W_SMALLPTS];
    cur_ ^= 1;
  } else {
    big_count_ = 0;
    big_points_ = 0;
  }
  if (small_count_ > 0 || small_count_w_ > 0) {
    launch_small(false);
    ENGINE_TRY(cudaGetLastError());
    small_count_ = small_count_w_ = 0;
    small_points_ = 0;
  }
  return KDT_OK;
}

void Engine::launch_small(bool from_device) {
  const uint32_t cap = plan_.cap_small;
  const uint32_t gn = plan_.sms * (uint32_t)kSubNarrow.ctas, gw = plan_.sms * (uint32_t)kSubWide.ctas;
  if (from_device) {
    // counts on the device (a recorded tick): the narrow front, then the wide
    // back walked from the end
    launch_subtree(kSubNarrow, trees_, small_, cap, words_ + W_SMALL, false, words_ + W_HEAD, slices_,
                   plan_.needs.slice_cells, gn, 0, st_);
    launch_subtree(kSubWide, trees_, small_, cap, words_ + W_SMALLW, true, words_ + W_HEAD, slices_,
                   plan_.needs.slice_cells, gw, 0, st_);
    return;
  }
  const uint64_t pts = small_points_;
  if (small_count_ > 0)
    launch_subtree(kSubNarrow, trees_, small_, small_count_, nullptr, false, words_ + W_HEAD, slices_,
                   plan_.needs.slice_cells, std::min(gn, small_count_), pts, st_);  // the points of both
  if (small_count_w_ > 0)
    launch_subtree(kSubWide, trees_, small_ + cap - small_count_w_, small_count_w_, nullptr, false,
                   words_ + W_HEAD, slices_, plan_.needs.slice_cells, std::min(gw, small_count_w_),
                   small_count_ ? 0 : pts, st_);
}

kdt_status Engine::done_slots(const std::vector<uint32_t>& slots, std::vector<uint32_t>* done) {
  const uint32_t mt = std::max<uint32_t>(plan_.needs.max_trees, 1);
  std::vector<int32_t> live(mt);
  ENGINE_TRY(cudaMemcpyAsync(live.data(), slot_words_ + (size_t)S_LIVE * mt, (size_t)mt * 4,
                             cudaMemcpyDeviceToHost, st_));
  ENGINE_TRY(cudaStreamSynchronize(st_));
  done->clear();
  for (uint32_t s : slots)
    if (s < mt && live[s] <= 0) done->push_back(s);
  return KDT_OK;
}

kdt_status Engine::finalize(const std::vector<uint32_t>& slots, std::vector<kdt_status>* status,
                            std::vector<int32_t>* levels) {
  const uint32_t mt = std::max<uint32_t>(plan_.needs.max_trees, 1);
  status->assign(slots.size(), KDT_OK);
  levels->assign(slots.size(), 0);
  if (slots.empty()) return KDT_OK;
  // trees with an error get no finalize (their outputs are undefined)
  std::vector<int32_t> st(mt), lv(mt);
  std::vector<uint32_t> tc(mt);
  ENGINE_TRY(cudaMemcpyAsync(tc.data(), slot_words_ + (size_t)S_TERM * mt, (size_t)mt * 4,
                             cudaMemcpyDeviceToHost, st_));
  ENGINE_TRY(cudaMemcpyAsync(st.data(), slot_words_ + (size_t)S_STATUS * mt, (size_t)mt * 4,
                             cudaMemcpyDeviceToHost, st_));
  ENGINE_TRY(cudaMemcpyAsync(lv.data(), slot_words_ + (size_t)S_LEVELS * mt, (size_t)mt * 4,
                             cudaMemcpyDeviceToHost, st_));
  ENGINE_TRY(cudaStreamSynchronize(st_));
  std::vector<uint32_t> ok;
  uint32_t max_rec = 0;
  for (uint32_t s : slots)
    if (st[s] == ST_OK) {
      ok.push_back(s);
      max_rec = std::max(max_rec, tc[s]);
    }
  std::vector<uint32_t> sorted;  // trees kept in subset order: their leaves need the leaf sort
  for (uint32_t s : ok)
    if (leafsort_[s]) sorted.push_back(s);
  if (!ok.empty()) {
    ENGINE_TRY(cudaMemcpyAsync(slots_list_, ok.data(), ok.size() * 4, cudaMemcpyHostToDevice, st_));
    launch_finalize_many(trees_, slots_list_, (uint32_t)ok.size(), max_rec, st_);
    ENGINE_TRY(cudaGetLastError());
    if (!sorted.empty()) {
      // the slot list is read by the finalize launch above: the sorted slots go after it
      ENGINE_TRY(cudaMemcpyAsync(slots_list_ + ok.size(), sorted.data(), sorted.size() * 4,
                                 cudaMemcpyHostToDevice, st_));
      launch_leaf_sort(trees_, slots_list_ + ok.size(), (uint32_t)sorted.size(), max_rec, st_);
      ENGINE_TRY(cudaGetLastError());
    }
    ENGINE_TRY(cudaStreamSynchronize(st_));
  }
  for (uint32_t s : sorted) {  // leaves too large for one CTA (shallow trees, cells that stop splitting)
    TreeDev h;
    uint32_t nh = 0;
    ENGINE_TRY(cudaMemcpyAsync(&h, trees_ + s, sizeof(h), cudaMemcpyDeviceToHost, st_));
    ENGINE_TRY(cudaStreamSynchronize(st_));
    ENGINE_TRY(cudaMemcpyAsync(&nh, h.huge_count, 4, cudaMemcpyDeviceToHost, st_));
    ENGINE_TRY(cudaStreamSynchronize(st_));
    nh = std::min(nh, h.huge_cap);
    if (nh == 0) continue;
    std::vector<uint32_t> idx(nh);
    std::vector<TermRec> all(std::min(tc[s], h.term_cap)), recs;
    ENGINE_TRY(cudaMemcpyAsync(idx.data(), h.huge, (size_t)nh * 4, cudaMemcpyDeviceToHost, st_));
    ENGINE_TRY(cudaMemcpyAsync(all.data(), h.terms, all.size() * sizeof(TermRec), cudaMemcpyDeviceToHost, st_));
    ENGINE_TRY(cudaStreamSynchronize(st_));
    for (uint32_t k : idx)
      if (k < all.size()) recs.push_back(all[k]);
    ENGINE_TRY(leaf_sort_huge(host_[s], recs, st_));
    ENGINE_TRY(cudaStreamSynchronize(st_));
  }
  for (size_t i = 0; i < slots.size(); ++i) {
    (*status)[i] = map_status(st[slots[i]]);
    (*levels)[i] = lv[slots[i]];
  }
  return KDT_OK;
}

kdt_status Engine::record_tick(int p) {
  // the counters a step appends to start from zero
  ENGINE_TRY(cudaMemsetAsync(words_ + W_NC0 + (p ^ 1), 0, 4, st_));
  ENGINE_TRY(cudaMemsetAsync(words_ + W_BIGPTS, 0, 4, st_));
  ENGINE_TRY(cudaMemsetAsync(words_ + W_OFFUSED, 0, 4, st_));
  ENGINE_TRY(cudaMemsetAsync(words_ + W_SMALL, 0, 4 * (W_SMALLPTS - W_SMALL + 1), st_));
  StepDev sd = s_;
  sd.cells = big_[p];
  sd.ncells = plan_.maxB;  // a capacity: the count is the device word
  sd.ncells_dev = words_ + W_NC0 + p;
  sd.next_big = big_[p ^ 1];
  sd.next_big_count = words_ + W_NC0 + (p ^ 1);
  sd.off_cur = off_[p];
  sd.obase_cur = obase_[p];
  sd.off_next = off_[p ^ 1];
  sd.obase_next = obase_[p ^ 1];
  const SelectTuning tune = current_tuning();
  sd.tiny_max = tune.tiny_max;
  sd.bitonic_max = tune.bitonic_max;
  sd.warp_max = tune.warp_max;
  launch_big_step(trees_, sd, plan_.max_tiles, plan_.nseg_cap, plan_.bigseg_cap, false, false, plan_.needs.widest,
                  plan_.needs.max_d, plan_.needs.min_d == plan_.needs.max_d ? plan_.needs.max_d : 0, tune, 0,
                  plan_.grid_step, st_, plan_.needs.fourier);
  ENGINE_TRY(cudaGetLastError());
  launch_small(true);
  ENGINE_TRY(cudaGetLastError());
  return KDT_OK;
}

kdt_status Engine::run_graph() {
  // the roots' step (presort, root dims) is sized and launched by the host
  if (!pending_big_.empty() || !pending_small_.empty() || !pending_small_w_.empty()) {
    const kdt_status s = tick();
    if (s != KDT_OK) return s;
  }
  if (!busy()) return KDT_OK;
  // every later step runs inside one graph launch: a while loop whose body is
  // a step over list p0 then one over list p0 ^ 1, each reading its count
  // from the device, until a step leaves no cell (the tick above has
  // launched the subtree kernel over its queue, so that queue is empty)
  const int p0 = cur_;
  uint32_t init[3] = {0u, 0u, 0u};  // W_NC0, W_NC1, W_ITERS
  init[p0] = big_count_;
  ENGINE_TRY(cudaMemcpyAsync(words_ + W_NC0, init, sizeof(init), cudaMemcpyHostToDevice, st_));
  ENGINE_TRY(cudaStreamSynchronize(st_));
  // the steps are recorded on a private stream (the caller's may be the
  // legacy default stream, which cannot be captured); the graph runs on the
  // caller's stream
  struct Graphs {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cs = nullptr;
    ~Graphs() {
      if (ex) cudaGraphExecDestroy(ex);
      if (g) cudaGraphDestroy(g);
      if (cs) cudaStreamDestroy(cs);
    }
  } gr;
  auto fail = [&](const char* what, cudaError_t e) {
    (void)cudaGetLastError();
    if (debug_) std::fprintf(stderr, "kdt graph run: %s: %s\n", what, cudaGetErrorString(e));
    return KDT_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&gr.cs, cudaStreamNonBlocking)) != cudaSuccess) return fail("stream", e);
  if ((e = cudaGraphCreate(&gr.g, 0)) != cudaSuccess) return fail("graph", e);
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, gr.g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return fail("conditional handle", e);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  if ((e = cudaGraphAddNode(&loop, gr.g, nullptr, nullptr, 0, &cp)) != cudaSuccess) return fail("while node", e);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(gr.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail("begin capture", e);
  const cudaStream_t caller = st_;
  st_ = gr.cs;
  const uint64_t l0 = kdt_launch_count();
  kdt_status rec = record_tick(p0);
  if (rec == KDT_OK) rec = record_tick(p0 ^ 1);
  if (rec == KDT_OK) launch_loop_cond(h, words_ + W_NC0 + p0, words_ + W_ITERS, kGraphIterMax, st_);
  const uint64_t per_iter = kdt_launch_count() - l0;
  st_ = caller;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(gr.cs, &captured);
  if (rec != KDT_OK) return rec;
  if (ce != cudaSuccess) return fail("end capture", ce);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("recording", e);
  if ((e = cudaGraphInstantiate(&gr.ex, gr.g, 0)) != cudaSuccess) return fail("instantiate", e);
  if ((e = cudaGraphLaunch(gr.ex, st_)) != cudaSuccess) return fail("launch", e);
  uint32_t fin[3];
  ENGINE_TRY(cudaMemcpyAsync(fin, words_ + W_NC0, sizeof(fin), cudaMemcpyDeviceToHost, st_));
  ENGINE_TRY(cudaStreamSynchronize(st_));
  if (fin[2] > 1) trace_add_launches((uint64_t)(fin[2] - 1) * per_iter);  // replays beyond the recorded one
  graph_iters_ = fin[2];
  if (fin[p0] != 0) return KDT_ERR_CUDA;  // stopped at the iteration cap with cells left
  big_count_ = small_count_ = small_count_w_ = 0;
  big_points_ = small_points_ = 0;
  return KDT_OK;
}

kdt_status Engine::run_to_completion() {
  for (int guard = 0; busy() || !pending_big_.empty() || !pending_small_.empty() || !pending_small_w_.empty();
       ++guard) {
    if (guard > 2 * KDT_MAX_LEVELS + 4) return KDT_ERR_CUDA;
    const kdt_status s = tick();
    if (s != KDT_OK) return s;
  }
  return KDT_OK;
}

}  // namespace kdt
