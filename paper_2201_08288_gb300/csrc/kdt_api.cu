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
#include "kdt_launch.h"

namespace kdt {
namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  // capacities
  int L_cap = 0;
  int small_max = 0;
  uint32_t maxB = 0, cap_small = 0, max_tiles = 0, nseg_cap = 0, bigseg_cap = 0;
  uint64_t term_cap = 0;
  uint32_t slice_cells = 0, grid_sub = 0;
  int sid_bytes = 0;
  // byte offsets into the workspace
  size_t xbuf[2] = {0, 0}, pbuf[2] = {0, 0}, sbuf[2] = {0, 0}, keys = 0, terms = 0, tree = 0,
         words = 0;
  size_t big[2] = {0, 0}, small = 0, tile_base = 0, seg_base = 0, tiles = 0, tile_left = 0,
         tile_loff = 0, tile_mm = 0, child_mm = 0, kdim = 0, mkey = 0, lcount = 0, seg_w = 0, seg_beg = 0,
         seg_cur = 0, seg_med = 0, seg_cell = 0, bigseg = 0, slices = 0;
  size_t total = 0;
};

// Device words at Layout::words.
enum Word {
  W_TERM = 0, W_STATUS, W_LEVELS, W_NTILES, W_BIGSEG, W_HEAD,
  W_NEXTBIG, W_SMALL, W_BIGPTS, W_SMALLPTS,  // read back together after each step
  W_COUNT
};

kdt_status validate(const kdt_params* p) {
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
  if (p->reserved != 0) return KDT_ERR_INVALID_ARG;
  return KDT_OK;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

Layout make_layout(const kdt_params& p) {
  Layout L;
  const uint64_t n = (uint64_t)p.n;
  const int d = p.d;
  L.L_cap = p.depth > 0 ? p.depth : p.max_levels;
  L.small_max = subtree_capacity(d);
  const uint64_t leaves = (uint64_t)1 << L.L_cap;
  L.maxB = (uint32_t)std::min<uint64_t>(n / (uint64_t)(L.small_max + 1) + 1, leaves);
  L.cap_small = (uint32_t)std::min<uint64_t>(n, leaves) + 1;
  L.max_tiles = (uint32_t)(n / kTile + L.maxB + 1);
  L.nseg_cap = L.maxB * (uint32_t)p.r;
  L.bigseg_cap = (uint32_t)(n / (kSelSmallMax + 1) + 1);
  L.term_cap = leaves + 1;
  L.slice_cells = (uint32_t)L.small_max;
  const int sms = device_sms();
  L.grid_sub = (uint32_t)(sms > 0 ? sms : 148);
  L.sid_bytes = p.subset_mode == KDT_SUBSET_EXPLICIT ? (p.subset_id16 ? 2 : 1) : 0;
  const bool widest = p.key_rule == KDT_KEY_WIDEST_SPREAD;

  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  };
  for (int b = 0; b < 2; ++b) {
    L.xbuf[b] = take((size_t)d * n * 4);
    L.pbuf[b] = take(n * 4);
    L.sbuf[b] = take(n * (size_t)L.sid_bytes);
  }
  L.keys = take(n * 4);
  L.terms = take(L.term_cap * sizeof(TermRec));
  L.tree = take(sizeof(TreeDev));
  L.words = take(W_COUNT * 4);
  L.big[0] = take((size_t)L.maxB * sizeof(Cell));
  L.big[1] = take((size_t)L.maxB * sizeof(Cell));
  L.small = take((size_t)L.cap_small * sizeof(Cell));
  L.tile_base = take(((size_t)L.maxB + 1) * 4);
  L.seg_base = take(((size_t)L.maxB + 1) * 4);
  L.tiles = take((size_t)L.max_tiles * sizeof(uint2));
  L.tile_left = take((size_t)L.max_tiles * 4);
  L.tile_loff = take((size_t)L.max_tiles * 4);
  L.tile_mm = take(widest ? (size_t)L.max_tiles * 2 * kMaxDims * 2 * 4 : 0);
  L.child_mm = take(widest ? (size_t)L.maxB * 2 * kMaxDims * 2 * 4 : 0);
  L.kdim = take((size_t)L.maxB * 4);
  L.mkey = take((size_t)L.maxB * 4);
  L.lcount = take((size_t)L.maxB * 4);
  L.seg_w = take((size_t)L.nseg_cap * 4);
  L.seg_beg = take((size_t)L.nseg_cap * 4);
  L.seg_cur = take((size_t)L.nseg_cap * 4);
  L.seg_med = take((size_t)L.nseg_cap * 4);
  L.seg_cell = take((size_t)L.nseg_cap * 4);
  L.bigseg = take((size_t)L.bigseg_cap * 4);
  L.slices = take((size_t)L.grid_sub * 2 * L.slice_cells * sizeof(LCell));
  L.total = off;
  return L;
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

#define KDT_CUDA_TRY(expr)                 \
  do {                                     \
    if ((expr) != cudaSuccess) {           \
      (void)cudaGetLastError();            \
      return KDT_ERR_CUDA;                 \
    }                                      \
  } while (0)

kdt_status build_device(const float* points, const kdt_params& p, uint8_t* ws, const Layout& L,
                        uint32_t* out_perm, float* out_vals, int8_t* out_dims, int64_t* out_offs,
                        int32_t* out_levels, cudaStream_t st) {
  KDT_CUDA_TRY(prepare_subtree_kernel());
  const uint64_t n = (uint64_t)p.n;
  TreeDev h{};
  h.n = p.n;
  h.d = p.d;
  h.r = p.r;
  h.subset_mode = p.subset_mode;
  h.key_rule = p.key_rule;
  h.depth = p.depth;
  h.leaf_size = p.leaf_size;
  h.max_levels = p.max_levels;
  h.stall_limit = p.key_rule == KDT_KEY_CYCLIC ? p.d : 1;
  h.sid_bytes = L.sid_bytes;
  h.small_max = L.small_max;
  h.x_in = points;
  h.sid_in = p.subset_id16 ? (const void*)p.subset_id16 : (const void*)p.subset_id8;
  for (int b = 0; b < 2; ++b) {
    h.xbuf[b] = (float*)(ws + L.xbuf[b]);
    h.pbuf[b] = (uint32_t*)(ws + L.pbuf[b]);
    h.sbuf[b] = (void*)(ws + L.sbuf[b]);
  }
  h.keys = (uint32_t*)(ws + L.keys);
  h.out_perm = out_perm;
  h.out_vals = out_vals;
  h.out_dims = out_dims;
  h.out_offs = out_offs;
  h.terms = (TermRec*)(ws + L.terms);
  h.term_cap = (uint32_t)std::min<uint64_t>(L.term_cap, 0xffffffffull);
  uint32_t* words = (uint32_t*)(ws + L.words);
  h.term_count = words + W_TERM;
  h.status = (int32_t*)(words + W_STATUS);
  h.levels = (int32_t*)(words + W_LEVELS);
  TreeDev* d_tree = (TreeDev*)(ws + L.tree);
  KDT_CUDA_TRY(cudaMemcpyAsync(d_tree, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  KDT_CUDA_TRY(cudaMemsetAsync(words, 0, W_COUNT * 4, st));

  Cell* big[2] = {(Cell*)(ws + L.big[0]), (Cell*)(ws + L.big[1])};
  Cell* small = (Cell*)(ws + L.small);
  LCell* slices = (LCell*)(ws + L.slices);

  // root
  const Cell root{0u, (uint32_t)n, 0u, 0, 0, 0, -1};
  const bool root_terminal = p.depth > 0 ? (n == 0) : (n <= (uint64_t)p.leaf_size);
  uint32_t B = 0, small_total = 0, small_done = 0;
  if (root_terminal) {
    const TermRec tr{0u, (uint32_t)n, 0u, 0};
    const uint32_t one = 1;
    KDT_CUDA_TRY(cudaMemcpyAsync(h.terms, &tr, sizeof(tr), cudaMemcpyHostToDevice, st));
    KDT_CUDA_TRY(cudaMemcpyAsync(h.term_count, &one, 4, cudaMemcpyHostToDevice, st));
    launch_iota(out_perm, (uint32_t)n, st);
  } else if (n <= (uint64_t)L.small_max) {
    KDT_CUDA_TRY(cudaMemcpyAsync(small, &root, sizeof(root), cudaMemcpyHostToDevice, st));
    small_total = 1;
    KDT_CUDA_TRY(cudaMemcpyAsync(words + W_SMALL, &small_total, 4, cudaMemcpyHostToDevice, st));
  } else {
    KDT_CUDA_TRY(cudaMemcpyAsync(big[0], &root, sizeof(root), cudaMemcpyHostToDevice, st));
    B = 1;
  }

  StepDev s{};
  s.tile_base = (uint32_t*)(ws + L.tile_base);
  s.seg_base = (uint32_t*)(ws + L.seg_base);
  s.tiles = (uint2*)(ws + L.tiles);
  s.ntiles_total = words + W_NTILES;
  s.kdim = (uint32_t*)(ws + L.kdim);
  s.mkey = (uint32_t*)(ws + L.mkey);
  s.lcount = (uint32_t*)(ws + L.lcount);
  s.tile_mm = (uint32_t*)(ws + L.tile_mm);
  s.child_mm = (uint32_t*)(ws + L.child_mm);
  s.seg_w = (uint32_t*)(ws + L.seg_w);
  s.seg_beg = (uint32_t*)(ws + L.seg_beg);
  s.seg_cur = (uint32_t*)(ws + L.seg_cur);
  s.seg_med = (uint32_t*)(ws + L.seg_med);
  s.seg_cell = (uint32_t*)(ws + L.seg_cell);
  s.bigseg = (uint32_t*)(ws + L.bigseg);
  s.bigseg_count = words + W_BIGSEG;
  s.tile_left = (uint32_t*)(ws + L.tile_left);
  s.tile_loff = (uint32_t*)(ws + L.tile_loff);
  s.next_big_count = words + W_NEXTBIG;
  s.small = small;
  s.small_count = words + W_SMALL;
  s.small_cap = L.cap_small;
  s.next_big_cap = L.maxB;
  s.next_big_points = words + W_BIGPTS;
  s.small_points = words + W_SMALLPTS;

  const bool widest = p.key_rule == KDT_KEY_WIDEST_SPREAD;
  int cur = 0;
  int level = 0;
  uint64_t big_points = B ? n : 0, small_points_done = 0;
  uint64_t small_points_total = (!root_terminal && B == 0) ? n : 0;
  while (B > 0) {
    s.cells = big[cur];
    s.ncells = B;
    s.next_big = big[cur ^ 1];
    KDT_CUDA_TRY(cudaMemsetAsync(s.next_big_count, 0, 4, st));
    KDT_CUDA_TRY(cudaMemsetAsync(s.next_big_points, 0, 4, st));
    launch_big_step(d_tree, s, L.max_tiles, B * (uint32_t)p.r, L.bigseg_cap, widest && level == 0, widest,
                    p.d, big_points, st);
    KDT_CUDA_TRY(cudaGetLastError());
    uint32_t counts[4];
    KDT_CUDA_TRY(cudaMemcpyAsync(counts, words + W_NEXTBIG, 16, cudaMemcpyDeviceToHost, st));
    KDT_CUDA_TRY(cudaStreamSynchronize(st));
    small_total = std::min(counts[1], L.cap_small);
    small_points_total = counts[3];
    if (small_total > small_done) {
      launch_subtree(d_tree, small + small_done, small_total - small_done, words + W_HEAD, slices,
                     L.slice_cells, std::min(L.grid_sub, small_total - small_done),
                     small_points_total - small_points_done, st);
      KDT_CUDA_TRY(cudaGetLastError());
      small_done = small_total;
      small_points_done = small_points_total;
    }
    B = std::min(counts[0], L.maxB);
    big_points = counts[2];
    cur ^= 1;
    ++level;
  }
  if (small_total > small_done) {
    launch_subtree(d_tree, small + small_done, small_total - small_done, words + W_HEAD, slices,
                   L.slice_cells, std::min(L.grid_sub, small_total - small_done),
                   small_points_total - small_points_done, st);
    KDT_CUDA_TRY(cudaGetLastError());
  }
  uint32_t fin[3];
  KDT_CUDA_TRY(cudaMemcpyAsync(fin, words, 12, cudaMemcpyDeviceToHost, st));
  KDT_CUDA_TRY(cudaStreamSynchronize(st));
  if (fin[W_STATUS] != ST_OK) return map_status((int32_t)fin[W_STATUS]);
  launch_finalize(d_tree, words + W_TERM, std::min<uint64_t>(fin[W_TERM], L.term_cap), st);
  KDT_CUDA_TRY(cudaGetLastError());
  KDT_CUDA_TRY(cudaStreamSynchronize(st));
  if (out_levels) *out_levels = p.depth > 0 ? p.depth : (int32_t)fin[W_LEVELS];
  return KDT_OK;
}

}  // namespace

// Build with a caller-provided workspace that is never NULL; used by entry
// points that own their workspace memory. Allocates nothing.
kdt_status build_in_workspace(const float* points, const kdt_params* p, void* workspace, size_t workspace_bytes,
                              uint32_t* out_perm, float* out_split_vals, int8_t* out_split_dims,
                              int64_t* out_node_offsets, int32_t* out_levels, cudaStream_t st) {
  const kdt_status v = validate(p);
  if (v != KDT_OK) return v;
  if ((p->n > 0 && (!points || !out_perm)) || !out_node_offsets || !workspace) return KDT_ERR_INVALID_ARG;
  const int L_cap = p->depth > 0 ? p->depth : p->max_levels;
  if (L_cap > 0 && (!out_split_vals || !out_split_dims)) return KDT_ERR_INVALID_ARG;
  const Layout L = make_layout(*p);
  if (workspace_bytes < L.total) return KDT_ERR_CAPACITY;
  if ((uintptr_t)workspace % kAlign) return KDT_ERR_INVALID_ARG;
  return build_device(points, *p, (uint8_t*)workspace, L, out_perm, out_split_vals, out_split_dims,
                      out_node_offsets, out_levels, st);
}

}  // namespace kdt

using namespace kdt;

extern "C" {

kdt_status kdt_workspace_size(const kdt_params* p, size_t* bytes) {
  const kdt_status v = validate(p);
  if (v != KDT_OK) return v;
  if (!bytes) return KDT_ERR_INVALID_ARG;
  *bytes = make_layout(*p).total;
  return KDT_OK;
}

kdt_status kdt_build(const float* points, const kdt_params* p, void* workspace, size_t workspace_bytes,
                     uint32_t* out_perm, float* out_split_vals, int8_t* out_split_dims,
                     int64_t* out_node_offsets, int32_t* out_levels, void* stream) {
  const kdt_status v = validate(p);
  if (v != KDT_OK) return v;
  if ((p->n > 0 && (!points || !out_perm)) || !out_node_offsets) return KDT_ERR_INVALID_ARG;
  const int L_cap = p->depth > 0 ? p->depth : p->max_levels;
  if (L_cap > 0 && (!out_split_vals || !out_split_dims)) return KDT_ERR_INVALID_ARG;
  const Layout L = make_layout(*p);
  cudaStream_t st = (cudaStream_t)stream;
  void* owned = nullptr;
  if (!workspace) {
    if (cudaMalloc(&owned, L.total) != cudaSuccess) {
      (void)cudaGetLastError();
      return KDT_ERR_OOM;
    }
    workspace = owned;
  } else if (workspace_bytes < L.total) {
    return KDT_ERR_CAPACITY;
  } else if ((uintptr_t)workspace % kAlign) {
    return KDT_ERR_INVALID_ARG;
  }
  kdt_status s = build_device(points, *p, (uint8_t*)workspace, L, out_perm, out_split_vals,
                              out_split_dims, out_node_offsets, out_levels, st);
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  return s;
}

kdt_status kdt_workspace_size_host(const kdt_params* p, size_t* bytes) {
  const kdt_status v = validate(p);
  if (v != KDT_OK) return v;
  if (!bytes) return KDT_ERR_INVALID_ARG;
  const Layout L = make_layout(*p);
  const uint64_t n = (uint64_t)p->n;
  const uint64_t leaves = (uint64_t)1 << L.L_cap;
  size_t extra = align_up((size_t)p->d * n * 4) + align_up(n * (size_t)L.sid_bytes) +
                 align_up(n * 4) + align_up(leaves * 4) + align_up(leaves) + align_up((leaves + 1) * 8);
  *bytes = L.total + extra;
  return KDT_OK;
}

kdt_status kdt_build_host(const float* points_host, const kdt_params* p, void* workspace,
                          size_t workspace_bytes, uint32_t* out_perm_host, float* out_split_vals_host,
                          int8_t* out_split_dims_host, int64_t* out_node_offsets_host, int32_t* out_levels,
                          void* stream) {
  const kdt_status v = validate(p);
  if (v != KDT_OK) return v;
  if ((p->n > 0 && (!points_host || !out_perm_host)) || !out_node_offsets_host) return KDT_ERR_INVALID_ARG;
  size_t need = 0;
  kdt_workspace_size_host(p, &need);
  const Layout L = make_layout(*p);
  cudaStream_t st = (cudaStream_t)stream;
  void* owned = nullptr;
  if (!workspace) {
    if (cudaMalloc(&owned, need) != cudaSuccess) {
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
  const uint64_t leaves = (uint64_t)1 << L.L_cap;
  size_t off = L.total;
  float* d_pts = (float*)(ws + off);
  off += align_up((size_t)p->d * n * 4);
  void* d_sid = ws + off;
  off += align_up(n * (size_t)L.sid_bytes);
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
    if (L.sid_bytes) {
      const void* hs = p->subset_id16 ? (const void*)p->subset_id16 : (const void*)p->subset_id8;
      if (n && cudaMemcpyAsync(d_sid, hs, n * (size_t)L.sid_bytes, cudaMemcpyHostToDevice, st) !=
                   cudaSuccess) {
        s = KDT_ERR_CUDA;
        break;
      }
      pd.subset_id8 = p->subset_id8 ? (const uint8_t*)d_sid : nullptr;
      pd.subset_id16 = p->subset_id16 ? (const uint16_t*)d_sid : nullptr;
    }
    s = build_device(d_pts, pd, ws, L, d_perm, d_vals, d_dims, d_offs, &levels, st);
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
  }
  return "unknown status";
}

}  // extern "C"
