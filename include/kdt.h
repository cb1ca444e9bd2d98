/*
 * kdt.h -- C ABI of the GB300 (sm_103a) level-by-level k-d tree build with
 * subset-median splits.
 *
 * Paper: A. Chakravorty, W. S. Cleveland, P. J. Wolfe, "Scalable k-d trees
 * for distributed data" (arXiv 2201.08288).
 *
 * What a build computes (all integer / compare arithmetic, bit-exact):
 *   - The canonical k-d tree structure of Sec. 1 and Sec. 2: level l (0-based)
 *     splits each of its 2^l cells along a key coordinate; a tree of depth D
 *     has 2^D - 1 split statistics in level order (Sec. 2, last paragraph;
 *     children of heap node h are 2h+1 and 2h+2).
 *   - Key coordinate: cycled x, y, z, ... by level (Sec. 1), or per cell the
 *     coordinate of widest dispersion (Sec. 1, Friedman rule), read as the
 *     range (double)max - (double)min of the cell's points; lowest index wins
 *     ties.
 *   - The index set is partitioned into r subsets (Sec. 3.2, additivity of the
 *     statistics over any partition; App. C.2, the user-supplied partition
 *     I_1..I_R). For every (cell, subset) the build takes the lower median of
 *     the subset's keys in the cell (0-based rank (w-1)/2); the cell's split is
 *     the count-weighted lower median of those medians: the smallest subset
 *     median m such that the subsets whose median is <= m hold at least half of
 *     the cell's points. (The paper combines additive Fourier moments instead,
 *     Sec. 3.2 Eq. (1)-(2); this combine rule is the library's.)
 *   - Points with key <= split go left ("ties to the left"), others right; the
 *     partition is stable, so every leaf lists its points in increasing
 *     original index. Keys compare as floats with -0.0 < +0.0.
 *   - Empty cells (depth mode) and terminal cells (leaf mode) record split
 *     dim -1 and value +inf and pass all their points to the left child. In
 *     leaf mode a cell is terminal when it holds <= leaf_size points or when
 *     its last s splits each left the right child empty (s = d for cyclic
 *     keys, s = 1 for widest spread); L is the first level whose cells are all
 *     terminal.
 *
 * Conventions: every pointer argument marked "device" is a CUDA device
 * pointer owned by the caller; the library never frees it. Calls are issued
 * on `stream` (a cudaStream_t; NULL = legacy default stream) and return after
 * the build has finished: the host waits on the stream while a build runs
 * (it reads the next level's cell counts between levels) and once at its end
 * (the status). So no build or query may be issued on a stream that is being
 * captured into a CUDA graph: such a call returns KDT_ERR_INVALID_ARG before
 * it touches the stream. No function allocates device memory except where
 * stated.
 */
#ifndef KDT_H
#define KDT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kdt_status {
  KDT_OK = 0,
  KDT_ERR_INVALID_ARG = 1, /* a parameter is out of range or a pointer is missing      */
  KDT_ERR_NAN_INPUT = 2,   /* a coordinate is NaN; outputs are undefined              */
  KDT_ERR_OOM = 3,         /* the library could not allocate memory it needed          */
  KDT_ERR_CUDA = 4,        /* a CUDA runtime call failed                              */
  KDT_ERR_CAPACITY = 5,    /* a caller-provided buffer is too small                   */
  KDT_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                           */
  KDT_ERR_LEVEL_CAP = 7,   /* leaf mode needs more than max_levels levels             */
  KDT_ERR_BUSY = 8,        /* the server cannot take the request now                  */
  KDT_ERR_NOT_FOUND = 9,   /* unknown server ticket                                   */
  KDT_ERR_CANCELLED = 10   /* the server request was cancelled before it ran          */
} kdt_status;

typedef enum kdt_key_rule { KDT_KEY_CYCLIC = 0, KDT_KEY_WIDEST_SPREAD = 1 } kdt_key_rule;

/* How points map to the r subsets (Sec. 3.2 / App. C.2 partition of I). */
typedef enum kdt_subset_mode {
  KDT_SUBSET_MOD = 0,        /* subset(i) = i mod r                                 */
  KDT_SUBSET_CONTIGUOUS = 1, /* subset(i) = floor(i * r / n), 64-bit arithmetic     */
  KDT_SUBSET_EXPLICIT = 2    /* subset(i) = subset_id8[i] or subset_id16[i] (< r)   */
} kdt_subset_mode;

/* Largest accepted depth / max_levels. */
#define KDT_MAX_LEVELS 30
/* Largest accepted number of subsets on the CUDA path. */
#define KDT_MAX_SUBSETS 4096
/* Largest accepted dimension. */
#define KDT_MAX_DIMS 64

/* How a cell's split is formed from the lower medians of its (cell, subset)
 * segments. WEIGHTED: the smallest subset median m such that the subsets
 * whose median is <= m hold at least half of the cell's points (each subset
 * weighs its size; the library's default). UNWEIGHTED: every non-empty subset
 * counts once, the split is the lower median (rank (m-1)/2 of m, ties by
 * subset id) of the subset medians, the plain median of medians. The paper
 * combines additive moments instead (Sec. 3.2); both rules are the
 * library's. */
typedef enum { KDT_COMBINE_WEIGHTED = 0, KDT_COMBINE_UNWEIGHTED = 1 } kdt_combine_rule;

typedef struct kdt_params {
  int64_t n;                     /* points, 0 <= n <= 2^32 - 1                          */
  int32_t d;                     /* coordinates per point, 1..64                        */
  int32_t subset_mode;           /* kdt_subset_mode                                     */
  int32_t r;                     /* subsets, 1..4096                                    */
  int32_t key_rule;              /* kdt_key_rule                                        */
  const uint8_t *subset_id8;     /* explicit mode: device, [n], exactly one of the two  */
  const uint16_t *subset_id16;   /*   id arrays non-NULL; every id < r                  */
  int32_t depth;                 /* > 0: fixed depth (2^depth leaves); 0: leaf mode     */
  int32_t leaf_size;             /* leaf mode: cells with <= leaf_size points stop (>= 1) */
  int32_t max_levels;            /* leaf mode: output capacity, 2^max_levels leaves     */
  int32_t fourier_j;             /* 0: the exact subset-median split (Sec. 2). 1..32: the  */
                                 /* paper's estimator (Sec. 3): each split is the root of  */
                                 /* Eq. (kd:eq:b) built from the cell's sums of the first  */
                                 /* 2J+1 terms of Lemma 1's expansion (cyclic keys, depth  */
                                 /* mode, every coordinate in (0,1); plain builds only;    */
                                 /* subsets do not change its sums, so r and the ids are   */
                                 /* ignored)                                               */
  int32_t combine_rule;          /* kdt_combine_rule: how a cell's split is formed from its */
                                 /* subsets' lower medians (ignored when fourier_j > 0)    */
} kdt_params;

/* Largest fourier_j. */
#define KDT_FOURIER_MAX_J 32

/*
 * Bytes of device workspace kdt_build needs for these parameters on the
 * current device. The workspace holds two ping-pong copies of the points,
 * permutation and subset ids, a key scratch array and per-level tables.
 * Errors: KDT_ERR_INVALID_ARG.
 */
kdt_status kdt_workspace_size(const kdt_params *p, size_t *bytes);

/*
 * Build one tree.
 *   points           device, float32 SoA [d][n]: points[j*n + i] = coordinate j
 *                    of point i. Read only.
 *   workspace        device, >= kdt_workspace_size bytes, 256-byte aligned; or
 *                    NULL, in which case the library allocates it (cudaMalloc)
 *                    and frees it before returning.
 *   out_perm         device [n]: original index of the point at each position of
 *                    the final order (leaves in order, increasing index inside).
 *   out_split_vals   device [2^L - 1]: split value of each node in level order
 *                    (bit-identical to a coordinate of the node's points; with
 *                    fourier_j > 0 the estimator's root rounded to float).
 *   out_split_dims   device [2^L - 1]: split coordinate, -1 for sentinels.
 *   out_node_offsets device [2^L + 1]: leaf k holds out_perm[offs[k]..offs[k+1]).
 *   out_levels       host: L, the number of split levels built (depth, or the
 *                    leaf-mode result). Capacity: outputs must hold
 *                    2^depth (depth mode) or 2^max_levels (leaf mode) leaves.
 * Errors: KDT_ERR_INVALID_ARG (also: fourier_j > 0 and a coordinate outside the
 *         open interval (0,1)), KDT_ERR_NAN_INPUT, KDT_ERR_LEVEL_CAP,
 *         KDT_ERR_CAPACITY (workspace too small), KDT_ERR_OOM, KDT_ERR_CUDA.
 */
kdt_status kdt_build(const float *points, const kdt_params *p, void *workspace,
                     size_t workspace_bytes, uint32_t *out_perm, float *out_split_vals,
                     int8_t *out_split_dims, int64_t *out_node_offsets, int32_t *out_levels,
                     void *stream);

/*
 * Same build with HOST buffers: points, the explicit subset ids in p and all
 * outputs are host pointers (pinned memory gives full copy bandwidth). The
 * inputs are copied to the device, the tree is built, the outputs are copied
 * back, all on `stream`, before returning.
 *   workspace  device, >= kdt_workspace_size_host bytes (or NULL: allocated
 *              and freed by the call).
 * Errors: as kdt_build.
 */
kdt_status kdt_workspace_size_host(const kdt_params *p, size_t *bytes);
kdt_status kdt_build_host(const float *points_host, const kdt_params *p, void *workspace,
                          size_t workspace_bytes, uint32_t *out_perm_host,
                          float *out_split_vals_host, int8_t *out_split_dims_host,
                          int64_t *out_node_offsets_host, int32_t *out_levels, void *stream);

/* ---- batched builds -----------------------------------------------------
 * Many independent trees (different n, d, r, rules) built together: every
 * level step runs once over the cells of all trees (each tree at its own
 * level), and every cell that fits in shared memory is finished by one
 * persistent launch per step. After the roots' step, all steps run as one
 * CUDA graph launch: a conditional while node repeats a recorded pair of
 * steps that read their cell counts on the device, until no cell is left.
 * Each tree's outputs equal its kdt_build outputs bit for bit. */
typedef struct kdt_tree_desc {
  const float *points;         /* device, float32 SoA [d][n] (as kdt_build)              */
  kdt_params params;           /* per tree; explicit subset ids are device pointers      */
  uint32_t *out_perm;          /* device outputs, sized as for kdt_build                 */
  float *out_split_vals;
  int8_t *out_split_dims;
  int64_t *out_node_offsets;
} kdt_tree_desc;

/* Device workspace for kdt_build_batched with these trees. */
kdt_status kdt_workspace_size_batched(const kdt_tree_desc *trees, int32_t num_trees, size_t *bytes);
/*
 * Build num_trees trees. workspace: device, >= kdt_workspace_size_batched
 * bytes (or NULL: allocated and freed by the call). out_levels, out_status:
 * host arrays of num_trees (may be NULL) receiving each tree's L and status;
 * a failing tree (NaN input, level cap) does not stop the others. Returns
 * KDT_OK when every tree succeeded, else the first tree's error (or a call
 * error: KDT_ERR_INVALID_ARG, KDT_ERR_CAPACITY, KDT_ERR_OOM, KDT_ERR_CUDA).
 */
kdt_status kdt_build_batched(const kdt_tree_desc *trees, int32_t num_trees, void *workspace,
                             size_t workspace_bytes, int32_t *out_levels, kdt_status *out_status,
                             void *stream);

/* ---- serving ------------------------------------------------------------
 * A request loop with continuous batching. The server allocates one device
 * arena of mem_budget_bytes at creation (its only allocation) and runs a
 * worker thread. Requests are admitted in arrival order whenever a slot
 * (max_trees_in_flight), arena memory for the tree's working buffers and
 * table capacity are free; between two level steps, so a request that
 * arrives while others are being built joins the next step and its work
 * overlaps theirs on the device. Points and outputs stay in the caller's
 * device buffers (they must stay valid until the request completes). A
 * request's outputs are identical to kdt_build's, alone or in any mix. */
typedef struct kdt_server kdt_server;
typedef struct kdt_server_info {
  uint64_t submitted, admitted, completed, ticks;
  int32_t in_flight, peak_in_flight;
  uint64_t arena_bytes, arena_bytes_in_use;
  uint64_t cancelled, engine_failures;
} kdt_server_info;

/* Create a server on the current device. Errors: KDT_ERR_INVALID_ARG (budget
 * below 64 MiB, max_trees_in_flight < 1), KDT_ERR_OOM, KDT_ERR_CUDA. */
kdt_status kdt_server_create(size_t mem_budget_bytes, int32_t max_trees_in_flight, kdt_server **out);
/* Queue a build. *ticket identifies it. The server reads the request's
 * device buffers on its own stream at some later time: the points (and
 * subset ids) must already be complete when kdt_server_submit is called (for
 * example, synchronise the stream that wrote them), and all buffers of the
 * request must stay valid until kdt_server_poll reports it finished.
 * KDT_ERR_CAPACITY: the request can never fit the budget; KDT_ERR_INVALID_ARG
 * as kdt_build. */
kdt_status kdt_server_submit(kdt_server *s, const kdt_tree_desc *request, uint64_t *ticket);
/* Wait up to wait_ms (< 0: forever, 0: do not wait) for a ticket. KDT_OK: the
 * request finished; *result holds its build status, *levels its L and
 * *latency_ms the time from submit to completion; the ticket is released.
 * KDT_ERR_BUSY: not finished yet. KDT_ERR_NOT_FOUND: unknown ticket. */
kdt_status kdt_server_poll(kdt_server *s, uint64_t ticket, int32_t wait_ms, kdt_status *result,
                           int32_t *levels, double *latency_ms);
/* Cancel a queued request: it is not built, and kdt_server_poll reports it
 * finished with *result = KDT_ERR_CANCELLED. A request already admitted to the
 * GPU (or finished) cannot be cancelled: KDT_ERR_BUSY (poll it as usual).
 * KDT_ERR_NOT_FOUND: unknown or already released ticket. */
kdt_status kdt_server_cancel(kdt_server *s, uint64_t ticket);
/* Counters of the server (requests, ticks, occupancy, failures). */
kdt_status kdt_server_stats(kdt_server *s, kdt_server_info *out);
/* Finish the requests in flight, drop the queued ones, free the arena. */
kdt_status kdt_server_destroy(kdt_server *s);
/* Failure isolation. A build whose tree fails on the device (NaN input, level
 * cap, a bounded wait that gave up) ends alone with that status; the other
 * requests are unaffected. If a level step of the engine itself fails, every
 * request on the GPU at that moment ends with the step's status and the
 * engine's tables are cleared; queued requests then proceed. If the tables
 * cannot be cleared (the device is unusable), every queued request ends with
 * the status too, waiting pollers are woken, and later submits return it. */

/* ---- tuning -------------------------------------------------------------
 * The lower median of every (cell, subset) segment (paper, Sec. 2: the
 * medians computed independently on the r subsets) takes one of four paths by
 * the segment's size: one thread sorting it in registers; one warp with a
 * bitonic network; one warp with a radix select; one CTA with a radix select.
 * Where the paths change, the CTA's size and the width of its radix digits
 * are tunable. Every choice gives the same outputs, bit for bit: the choices
 * trade only speed, and kdt_autotune times them on the caller's own trees.
 */
typedef struct kdt_tuning {
  int32_t tiny_max;     /* one thread per segment up to this many keys: 8 to 64 (x2)   */
  int32_t bitonic_max;  /* a warp's bitonic network up to this many: 64, 128 or 256    */
  int32_t warp_max;     /* a warp's radix select up to this many: 1024, 2048 or 4096   */
  int32_t cta_threads;  /* threads of the CTA radix select: 256 or 512                 */
  int32_t digit_bits;   /* digit width of the CTA radix select: 8 (4 passes) or 11 (3) */
  int32_t reserved[3];  /* zero                                                        */
} kdt_tuning;

/* The library's defaults. t: host, filled. */
void kdt_tuning_default(kdt_tuning *t);
/* Install t (host; NULL: the defaults) for the level steps that start after
 * the call, in every build of this process (plain, batched, served). Errors:
 * KDT_ERR_INVALID_ARG (a field outside its choices, reserved not zero), and
 * the tuning in force is kept. */
kdt_status kdt_set_tuning(const kdt_tuning *t);
/* The tuning in force. t: host, filled. Errors: KDT_ERR_INVALID_ARG (NULL). */
kdt_status kdt_get_tuning(kdt_tuning *t);
/*
 * Autotuner: time candidate tunings on these trees and keep the fastest.
 * Starting from the tuning in force, it sweeps one field at a time over its
 * choices (the others held at the best found so far); each candidate is timed
 * as `repeats` batched builds of the trees (CUDA events on `stream`) after
 * one untimed build. The fastest is installed (kdt_set_tuning) and returned in
 * *best, its time per build in *best_ms (host, may be NULL). Arguments as
 * kdt_build_batched (the trees' outputs are overwritten; workspace NULL:
 * allocated once for all candidates and freed). repeats: 1..100.
 * Errors: those of kdt_build_batched; KDT_ERR_INVALID_ARG (best NULL,
 * repeats out of range). On an error the tuning in force is unchanged.
 */
kdt_status kdt_autotune(const kdt_tree_desc *trees, int32_t num_trees, void *workspace, size_t workspace_bytes,
                        int32_t repeats, kdt_tuning *best, float *best_ms, void *stream);

/* ---- tracing ------------------------------------------------------------
 * Every kernel launch of the library is counted. With tracing enabled, each
 * launch is also bracketed by two CUDA events recorded on its stream;
 * kdt_trace_read waits for them and reports, per kernel, the number of
 * launches, their summed device time and the points they processed. */
typedef struct kdt_kernel_stat {
  const char *name;   /* kernel name (static string)                       */
  uint64_t launches;  /* timed launches                                    */
  double total_ms;    /* summed event-to-event device time                 */
  uint64_t units;     /* points processed by those launches (0: not counted) */
} kdt_kernel_stat;

/* Turn per-launch event timing on (1) or off (0). Process-wide. */
void kdt_trace_enable(int32_t on);
/* Kernel launches issued by the library since the process started. */
uint64_t kdt_launch_count(void);
/* Fill up to max entries (out may be NULL); returns the number of kernels
 * with data. Synchronises on the recorded events. reset != 0 clears totals. */
int32_t kdt_trace_read(kdt_kernel_stat *out, int32_t max, int32_t reset);

/*
 * kdt_build without any memory allocation, for callers that cannot call
 * cudaMalloc (for example a host application that runs this library under a
 * fixed device-memory budget owned by its own allocator, or a latency-critical
 * path that cannot afford cudaMalloc's cost and implicit synchronisation). The
 * paper has no counterpart: this is a property of the library, not of the
 * method.
 *   The workspace is a 64 MiB array in device memory that the library defines
 *   statically; every GPU that loads the library keeps it until the process
 *   exits. Problems whose kdt_workspace_size exceeds 64 MiB are rejected with
 *   KDT_ERR_CAPACITY (about one million 3-D points; fewer in higher d).
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; later calls reuse it.
 *   Like kdt_build, every call waits on its stream while it runs, so none
 *   may be issued during a stream capture (see the conventions at the top of
 *   this file).
 *   All calls on a device share the array: calls that overlap on the GPU (for
 *   example on two streams) race and produce garbage. Issue them in order.
 *   Arguments, outputs and errors are those of kdt_build (without workspace).
 */
kdt_status kdt_build_noalloc(const float *points, const kdt_params *p, uint32_t *out_perm,
                             float *out_split_vals, int8_t *out_split_dims,
                             int64_t *out_node_offsets, int32_t *out_levels, void *stream);

/* ---- sharded build --------------------------------------------------------
 * The paper's distributed setting (App. C.2: the data stays in its R subsets,
 * a map step runs on each and a reduce combines their statistics; Sec. 3.2:
 * statistics of any partition into subsets combine exactly), emulated with
 * `shards` logical shards on the current device. Subset s belongs to shard
 * s % shards; each shard holds only its own points. Every level, each shard
 * takes the lower median and size of its (cell, subset) segments, an
 * all-gather among the shards hands everyone the other shards' pairs of the
 * same cell (and, for widest spread, the per-coordinate min / max of the
 * root and of every child), every shard runs the same combine, and the
 * partition is local. At the end the shards' leaves are merged by original
 * index. The outputs are bit-identical to kdt_build's for the same points and
 * parameters.
 *   Depth mode only (p->depth >= 1; fourier_j = 0); 1 <= shards <= 16.
 *   Arguments and outputs as kdt_build (no workspace: the call allocates its
 *   own with cudaMalloc, in two parts, and frees it before returning).
 * Errors: KDT_ERR_INVALID_ARG (also: depth 0, fourier_j > 0, shards out of
 *         range, an explicit subset id >= r), KDT_ERR_NAN_INPUT, KDT_ERR_OOM,
 *         KDT_ERR_CUDA. */
kdt_status kdt_build_sharded(const float *points, const kdt_params *p, int32_t shards, uint32_t *out_perm,
                             float *out_split_vals, int8_t *out_split_dims, int64_t *out_node_offsets,
                             int32_t *out_levels, void *stream);

/* ---- queries on a built tree ----------------------------------------------
 * The searches a k-d tree is built for (Sec. 1): only the cells a query's
 * region can reach are visited. The tree is a build's output: points (device,
 * float32 SoA [d][n], the build's input), perm, split_vals, split_dims and
 * node_offsets (device) and L = levels. Query arrays are device SoA [d][nq].
 * One CUDA thread per query; the call returns when the results are written.
 * Errors: KDT_ERR_INVALID_ARG (sizes out of range, missing pointers),
 *         KDT_ERR_CUDA. */

/* Box query: point i is inside query q when lo[j][q] <= x_j(i) <= hi[j][q] for
 * every coordinate j, comparing as the build does (float order with -0.0
 * below +0.0). out_count [nq]: the number of points inside. out_list (device
 * [nq][list_cap], or NULL): the original indices of the first list_cap points
 * found (in no particular order; out_count may exceed list_cap). */
kdt_status kdt_query_box(const float *points, int64_t n, int32_t d, const uint32_t *perm,
                         const float *split_vals, const int8_t *split_dims, const int64_t *node_offsets,
                         int32_t levels, const float *lo, const float *hi, int32_t nq, uint32_t *out_count,
                         uint32_t *out_list, uint32_t list_cap, void *stream);

/* Largest k of kdt_query_knn. */
#define KDT_KNN_MAX_K 32

/* k nearest neighbours of each query (1 <= k <= KDT_KNN_MAX_K): out_idx
 * [nq][k] original indices and out_dist2 [nq][k] squared Euclidean distances
 * (float64: each coordinate's difference and square rounded to double, summed
 * over j = 0..d-1 in order, no fused multiply-add), nearest first, ties by the
 * smaller index. With fewer than k points, the remaining entries hold index
 * 0xffffffff and distance +inf. */
kdt_status kdt_query_knn(const float *points, int64_t n, int32_t d, const uint32_t *perm,
                         const float *split_vals, const int8_t *split_dims, const int64_t *node_offsets,
                         int32_t levels, const float *queries, int32_t nq, int32_t k, uint32_t *out_idx,
                         double *out_dist2, void *stream);

/* ---- fault injection ----------------------------------------------------
 * Host-side hooks that make a failure happen on purpose, so that the error
 * paths can be tested without faulting a GPU. All are off by default; each
 * kind holds a count of the events it still fails (0 = off).
 *   KDT_FAULT_ALLOC        the library's next `count` device allocations
 *                          (kdt_build, kdt_build_host, kdt_build_batched and
 *                          kdt_autotune with a NULL workspace; the server's
 *                          arena) fail as if the device were out of memory:
 *                          the call returns KDT_ERR_OOM, having freed
 *                          whatever it had allocated.
 *   KDT_FAULT_SERVER_STEP  a server's next `count` level steps fail with
 *                          KDT_ERR_CUDA before launching anything.
 *   KDT_FAULT_SERVER_RESET the engine's next `count` table clears after a
 *                          failed server step fail (the device counts as
 *                          unusable for that server).
 *   KDT_FAULT_WAIT         in the next `count` launches of the in-shared-memory
 *                          subtree kernel, every CTA first waits on an
 *                          mbarrier phase that nothing completes, with a
 *                          bound of 1024 tries and no copy in flight; the wait
 *                          gives up, the trees whose cells the launch held end
 *                          with KDT_ERR_TIMEOUT, and the CTAs drain the rest of
 *                          their queue without touching it.
 * Errors: KDT_ERR_INVALID_ARG (unknown kind, count < 0). */
typedef enum kdt_fault {
  KDT_FAULT_ALLOC = 1,
  KDT_FAULT_SERVER_STEP = 2,
  KDT_FAULT_SERVER_RESET = 3,
  KDT_FAULT_WAIT = 4
} kdt_fault;
kdt_status kdt_fault_inject(kdt_fault kind, int32_t count);
/* Turn every fault kind off. */
void kdt_fault_clear(void);

/* Largest cell (points) the in-shared-memory subtree kernel takes for d
 * coordinates; larger cells are split by the multi-CTA level pipeline. */
int32_t kdt_subtree_capacity(int32_t d);

/* Static description of a status code. */
const char *kdt_status_str(kdt_status s);

#ifdef __cplusplus
}
#endif
#endif /* KDT_H */
