/*
 * slimsell.h -- C ABI of the GB300 SlimSell BFS library (libslimsell.so).
 *
 * BFS as repeated sparse-matrix x dense-vector products over the tropical,
 * real, boolean and sel-max semirings (Section III-A) on the SlimSell layout
 * (Section III-B: Sell-C-sigma with the value array dropped and padding
 * marked by -1 in col), with SlimWork chunk skipping (Section III-C) and
 * SlimChunk splitting of long chunks (Section III-D).
 *
 * Conventions for every entry point:
 *  - Pointers prefixed d_ are DEVICE pointers on the current CUDA device;
 *    h_ pointers are host pointers.  Sizes are element counts.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The caller owns every buffer it passes in; the handle owns its layout and
 *    scratch buffers, which slimsell_destroy frees.
 *  - Vertex ids are the caller's original ids in [0, n).  Unreached vertices get
 *    dist = parent = -1; the root gets dist = 0 and parent = root.
 *  - Parents are canonical: the largest-id neighbour one level closer to the
 *    root, for every semiring (sel-max yields it directly, the others through
 *    the DP transformation of Section II-C).  Results do not depend on C, sigma,
 *    the split width or the iteration variant.
 *  - Errors: a non-zero ss_status is returned and slimsell_last_error() gives a
 *    message (thread-local, valid until the next call on that thread).
 *    Invalid arguments are detected on the host before any work is queued.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef SLIMSELL_H
#define SLIMSELL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slimsell_graph* slimsell_handle;
typedef struct slimsell_batch* slimsell_batch_handle;

/* Semirings of Section III-A. */
typedef enum {
  SS_TROPICAL = 0, /* (R u {inf}, min, +, inf, 0): f_k = x_k = A' (x) f_{k-1}          */
  SS_REAL = 1,     /* (R, +, *, 0, 1): f_k = x_k (.) g_k; fp32 values (path counts)    */
  SS_BOOLEAN = 2,  /* ({0,1}, |, &, 0, 1): f_k = x_k & g_k; 1-bit frontier            */
  SS_SELMAX = 3    /* (R, max, *, -inf, 1): x carries vertex ids; parents come out directly */
} ss_semiring;

typedef enum {
  SS_OK = 0,
  SS_ERR_INVALID = 1,     /* bad argument (checked on the host, nothing queued)  */
  SS_ERR_OOM = 2,         /* device allocation failed                            */
  SS_ERR_CUDA = 3,        /* a CUDA call failed; see slimsell_last_error()       */
  SS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                  */
  SS_ERR_UNSUPPORTED = 5  /* combination not implemented                         */
} ss_status;

/* Per-iteration schedule (how each frontier expansion is executed; results are
 * identical for all of them). */
typedef enum {
  SS_V_FULL = 0,          /* every chunk, every column (plain BFS-SpMV, Section III-A)        */
  SS_V_SLIMWORK = 1,      /* skip chunks whose rows are all visited (SlimWork, Section III-C) */
  SS_V_PUSH = 2,          /* compacted-frontier push (work-avoidance variant, Section V); falls
                             back to PULL_FILTERED when the frontier exceeds the unit buffer;
                             frontiers of at most 4096 vertices and 8192 edges per CTA of a
                             thread-block cluster run in the cluster push
                             (SS_VARIANT_PUSH_LOCAL)                                           */
  SS_V_PULL_FILTERED = 3, /* pull over unvisited rows only, stopping at the first hit         */
  SS_V_HEURISTIC = 4,     /* per-iteration choice by a frontier-size rule                      */
  SS_V_LEARNED = 5        /* per-iteration choice by the loaded selector MLP; frontiers the
                             cluster push takes go to it, as in SS_V_HEURISTIC                 */
} ss_policy;

/* Executed-variant id (ss_iter_stats.variant, not a policy) of the cluster
 * push: one thread-block cluster (16 CTAs of 1024 threads, else 8) runs
 * consecutive small levels in one launch with the frontier kept as vertex
 * lists in shared memory; push and the adaptive policies use it for frontiers
 * of at most 4096 vertices and 8192 edges per CTA (high-diameter graphs). */
#define SS_VARIANT_PUSH_LOCAL 4

/* Layout summary of a built handle. */
typedef struct {
  int32_t n, C, sigma, split_w;
  int32_t n_chunks;        /* ceil(n / C)                                             */
  int32_t n_items;         /* work items after SlimChunk splitting                    */
  int32_t n_split_chunks;  /* chunks with cl > split_w                                */
  int32_t max_degree;
  int64_t nnz;             /* directed nonzeros of the input CSR                      */
  int64_t slots;           /* |col| = sum_i C * cl_i = nnz + P                        */
  int64_t padding;         /* P                                                       */
  int64_t device_bytes;    /* bytes the handle holds on the device                    */
} ss_info;

/* One frontier expansion (iteration k discovers the vertices at distance k). */
typedef struct {
  int64_t frontier;        /* vertices discovered in this iteration                   */
  int64_t frontier_degree; /* sum of their degrees                                    */
  int64_t slots;           /* col slots read by the iteration kernels                 */
  int64_t active_chunks;   /* chunks processed (not skipped)                          */
  int32_t variant;         /* variant actually executed (0 FULL, 1 SLIMWORK, 2 PUSH, 3 FILTERED,
                              SS_VARIANT_PUSH_LOCAL)                                     */
  int32_t kernel_ns;       /* iteration kernel time in ns when profiling is on, else 0;
                              levels run inside one cluster-push launch are timed on
                              the device, the launch's entry counted in its first  */
} ss_iter_stats;

/* Summary of the last slimsell_bfs call on a handle. */
typedef struct {
  int32_t iterations;      /* SpMV passes, including the final one that adds nothing */
  int32_t semiring;
  int64_t reached;         /* vertices with a finite distance                         */
  int64_t reached_degree;  /* sum of their degrees = 2 * edges in the component       */
  int64_t slots;           /* total col slots read                                    */
  int64_t dp_slots;        /* col slots read by the DP pass (0 for sel-max)           */
  double iter_kernel_ms;   /* CUDA-event time of the iteration kernels (if profiling) */
  double total_ms;         /* CUDA-event time of the whole call (if profiling)        */
} ss_run_stats;

/*
 * Build the SlimSell layout from a CSR graph on the device (Sections II-D, III-B).
 *   d_row_ptr  int64[n + 1], d_col int32[nnz]: symmetric graph without
 *              self-loops or duplicate entries (not checked); neighbour lists
 *              sorted by ascending id.  Not retained after the call returns.
 *   C          chunk height, one of 8, 16, 32, 64.
 *   sigma      sorting scope: rows are sorted by descending degree (ties by
 *              ascending id) inside windows of sigma consecutive vertices;
 *              sigma <= 1 keeps the input order, sigma > 1 is first rounded up
 *              to a multiple of C (the paper takes sigma as a multiple of C,
 *              Section IV; ss_info.sigma reports the value used), sigma >= n
 *              sorts globally.
 *   split_w    SlimChunk width: chunks with more than split_w columns are split
 *              into ceil(cl / split_w) work items (Section III-D); 0 disables.
 * The call synchronises `stream` (it needs the layout size to allocate col).
 * Errors: SS_ERR_INVALID (n < 1, nnz < 0, bad C, sigma < 1, split_w < 0,
 * NULL pointers), SS_ERR_OOM, SS_ERR_CUDA (also when the device cannot place
 * the cluster push's thread-block cluster of 8 or 16 CTAs).  *out is NULL on
 * failure.
 */
ss_status slimsell_build(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                         int32_t C, int32_t sigma, int32_t split_w, void* stream,
                         slimsell_handle* out);

/*
 * Single-source BFS (Section III-A semiring BFS-SpMV; SlimWork Section III-C;
 * SlimChunk Section III-D; DP Section II-C for non-sel-max parents).
 *   root       vertex id in [0, n).
 *   semiring   ss_semiring.
 *   policy     ss_policy.
 *   d_dist     int32[n] or NULL; d_parent int32[n] or NULL (NULL skips the DP pass).
 * By default the iterations run as a device-side loop (a conditional CUDA graph
 * that stops when an iteration discovers nothing) and the call returns once the
 * work is queued on `stream`; slimsell_get_run_stats waits for it.  With
 * profiling on (or SS_OPT_DEVICE_LOOP = 0) the host drives the loop (see
 * SS_OPT_PROFILE_QUEUE for how often it reads the run's counter), and the call
 * returns after the BFS has finished.
 * The outputs, and the handle's state, belong to this call until `stream`
 * reaches its end: do not start another call on the same handle from a
 * different stream before that.  Calls on the same stream queue behind one
 * another without a host wait (the previous call's statistics are dropped);
 * slimsell_set_option and slimsell_selector_load wait for a queued run first.
 * Errors: SS_ERR_INVALID, SS_ERR_CUDA, SS_ERR_UNSUPPORTED.
 */
ss_status slimsell_bfs(slimsell_handle h, int32_t root, int32_t semiring, int32_t policy,
                       int32_t* d_dist, int32_t* d_parent, void* stream);

/*
 * The real-semiring frontier values of the handle's last slimsell_bfs call
 * (Section III-A: over (R, +, *, 0, 1) the frontier keeps x_k on the rows it
 * adds, and x_k sums the values of a row's neighbours in f_{k-1}; starting
 * from f_0 = e_root that is the number of shortest root-v paths).
 *   d_out  float[n] device, written in original vertex order: the value v
 *          entered the frontier with (1 for the root), 0 where the run did not
 *          reach.  fp32 sums in no fixed order, so exact while a count stays
 *          below 2^24.
 * Queued on `stream`; order it after the BFS call's work when that ran on
 * another stream.
 * Errors: SS_ERR_INVALID (NULL arguments, or the handle's last run was not a
 * real-semiring slimsell_bfs: any other run on the handle, a multi-source,
 * betweenness, format-comparison or batch call included, replaces the values),
 * SS_ERR_CUDA.
 */
ss_status slimsell_get_values(slimsell_handle h, float* d_out, void* stream);

/*
 * Multi-source BFS (an extension beyond the paper): the boolean semiring of
 * Section III-A run for k sources at once, frontiers bit-packed as
 * ceil(k / 64) uint64 words per vertex, rounded up to a power of two and to at
 * least 32 / C words.
 *   d_roots  int32[k] device, vertex ids in [0, n) (checked; duplicates allowed).
 *   k        1 .. 1024.
 *   policy   SS_V_FULL or SS_V_SLIMWORK (SlimWork skips chunks whose rows
 *            have every source visited; SlimChunk splitting applies).
 *   d_dist   int32[n][k] device or NULL: VERTEX-major, d_dist[v * k + s] =
 *            distance from roots[s] to v, -1 if unreached.
 * Synchronous (returns when done).  Run statistics: reached = reached
 * (vertex, source) pairs, reached_degree = their degree sum (= 2 x the sum
 * over sources of the edges in each source's component).
 * Errors: SS_ERR_INVALID, SS_ERR_OOM, SS_ERR_CUDA.
 */
ss_status slimsell_bfs_multi(slimsell_handle h, const int32_t* d_roots, int32_t k, int32_t policy,
                             int32_t* d_dist, void* stream);

/*
 * Multi-source BFS with parents (an extension beyond the paper): as
 * slimsell_bfs_multi, plus
 *   d_parent int32[n][k] device or NULL: VERTEX-major, d_parent[v * k + s] =
 *            the largest-id neighbour of v one level closer to roots[s]
 *            (roots[s] for the root itself, -1 if unreached): for every source,
 *            the canonical parent that slimsell_bfs returns for that root.
 * Parents are found by a pass after each level, in one of two directions
 * chosen per level from the previous level's counters: while the run grows and
 * the previous frontier's rows carry at most half of the edges, a push from
 * that frontier (each frontier row u offers itself to its neighbours that
 * gained a source u's frontier holds; atomicMax keeps the largest id);
 * otherwise a walk from the gaining rows (neighbours are stored in descending
 * original id, so for each source a vertex gained, the first neighbour that was
 * in that source's previous frontier is its parent).
 * slimsell_bfs_multi is this call with d_parent = NULL.
 * Errors: as slimsell_bfs_multi.
 */
ss_status slimsell_bfs_multi_parents(slimsell_handle h, const int32_t* d_roots, int32_t k,
                                     int32_t policy, int32_t* d_dist, int32_t* d_parent, void* stream);

/* Storage formats of slimsell_bfs_spmv. */
typedef enum {
  SS_FORMAT_SLIMSELL = 0, /* value inferred from col (-1 = padding, skipped), Section III-B */
  SS_FORMAT_SELL = 1      /* Sell-C-sigma: explicit val array, padding col 0 with the
                             semiring's zero as its value, Section II-D                    */
} ss_format;

/*
 * Storage-format comparison (Section IV, the speedup of SlimSell over
 * Sell-C-sigma): single-source BFS as the plain value-vector BFS-SpMV of
 * Section III-A (fp32 value vectors; every iteration streams every slot of the
 * handle's layout, SlimChunk items combined with atomics; no SlimWork, no
 * bitmaps), in either format.  The two formats differ only in where a slot's
 * matrix value comes from; results are identical.
 *   root      vertex id in [0, n)
 *   semiring  ss_semiring
 *   format    ss_format; SS_FORMAT_SELL builds the Sell-C-sigma arrays (col with
 *             padding 0, and one val array per value encoding: 1/inf for the
 *             tropical semiring, 1/0 for the others; 12 bytes per slot) from the
 *             handle's layout on first use and keeps them until
 *             slimsell_destroy.
 *   d_dist    int32[n] device, required: BFS distances (-1 unreached).
 *   kernel_ms host double* or NULL: if given, the summed device time of the
 *             iterations' kernels (CUDA events around each level's two launches).
 * Synchronous with respect to the host (the loop reads a counter per level).
 * Errors: SS_ERR_INVALID (NULL, root or semiring out of range, unknown format),
 *         SS_ERR_OOM, SS_ERR_CUDA.
 */
ss_status slimsell_bfs_spmv(slimsell_handle h, int32_t root, int32_t semiring, int32_t format,
                            int32_t* d_dist, double* kernel_ms, void* stream);

/*
 * Betweenness centrality on the SlimSell layout (an extension: the paper's
 * conclusion names BC as an algorithm SlimSell can accelerate), by Brandes'
 * dependency accumulation over a set of sources:
 *   bc[v] = sum over s in sources, t != s, v of sigma_st(v) / sigma_st
 * (sigma_st = number of shortest s-t paths, sigma_st(v) those through v).  On
 * an undirected graph with every vertex as a source each unordered pair counts
 * twice; halve for the one-direction convention.
 * Sources go in batches of 64.  Per batch, the bit-packed multi-source BFS
 * (slimsell_bfs_multi's SlimWork pull) finds the level words of every vertex
 * (bit s set at level L when the vertex is at distance L from source s); a
 * forward pass per level sums the path counts sigma of the neighbours one
 * level up, per source (the real-semiring BFS step with the counts kept), and a
 * backward pass per level from the deepest sums (1 + delta(w)) / sigma(w) over
 * the neighbours one level down.  fp64 throughout; a row's neighbours are cut
 * into units of 256 that combine with atomicAdd, so the result may differ from
 * a serial sum in the last bits.
 *   d_sources int32[k] device, k >= 1, each in [0, n) (copied to the host)
 *   d_bc      double[n] device, overwritten
 *   kernel_ms host double* or NULL: summed device time of the level kernels
 * Synchronous with respect to the host.  Scratch (1.5 KB per row, plus 8 bytes
 * per row and level) is allocated on first use and kept until
 * slimsell_destroy; the call also uses the multi-source scratch.
 * Errors: SS_ERR_INVALID (NULL, k < 1, a source out of range), SS_ERR_OOM,
 *         SS_ERR_CUDA.
 */
ss_status slimsell_bc(slimsell_handle h, const int32_t* d_sources, int32_t k, double* d_bc,
                      double* kernel_ms, void* stream);

/*
 * Batched BFS over many graphs (an extension beyond the paper): one executable
 * CUDA graph holding, per handle, the chain init -> root -> device-side
 * iteration loop -> output, so that one launch runs every BFS and the chains
 * overlap on the GPU.
 *   slimsell_batch_create: hs = g distinct handles on the current device,
 *     semiring / policy as for slimsell_bfs (applied to every graph).  The
 *     handles stay owned by the caller and must outlive the batch; while a batch
 *     run is in flight they must not be used by other calls.
 *   slimsell_batch_run: d_roots int32[g] device (root of graph i, checked);
 *     h_dist / h_parent: host arrays of g device pointers (int32[n_i] each, an
 *     entry or the whole array may be NULL).  Stream-ordered, returns once queued.
 *   slimsell_batch_get_stats: waits for the last run; out[g] (host) receives
 *     each graph's iterations, reached vertices and reached degree sum.
 * Errors: SS_ERR_INVALID, SS_ERR_OOM, SS_ERR_CUDA.
 */
ss_status slimsell_batch_create(const slimsell_handle* hs, int32_t g, int32_t semiring,
                                int32_t policy, slimsell_batch_handle* out);
ss_status slimsell_batch_run(slimsell_batch_handle b, const int32_t* d_roots,
                             int32_t* const* h_dist, int32_t* const* h_parent, void* stream);
ss_status slimsell_batch_get_stats(slimsell_batch_handle b, ss_run_stats* out);
void slimsell_batch_destroy(slimsell_batch_handle b);

/*
 * Layout autotuner (an extension; the paper tunes C, sigma and the SlimChunk
 * split by hand, Sections III-D and IV).  For every point of the grid
 * C x sigma x split_w it builds the layout (slimsell_build), runs one untimed
 * BFS from h_roots[0] (which builds the handle's device-side loop), then times
 * `repeats` passes over all roots with CUDA events on `stream`, and keeps the
 * point with the smallest mean time per BFS (no outputs written: dist and
 * parent NULL).
 *   d_row_ptr, d_col, n, nnz  the graph, as for slimsell_build (device).
 *   semiring, policy          as for slimsell_bfs.
 *   h_roots[nroots]           host, each in [0, n).
 *   h_C[nC]                   host, each 8, 16, 32 or 64.
 *   h_sigma[nsigma]           host, each >= 0; 0 means n (a global sort).
 *   h_split_w[nw]             host, each >= 0 (0 = no splitting).
 *   use_cache                 1: a graph whose signature matches a cached search
 *                             (slimsell_tune_match) with the same semiring,
 *                             policy and grid reuses it without timing.
 *   h_result                  host: the best point, the number of points timed
 *                             (0 when cached) and whether the cache answered.
 *   h_table[table_cap]        host or NULL: every grid point and its time, C
 *                             slowest-varying, then sigma, then split_w.
 * Every search is added to a process-wide cache (guarded by a mutex).  The call
 * synchronises `stream`.  Errors: SS_ERR_INVALID (NULL pointers, empty grids or
 * roots, a root, C, sigma or split_w out of range), SS_ERR_OOM, SS_ERR_CUDA.
 */
typedef struct {
  int32_t C;        /* chunk height                                            */
  int32_t sigma;    /* sorting scope as in the grid (0 = n)                     */
  int32_t split_w;  /* SlimChunk split width                                    */
  float ms;         /* mean time of one BFS in milliseconds                     */
} ss_tune_point;

typedef struct {
  ss_tune_point best;
  int32_t points;   /* grid points timed by this call (0 if the cache answered) */
  int32_t cached;   /* 1 if a cached search of a matching graph was reused      */
} ss_tune_result;

/* Cache key of a graph: n, nnz rounded to two significant digits, and
 * hist[b] = 50 x (vertices with floor(log2 degree) = b) / n, rounded to the
 * nearest integer, for b = 0 .. 23 (isolated vertices are not counted). */
typedef struct {
  int32_t n;
  int64_t nnz_rounded;
  int32_t hist[24];
} ss_tune_signature;

ss_status slimsell_autotune(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                            int32_t semiring, int32_t policy, const int32_t* h_roots, int32_t nroots,
                            const int32_t* h_C, int32_t nC, const int32_t* h_sigma, int32_t nsigma,
                            const int32_t* h_split_w, int32_t nw, int32_t repeats, int32_t use_cache,
                            ss_tune_result* h_result, ss_tune_point* h_table, int32_t table_cap,
                            void* stream);

/* Signature of a graph from its HOST row offsets h_row_ptr[n + 1] (host-only
 * computation, the same one slimsell_autotune makes on the device).
 * Errors: SS_ERR_INVALID (NULL pointers, n < 0). */
ss_status slimsell_tune_signature(const int64_t* h_row_ptr, int32_t n, ss_tune_signature* out);

/* 1 if two signatures would share a cached search: equal n and rounded nnz and
 * histograms within 3 units in L1 distance (so graphs of one family and size
 * share a search even where two seeds' shares fall on opposite sides of a
 * rounding edge); 0 otherwise (also for NULL arguments). */
int32_t slimsell_tune_match(const ss_tune_signature* a, const ss_tune_signature* b);

/* Layout summary. */
ss_status slimsell_get_info(slimsell_handle h, ss_info* out);

/*
 * Statistics of the last slimsell_bfs on this handle (waits for that call's
 * work to finish).  h_iters (host, may be NULL) receives up to cap
 * per-iteration records.
 */
ss_status slimsell_get_run_stats(slimsell_handle h, ss_run_stats* out, ss_iter_stats* h_iters,
                                 int32_t cap);

/* Options for slimsell_set_option. */
typedef enum {
  SS_OPT_DP_PASS = 1,     /* 1: tropical/real/boolean parents by a separate DP pass after the
                             iterations (Section II-C as written); 0 (default): the same parents
                             computed on the fly inside the iterations                        */
  SS_OPT_SMEM_BYTES = 2,  /* bytes of the frontier bitmap staged in shared memory per block,
                             0 .. 212992 (default 212992); results do not depend on it          */
  SS_OPT_DEVICE_LOOP = 3, /* 1 (default): iterate on the device in a conditional CUDA graph;
                             0: the host launches each iteration and reads its counter          */
  SS_OPT_SELECTOR_MARGIN = 4, /* learned policy, in thousandths of a log-time unit, 0 .. 100000
                             (default 0): the network's choice replaces the frontier-size rule's
                             only when it predicts a gain larger than this margin             */
  SS_OPT_PROFILE_QUEUE = 5, /* host-driven loop (profiling on, or SS_OPT_DEVICE_LOOP = 0) with a
                             fixed variant (FULL, SLIMWORK, PULL_FILTERED): 1 (default) queues
                             the iterations eight at a time, each launch between its own pair of
                             CUDA events, and reads the run's counter once per batch (launches
                             past the end of the run return at once); 0: one launch, one event
                             pair and one counter read per iteration, as for the adaptive
                             policies                                                         */
  SS_OPT_PUSH_BLOCKS = 6,  /* the push variant's view of the frontier f_{k-1} (block-sparse with
                             the layout's block size C, after the paper's closing author note):
                             1 (default) chunks whose block holds at least C/4 frontier rows are
                             pushed as blocks, reading whole columns of the chunk with coalesced
                             16-byte loads, the other frontier rows one row each (stride C);
                             2: every non-empty block as a block; 0: every frontier row alone.
                             Results do not depend on it                                      */
  SS_OPT_FORMAT = 8        /* storage format the pull streams (ss_format): SS_FORMAT_SLIMSELL
                             (default), or SS_FORMAT_SELL: the same pull over the Sell-C-sigma
                             arrays (column with padding 0 and an explicit value per slot: 1 for
                             an edge, the semiring's zero for padding; built on first use, 12
                             bytes per slot, kept until slimsell_destroy), for the format
                             comparison of Section IV at the production kernel's speed; with the
                             FULL and SLIMWORK policies only (others: SS_ERR_UNSUPPORTED).
                             Results do not depend on it                                      */
} ss_option;

/* Set a handle option (applies to later calls).  Errors: SS_ERR_INVALID. */
ss_status slimsell_set_option(slimsell_handle h, int32_t option, int64_t value);

/* Record CUDA events around the iteration kernels of later calls (0 = off). */
ss_status slimsell_set_profiling(slimsell_handle h, int32_t on);

/*
 * Copy the layout into caller-owned device buffers (any may be NULL):
 *   d_perm int32[n_chunks * C] (vertex at each row position, -1 for padding rows),
 *   d_cl int32[n_chunks], d_cs int64[n_chunks + 1], d_col int32[slots],
 *   d_items int32[4 * n_items] as (chunk, j0, j1, split index or -1).
 * Synchronises `stream`.
 */
ss_status slimsell_export_layout(slimsell_handle h, int32_t* d_perm, int32_t* d_cl, int64_t* d_cs,
                                 int32_t* d_col, int32_t* d_items, void* stream);

/*
 * Allocation-free sigma-window degree sort (the paper has no counterpart; this
 * is a library convenience).  Writes perm[r] = the vertex placed at row
 * position r by the same ordering slimsell_build uses (descending degree inside
 * windows of sigma consecutive vertices, ties by ascending id; sigma <= 1 keeps
 * the input order), for r in [0, n).  sigma is used as given: slimsell_build
 * first rounds its sigma up to a multiple of C, so pass that value to match it.
 *
 * For callers that must not allocate device memory: processes whose device
 * memory is fully reserved by another allocator, where cudaMalloc would fail,
 * and latency-bound loops that cannot accept the implicit synchronisation and
 * unpredictable cost of cudaMalloc/cudaFree.  This call performs no device
 * allocation and no freeing.  Its scratch is one fixed device array of about
 * 12.3 MiB that every GPU loading the library holds until the process exits.
 *   d_row_ptr  int64[n + 1] CSR offsets (degrees must be below n, i.e. no
 *              duplicate entries or self-loops; a larger degree is clamped to
 *              2^19 - 1 in the sort key), device memory, not modified.
 *   n          1 <= n <= 524288 (2^19); larger n returns SS_ERR_INVALID.
 *   sigma      >= 1.
 *   d_perm     int32[n] output, device memory owned by the caller.
 * Stream-ordered and asynchronous: it returns after queueing its kernels.  Each
 * call made outside stream capture looks up the array's device address on the
 * current device (so a context reset, which may move the array, is followed);
 * a call made while `stream` is being captured reuses the address of the last
 * lookup on that device, so make the first call on a device before any stream
 * capture (a first call during capture returns SS_ERR_INVALID).
 * All calls share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (different streams, or different host threads
 * without ordering) race and corrupt each other's results, so order them.
 * Errors: SS_ERR_INVALID (NULL pointers, n out of range, sigma < 1), SS_ERR_CUDA.
 */
ss_status slimsell_sigma_sort_noalloc(const int64_t* d_row_ptr, int32_t n, int32_t sigma,
                                      int32_t* d_perm, void* stream);

/*
 * Variant selector (an extension beyond the paper).  The learned policy feeds
 * 16 features of each iteration to a 16-64-64-4 ReLU MLP whose outputs predict
 * the log-time of the four variants (FULL, SLIMWORK, PUSH, PULL_FILTERED, in
 * ss_policy order) and runs the argmin.  Parameters are fp32, inputs first:
 * W1[16][64], b1[64], W2[64][64], b2[64], W3[64][4], b3[4] (5508 values),
 * h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3.
 */
#define SS_SELECTOR_FEATURES 16
#define SS_SELECTOR_HIDDEN 64
#define SS_SELECTOR_OUTPUTS 4
#define SS_SELECTOR_PARAMS 5508

/* Copy selector weights (host, len = SS_SELECTOR_PARAMS) to the handle's device
 * memory; h_weights = NULL unloads them (the learned policy then uses the
 * heuristic).  Errors: SS_ERR_INVALID, SS_ERR_OOM, SS_ERR_CUDA. */
ss_status slimsell_selector_load(slimsell_handle h, const float* h_weights, int64_t len);

/* Features of each iteration of the last slimsell_bfs (host, row-major
 * [min(cap, iterations + 1)][16]; row k = features seen before iteration k). */
ss_status slimsell_get_features(slimsell_handle h, float* h_out, int32_t cap);

/* Batched MLP forward: d_y[batch][4] = MLP(d_w; d_x[batch][16]) (device, fp32). */
ss_status slimsell_mlp_forward(const float* d_w, const float* d_x, int32_t batch, float* d_y,
                               void* stream);

/*
 * One training step on a minibatch (1 <= batch <= 128): forward, loss =
 * sum(mask * (y - t)^2) / max(sum(mask), 1) over d_t, d_mask [batch][4],
 * backward, and (lr > 0) an Adam update (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected with `step` >= 1) of d_w using the moment buffers d_adam_m,
 * d_adam_v [5508].  d_grad [5508] (may be NULL) receives the gradient and
 * d_loss [1] (may be NULL) the loss, both before the update.  All device.
 */
ss_status slimsell_mlp_train_step(float* d_w, float* d_adam_m, float* d_adam_v, int32_t step,
                                  const float* d_x, const float* d_t, const float* d_mask,
                                  int32_t batch, float lr, float* d_grad, float* d_loss,
                                  void* stream);

/* Free the handle and its device buffers (NULL is ignored). */
void slimsell_destroy(slimsell_handle h);

/* Message of the last error on the calling thread ("" if none). */
const char* slimsell_last_error(void);

/* Library version string. */
const char* slimsell_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SLIMSELL_H */
