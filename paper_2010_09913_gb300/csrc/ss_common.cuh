// Internal definitions shared by the CUDA translation units of libslimsell.
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "slimsell.h"

#define SS_INF 0x7fffffff          // tropical infinity / "unvisited" level
#define SS_PAD_LEVEL (-1)          // level of padding rows (never unvisited, never in a frontier)
#define SS_FULL_MASK 0xffffffffu
#define SS_PBEST_VISITED 0x7fffffff  // pbest of a visited vertex (above every original id)
#define SS_SMEM_MAX_BYTES 212992   // frontier-bitmap prefix staged per block (1,703,936 vertices)
#define SS_SMEM_LIMIT_BYTES 214016 // dynamic shared memory requested at most (prefix + guard)
// threads of a pull-iteration block (one block per SM); the item order assumes it
#ifndef SS_PULL_THREADS
#define SS_PULL_THREADS 1024
#endif
// cluster push: frontier entries and frontier edges per CTA, largest cluster, list capacity
#define SS_LOCAL_SLICE 4096
#define SS_LOCAL_EDGES_PER_CTA 8192
#define SS_LOCAL_CLUSTER_MAX 16
#define SS_LSTAT 8  // words per level in lstat
#define SS_LOCAL_LIST_CAP (SS_LOCAL_CLUSTER_MAX * SS_LOCAL_EDGES_PER_CTA)

namespace ss {

void set_error(const char* fmt, ...);
ss_status cuda_fail(cudaError_t e, const char* what);

#define SS_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return ::ss::cuda_fail(_e, #call);           \
  } while (0)

// Device control block for one BFS run (one per handle).
struct Ctl {
  int k;          // level being discovered by the current iteration
  int done;       // 1 once an iteration discovered nothing
  int error;      // device-side error flags
  int variant;    // variant executed by the current iteration
  unsigned long long new_count;   // vertices discovered by the current iteration
  unsigned long long new_deg;     // their degree sum
  unsigned long long slots;       // col slots read by the current iteration
  unsigned long long active;      // chunks processed by the current iteration
  unsigned long long reached;     // cumulative vertices reached
  unsigned long long reached_deg; // cumulative degree sum
  unsigned long long total_slots; // cumulative slots
  unsigned long long dp_slots;    // slots read by the DP pass
  unsigned int blocks_done;       // blocks of the current iteration kernel that finished
  int prev_variant;               // variant of the previous iteration (-1 before the first)
  unsigned long long prev_slots;  // slots read by the previous iteration
  unsigned long long prev_new;    // |f_{k-1}|: vertices discovered by the previous iteration
  unsigned long long prev_deg;    // their degree sum (frontier edges)
  unsigned long long prev2_new;   // |f_{k-2}|
  unsigned long long prev_active; // chunks processed by the previous iteration
  unsigned int new_maxdeg;        // largest degree discovered by the current iteration
  unsigned int prev_maxdeg;       // ... by the previous iteration
  unsigned long long units;       // push work units queued by the current iteration
  unsigned long long variant_count[5];  // iterations run with each variant
  int list_level;                 // level whose vertex list is in qlist[level & 1] (-1: none)
  int list_prev_ok;               // qlist also holds the list of list_level - 1
  unsigned long long qlen[2];     // vertex-list lengths, by level parity
  unsigned long long qprep;       // length of a list just built from the bitmap
  unsigned long long loop_guard;  // decide-kernel executions in this run (device loop bound)
  unsigned long long bunits;      // push block units queued by the current iteration
  unsigned long long new_rowdeg;  // multi-source: degree sum of the rows that gained a source
                                  // in the current iteration (each row counted once)
  unsigned long long prev_rowdeg; // ... in the previous iteration
};

// Flat view of the handle's device buffers handed to kernels by value.
struct Dev {
  int n, C, n_c, n_pad, n_items, n_split;
  const int* perm;      // [n_pad] vertex at row position (-1 for padding rows)
  const int* invperm;   // [n] row position of vertex
  const int* rdeg;      // [n_pad] degree of the vertex at each row (0 for padding)
  const int* cl;        // [n_c] chunk lengths
  const long long* cs;  // [n_c + 1] chunk starts (in slots)
  const int* col;       // [slots] SlimSell column array (-1 = padding)
  int format;           // SS_FORMAT_SLIMSELL, or SS_FORMAT_SELL: the pull streams scol and sval
  const int* scol;      // [slots] Sell-C-sigma column array (padding 0), when format is Sell
  const float* sval;    // [slots] Sell-C-sigma values of the run's semiring (1 edge, its zero padding)
  const int4* items;    // [n_items] (chunk, j0, j1, split index or -1)
  const int* split_n;   // [n_split] items per split chunk
  int* lvl;             // [n_pad] level (SS_INF = unvisited); the tropical f vector
  unsigned char* act;   // [n_c] SlimWork state: 1 active, 3/2 inactive with zero writes pending, 0 inactive
  unsigned* fb[2];      // frontier bitmaps (n_pad bits each), indexed by level parity
  long long fb_words;   // allocated words per bitmap
  int smem_words;       // bitmap words staged in shared memory per block (multiple of 4)
  float* fr;            // [n_pad] real-semiring value of a row when it entered the frontier
  int* par;             // [n_pad] parent original id + 1 (0 = none)
  float* xacc;          // [n_split * C] SlimChunk partial sums (real semiring)
  int* xpar;            // [n_split * C] SlimChunk partial parents (original id, -1 = none)
  unsigned* arrive;     // [n_split] SlimChunk arrival counters
  int2* units;          // [units_cap] push work units (row, first neighbour index)
  long long units_cap;
  int2* bunits;         // [bunits_cap] push block units (chunk, first column) of the
                        // block-sparse frontier: chunks whose frontier block is dense
  long long bunits_cap;
  int push_blocks;      // 0: vertex units only, 1: block units for dense blocks, 2: for every block
  int* pbest;           // [n_pad] push: largest frontier-neighbour original id (-1 = none yet,
                        // SS_PBEST_VISITED once the vertex has a level)
  float* psum;          // [n_pad] push: real-semiring sum of frontier-neighbour values
  unsigned* touched;    // [fb_words] push: rows reached by the current push
  int* qlist[2];        // [n_pad] vertex lists of a level (cluster push), by parity
  int* qdeg[2];         // [SS_LOCAL_LIST_CAP] cluster push: degree of each listed vertex
  long long* qbase[2];  // [SS_LOCAL_LIST_CAP] ... start of its column-major row (cs + row % C)
  int* qorig[2];        // [SS_LOCAL_LIST_CAP] ... its original id
  int* qovf;            // [SS_LOCAL_LIST_CAP] cluster push: new vertices past a CTA's list
  unsigned long long* qovf_n;  // [2] their counts, by level parity
  int local_cluster;    // CTAs in the cluster push's cluster
  long long local_max_nf, local_max_e;  // largest frontier (vertices, edges) it takes
  const float* mlp;     // selector weights (16-64-64-4 MLP), or NULL
  float sel_margin;     // learned policy: predicted log-time gain needed to leave the heuristic
  float* feats;         // [iter_cap][16] selector features of each iteration of the last run
  long long nnz, total_slots;
  unsigned long long reach_cap;  // most reached units a correct run can count (n, or n * k)
  Ctl* ctl;
  ss_iter_stats* iters; // [iter_cap]
  unsigned long long* lstat;  // [iter_cap][LSTAT] cluster push: per-level totals for the features
  int iter_cap;
};

}  // namespace ss

namespace ss {
// True the first time a call site asks on the current device (host code sets
// per-device kernel attributes once per device; the bit is per call site).
inline bool first_on_device(std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  return !(done.fetch_or(bit) & bit);
}
}  // namespace ss

struct slimsell_graph {
  int device = 0;
  int n = 0, C = 0, sigma = 0, split_w = 0, n_c = 0, n_pad = 0;
  long long nnz = 0, slots = 0;
  int n_items = 0, n_split = 0, max_degree = 0;
  int num_sms = 0;
  // layout
  int* perm = nullptr;
  int* invperm = nullptr;
  int* rdeg = nullptr;
  int* cl = nullptr;
  long long* cs = nullptr;
  int* col = nullptr;
  int4* items = nullptr;
  int* split_n = nullptr;
  // BFS state
  int* lvl = nullptr;
  unsigned char* act = nullptr;
  unsigned* fb[2] = {nullptr, nullptr};
  long long fb_words = 0;
  float* fr = nullptr;
  int* par = nullptr;
  float* xacc = nullptr;
  int* xpar = nullptr;
  unsigned* arrive = nullptr;
  int2* units = nullptr;
  long long units_cap = 0;
  int2* bunits = nullptr;
  long long bunits_cap = 0;
  int push_blocks = 1;                 // see SS_OPT_PUSH_BLOCKS
  int* pbest = nullptr;
  float* psum = nullptr;
  unsigned* touched = nullptr;
  int* qlist[2] = {nullptr, nullptr};
  int* qdeg[2] = {nullptr, nullptr};
  long long* qbase[2] = {nullptr, nullptr};
  int* qorig[2] = {nullptr, nullptr};
  int* qovf = nullptr;
  unsigned long long* qovf_n = nullptr;
  int local_cluster = 0;
  float* mlp = nullptr;       // selector weights on the device (NULL until loaded)
  float sel_margin = 0.0f;    // see SS_OPT_SELECTOR_MARGIN
  float* feats = nullptr;
  // multi-source scratch ([n_pad][W] words), grown on demand
  int multi_w = 0;
  unsigned long long* mF[2] = {nullptr, nullptr};
  unsigned long long* mV = nullptr;
  unsigned long long* mxacc = nullptr;
  int* mroots = nullptr;
  int smem_bytes = SS_SMEM_MAX_BYTES;  // bitmap prefix staged in shared memory
  int dp_pass = 0;                     // 1: parents by a separate DP pass after the iterations
  ss::Ctl* ctl = nullptr;
  ss::Ctl* h_ctl = nullptr;  // pinned host copy
  ss_iter_stats* iters = nullptr;
  unsigned long long* lstat = nullptr;
  int iter_cap = 0;
  long long device_bytes = 0;
  // last run
  ss_run_stats last{};
  int profiling = 0;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr, ev_d = nullptr;
  cudaEvent_t ev_done = nullptr;       // end of the last call's work on its stream
  int pending = 0;                     // last-run statistics not yet read back
  int values_semiring = -1;            // semiring of the slimsell_bfs call whose values fr holds (-1: none)
  int device_loop = 1;                 // iterate with a conditional CUDA graph
  int profile_queue = 1;               // host-driven fixed variants: queue iterations in batches
  int format = SS_FORMAT_SLIMSELL;     // storage format the pull streams (SS_OPT_FORMAT)
  const int* sell_col = nullptr;       // Sell-C-sigma arrays, built on first use (ss_sell.cu)
  const float* sell_vtrop = nullptr;
  const float* sell_vmul = nullptr;
  cudaGraphExec_t loop_exec[4][6] = {};  // [semiring][policy] device-side iteration loops
  int loop_smem_words[4][6] = {};
  std::vector<int> iter_ns;            // per-iteration kernel time of the last profiled call
  std::vector<cudaEvent_t> evq;        // event pairs of a queued host-driven batch of iterations

  ss::Dev dev() const;
};

namespace ss {
ss_status dmalloc(slimsell_graph* h, void** p, size_t bytes);
}  // namespace ss
