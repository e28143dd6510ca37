// Device-side pieces shared by the iteration kernels (pull, push) and the driver.
#pragma once

#include "ss_common.cuh"

namespace ss {

// Variant ids executed by one iteration (0..3 are the ss_policy values; 4 is
// the cluster push that runs several small levels in one launch).
enum { VAR_FULL = SS_V_FULL, VAR_SLIMWORK = SS_V_SLIMWORK, VAR_PUSH = SS_V_PUSH,
       VAR_FILTERED = SS_V_PULL_FILTERED, VAR_PUSH_LOCAL = 4, N_VARIANTS = 5 };

// Frontiers the cluster push takes: at most d.local_max_nf vertices and
// d.local_max_e edges (SS_LOCAL_SLICE and SS_LOCAL_EDGES_PER_CTA per CTA).
__device__ __forceinline__ bool local_fits(const Dev& d, unsigned long long nf, unsigned long long mf) {
  return nf <= (unsigned long long)d.local_max_nf && mf <= (unsigned long long)d.local_max_e;
}

// Neighbours per push work unit: a frontier row of degree D becomes ceil(D / PUSH_UNIT)
// units (row, first neighbour index), so hub rows spread over many warps.
constexpr int PUSH_UNIT = 256;
// Slots per push block unit (PUSH_BLOCK_SLOTS / C columns of one chunk).
constexpr int PUSH_BLOCK_SLOTS = 2048;

// Emit the work units of frontier vertex u (deg > 0), warp-aggregated.  All
// lanes of the warp call; lanes with u < 0 emit nothing.
__device__ __forceinline__ void emit_units(const Dev& d, int u, int lane) {
  const int deg = (u >= 0) ? d.rdeg[u] : 0;
  const unsigned nu = (unsigned)((deg + PUSH_UNIT - 1) / PUSH_UNIT);
  unsigned incl = nu;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(SS_FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned total = __shfl_sync(SS_FULL_MASK, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(&d.ctl->units, (unsigned long long)total);
  base = __shfl_sync(SS_FULL_MASK, base, 31);
  const unsigned long long first = base + incl - nu;
  if (first + nu > (unsigned long long)d.units_cap) {  // cannot happen after the decide check
    if (nu) atomicOr(&d.ctl->error, 2);
    return;
  }
  for (unsigned q = 0; q < nu; ++q) d.units[first + q] = make_int2(u, (int)(q * PUSH_UNIT));
}

struct IterLaunch {
  int variant;
  cudaGraphConditionalHandle cond;  // WHILE-loop condition of the device-side loop
  int use_cond;
};

// Record the finished level k (nc vertices discovered, nd their degree sum, sl
// slots read, ac chunks processed, md largest new degree) and advance k.
// Returns true when the run must stop: an iteration that discovered nothing,
// or (an error) k past n + 1 or more units reached than a correct run can count.
// record = false keeps d.iters untouched (copies of the control block).
__device__ __forceinline__ bool advance_level(const Dev& d, Ctl* c, int k, unsigned long long nc,
                                              unsigned long long nd, unsigned long long sl,
                                              unsigned long long ac, unsigned md, int variant,
                                              bool record = true) {
  if (record && k < d.iter_cap) {
    ss_iter_stats s;
    s.frontier = (long long)nc;
    s.frontier_degree = (long long)nd;
    s.slots = (long long)sl;
    s.active_chunks = (long long)ac;
    s.variant = variant;
    s.kernel_ns = 0;
    d.iters[k] = s;
  }
  c->reached += nc;
  c->reached_deg += nd;
  c->total_slots += sl;
  c->prev_slots = sl;
  c->prev2_new = c->prev_new;
  c->prev_new = nc;
  c->prev_deg = nd;
  c->prev_active = ac;
  c->prev_maxdeg = md;
  c->prev_variant = variant;
  c->variant = variant;
  if (variant >= 0 && variant < N_VARIANTS) c->variant_count[variant] += 1;
  c->units = 0;
  c->bunits = 0;
  c->qprep = 0;
  bool stop = (nc == 0);
  if (k >= d.n + 1 || c->reached > d.reach_cap) {
    c->error |= 1;
    stop = true;
  }
  if (stop) c->done = 1;
  c->k = k + 1;
  return stop;
}

// End of an iteration, run by the last block of its final kernel: record the
// level, reset the per-iteration counters and (device-side loop) set the loop
// condition.  The vertex list of the single-block push is no longer current.
__device__ __forceinline__ void iteration_tail(const Dev& d, int variant,
                                               cudaGraphConditionalHandle cond, int use_cond) {
  Ctl* c = d.ctl;
  const int k = c->k;
  const unsigned long long nc = atomicAdd(&c->new_count, 0ull);
  const unsigned long long nd = atomicAdd(&c->new_deg, 0ull);
  const unsigned long long sl = atomicAdd(&c->slots, 0ull);
  const unsigned long long ac = atomicAdd(&c->active, 0ull);
  const unsigned md = atomicMax(&c->new_maxdeg, 0u);
  const bool stop = advance_level(d, c, k, nc, nd, sl, ac, md, variant);
  c->prev_rowdeg = c->new_rowdeg;
  c->new_rowdeg = 0;
  c->list_level = -1;
  c->new_count = 0;
  c->new_deg = 0;
  c->slots = 0;
  c->active = 0;
  c->new_maxdeg = 0;
  c->blocks_done = 0;
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// Block-wide reduction of a kernel's counters (new vertices, their degree sum,
// slots read, chunks processed, largest new degree), one atomic per block and
// counter; the last block to finish runs the iteration tail.  All threads call.
template <int THREADS>
__device__ __forceinline__ void finish_iteration_block(const Dev& d, unsigned long long nw,
                                                       unsigned long long deg, unsigned long long slots,
                                                       unsigned long long act, unsigned maxdeg,
                                                       const IterLaunch& il) {
  __shared__ unsigned long long red[4][THREADS / 32];
  __shared__ unsigned redmax[THREADS / 32];
  const int lane = threadIdx.x & 31;
  unsigned long long v[4] = {nw, deg, slots, act};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(SS_FULL_MASK, v[i], off);
    if (lane == 0) red[i][threadIdx.x >> 5] = v[i];
  }
  maxdeg = __reduce_max_sync(SS_FULL_MASK, maxdeg);
  if (lane == 0) redmax[threadIdx.x >> 5] = maxdeg;
  __syncthreads();
  if (threadIdx.x < 5) {
    if (threadIdx.x < 4) {
      unsigned long long s = 0;
#pragma unroll
      for (int w = 0; w < THREADS / 32; ++w) s += red[threadIdx.x][w];
      if (s) {
        unsigned long long* dst = threadIdx.x == 0 ? &d.ctl->new_count
                                : threadIdx.x == 1 ? &d.ctl->new_deg
                                : threadIdx.x == 2 ? &d.ctl->slots
                                                   : &d.ctl->active;
        atomicAdd(dst, s);
      }
    } else {
      unsigned m = 0;
#pragma unroll
      for (int w = 0; w < THREADS / 32; ++w) m = max(m, redmax[w]);
      if (m) atomicMax(&d.ctl->new_maxdeg, m);
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&d.ctl->blocks_done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      iteration_tail(d, il.variant, il.cond, il.use_cond);
    }
  }
}

// Selector features of iteration c->k (statistics of the frontier f_{k-1} and
// the state), logged before every iteration; the 16-64-64-4 MLP reads them.
// fp32 throughout: double-precision transcendentals are very slow on this GPU.
__device__ __forceinline__ float feat_lg(float x) { return __log2f(1.0f + fmaxf(x, 0.0f)); }

// Every feature describes the BFS state, never the schedule that reached it
// (a feature of the previous pass's work, for instance, reads 0 after levels
// the cluster push ran and would mislead the network there).
__device__ __forceinline__ void features_of(const Dev& d, int k, unsigned long long prev_new,
                                            unsigned long long prev_deg, unsigned long long reached,
                                            unsigned long long reached_deg, unsigned prev_maxdeg,
                                            unsigned long long prev2_new, float* f) {
  const float n = (float)d.n, nnz = (float)(d.nnz > 0 ? d.nnz : 1);
  const float nf = (float)prev_new, mf = (float)prev_deg;
  const float unv = (float)((unsigned long long)d.n - reached);
  const float mu = (float)((unsigned long long)d.nnz - reached_deg);  // unexplored edge endpoints
  f[0] = feat_lg(nf) / 32.f;
  f[1] = nf / n;
  f[2] = feat_lg(mf) / 32.f;
  f[3] = mf / nnz;
  f[4] = feat_lg(unv) / 32.f;
  f[5] = unv / n;
  f[6] = mu / nnz;                      // share of the edge endpoints still unexplored
  f[7] = mf / fmaxf(mf + mu, 1.f);      // frontier edges against the unexplored ones
  f[8] = (float)k / 32.f;
  f[9] = (float)k / (float)(k + 1);
  f[10] = feat_lg(mf / fmaxf(nf, 1.f)) / 32.f;
  f[11] = feat_lg((float)prev_maxdeg) / 32.f;
  f[12] = feat_lg(mu) / 32.f;
  f[13] = feat_lg(n) / 32.f;
  f[14] = feat_lg(nnz) / 32.f;
  f[15] = feat_lg(nf / fmaxf((float)prev2_new, 1.f)) / 32.f;
}

__device__ __forceinline__ void compute_features(const Dev& d, const Ctl* c, float* f) {
  features_of(d, c->k, c->prev_new, c->prev_deg, c->reached, c->reached_deg, c->prev_maxdeg, c->prev2_new, f);
}

// Write the features of iteration k into d.feats (one thread).
__device__ __forceinline__ void store_features(const Dev& d, int k, const float* f) {
  if (k >= d.iter_cap) return;
#pragma unroll
  for (int i = 0; i < SS_SELECTOR_FEATURES; ++i) d.feats[(size_t)k * SS_SELECTOR_FEATURES + i] = f[i];
}

// Root state and control block of a new single-source run (one thread).
__device__ __forceinline__ void init_root_state(const Dev& d, int root) {
  const int r = d.invperm[root];
  d.lvl[r] = 0;
  d.pbest[r] = SS_PBEST_VISITED;
  d.fb[0][r >> 5] |= 1u << (r & 31);
  d.fr[r] = 1.0f;
  d.par[r] = root + 1;
  Ctl* c = d.ctl;
  c->k = 1; c->done = 0; c->error = 0; c->variant = -1;
  c->new_count = 0; c->new_deg = 0; c->slots = 0; c->active = 0;
  c->reached = 1; c->reached_deg = (unsigned long long)d.rdeg[r];
  c->total_slots = 0; c->dp_slots = 0; c->blocks_done = 0;
  c->prev_variant = -1; c->prev_slots = 0; c->prev_new = 1; c->prev_deg = (unsigned long long)d.rdeg[r];
  c->prev2_new = 0; c->prev_active = 0; c->new_maxdeg = 0; c->prev_maxdeg = (unsigned)d.rdeg[r];
  c->units = 0;
  c->bunits = 0;
  for (int v = 0; v < N_VARIANTS; ++v) c->variant_count[v] = 0;
  c->loop_guard = 0;
  c->list_level = -1; c->list_prev_ok = 0; c->qlen[0] = c->qlen[1] = 0; c->qprep = 0;
  ss_iter_stats s;
  s.frontier = 1; s.frontier_degree = d.rdeg[r]; s.slots = 0; s.active_chunks = 0;
  s.variant = -1; s.kernel_ns = 0;
  d.iters[0] = s;
}

// Distances and parents in original vertex ids (grid-stride over vertices).
__device__ __forceinline__ void write_outputs(const Dev& d, int* dist, int* parent) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < d.n;
       v += (long long)gridDim.x * blockDim.x) {
    const int r = d.invperm[v];
    const int L = d.lvl[r];
    if (dist) dist[v] = (L == SS_INF) ? -1 : L;
    if (parent) parent[v] = (L == SS_INF) ? -1 : d.par[r] - 1;
  }
}

// View of a multi-source BFS run (ss_multi.cu): F[level & 1][row * W + w] holds bit s of
// word w when row entered source 64 w + s's frontier at that level; V the visited bits.
struct MultiDev {
  Dev d;
  unsigned long long* F[2];
  unsigned long long* V;
  unsigned long long* xacc;  // [n_split][C][W]
  int* dist;                 // [n][k] in original vertex order, or NULL
  int vec_dist;              // k % 4 == 0 and dist 16-byte aligned: 16-byte group writes
  const int* roots;          // [k]
  int k;
};

ss_status multi_start(slimsell_graph* h, const int32_t* d_roots, int k, cudaStream_t st, MultiDev* m,
                      int* W_out);
ss_status multi_level(slimsell_graph* h, const MultiDev& m, int W, cudaStream_t st, bool* done,
                      cudaEvent_t before = nullptr, cudaEvent_t after = nullptr);

// The handle's Sell-C-sigma arrays, built on first use (ss_sell.cu).
ss_status sell_arrays(slimsell_graph* h, cudaStream_t st);

__global__ void k_init(Dev d);

// Grid sizes that follow the graph size (ss_bfs.cu).
int pull_grid(const slimsell_graph* h);
int vertex_grid(const slimsell_graph* h, int threads);

// Add a device-side iteration loop (conditional WHILE node) to graph g (ss_bfs.cu).
ss_status add_loop_node(slimsell_graph* h, const Dev& d, int sr, int policy, cudaGraph_t g,
                        const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* out);

// Launchers implemented in the other translation units.
ss_status launch_push(const slimsell_graph* h, const Dev& d, int sr, const IterLaunch& il,
                      cudaStream_t st);
ss_status launch_push_local(const slimsell_graph* h, const Dev& d, int sr, const IterLaunch& il,
                            int max_levels, cudaStream_t st);
int push_local_cluster_size();
void drop_loop_graphs(slimsell_graph* h);  // forget captured loops (they hold handle state)  // CTAs per cluster of the cluster push on the current device (0: none)
ss_status launch_decide(const slimsell_graph* h, const Dev& d, int policy,
                        cudaGraphConditionalHandle sw, int use_sw, cudaStream_t st);
ss_status add_decide_node(const slimsell_graph* h, const Dev& d, int policy,
                          cudaGraphConditionalHandle sw, cudaGraphConditionalHandle cw,
                          cudaGraph_t g, cudaGraphNode_t* out);

}  // namespace ss
