// Single-source BFS-SpMV on SlimSell (Section III-A semirings, Section III-B
// SlimSell, Section III-C SlimWork, Section III-D SlimChunk, Section II-C DP).
//
// Vertex state lives in the relabelled row space of the layout:
//   lvl[r]        level of row r (SS_INF while unvisited).  For the tropical
//                 semiring lvl *is* f_{k-1}: iteration k reads neighbours with
//                 lvl <= k-1 and writes k into newly reached rows, which readers
//                 of the same iteration treat as infinity, so a single buffer
//                 reproduces x_k = A' (x) f_{k-1} exactly.
//   fb/fr/fx[k&1] the frontier f_k of the boolean (1 bit), real (fp32 value) and
//                 sel-max (original id + 1) semirings, double-buffered by parity.
//   par           sel-max parent vector p_k (original id + 1; 0 = none).
//
// One warp processes one work item (chunk i, columns [j0, j1)).  Each lane loads
// 16-byte quads of col: a quad is 4 consecutive rows of one column, so lane l
// always meets the same 4 rows 4*(l mod C/4) .. +3 and keeps 4 accumulators;
// the lanes sharing rows are combined with xor-shuffles at the end of the item.
// Split chunks (SlimChunk) combine partial rows with atomics in xacc; the last
// item of the chunk to arrive runs the post-processing.
#include "ss_common.cuh"

namespace ss {

// ---------------------------------------------------------------------------
// semiring traits: accumulator, identity, combine, neighbour value, atomic
// ---------------------------------------------------------------------------
template <int SR> struct Semi;

template <> struct Semi<SS_TROPICAL> {  // (min, +): value of u is f^u + 1 if f^u <= k-1
  using T = int;
  static __device__ __forceinline__ T id() { return SS_INF; }
  static __device__ __forceinline__ T op(T a, T b) { return min(a, b); }
  static __device__ __forceinline__ T load(const Dev& d, int km1, int c) {
    int t = d.lvl[c];
    return ((unsigned)t <= (unsigned)km1) ? t + 1 : SS_INF;
  }
  static __device__ __forceinline__ bool found(T a) { return a != SS_INF; }
  static __device__ __forceinline__ void atomic(unsigned* p, T v) { atomicMin((int*)p, v); }
  static __device__ __forceinline__ unsigned bits(T v) { return (unsigned)v; }
  static __device__ __forceinline__ T from_bits(unsigned b) { return (T)b; }
};

template <> struct Semi<SS_REAL> {  // (+, *): value of u is f^u (0 outside the frontier)
  using T = float;
  static __device__ __forceinline__ T id() { return 0.0f; }
  static __device__ __forceinline__ T op(T a, T b) { return a + b; }
  static __device__ __forceinline__ T load(const Dev& d, int km1, int c) {
    return __ldg(d.fr[km1 & 1] + c);
  }
  static __device__ __forceinline__ bool found(T a) { return a != 0.0f; }
  static __device__ __forceinline__ void atomic(unsigned* p, T v) { atomicAdd((float*)p, v); }
  static __device__ __forceinline__ unsigned bits(T v) { return __float_as_uint(v); }
  static __device__ __forceinline__ T from_bits(unsigned b) { return __uint_as_float(b); }
};

template <> struct Semi<SS_BOOLEAN> {  // (|, &): value of u is its frontier bit
  using T = unsigned;
  static __device__ __forceinline__ T id() { return 0u; }
  static __device__ __forceinline__ T op(T a, T b) { return a | b; }
  static __device__ __forceinline__ T load(const Dev& d, int km1, int c) {
    return (__ldg(d.fb[km1 & 1] + (c >> 5)) >> (c & 31)) & 1u;
  }
  static __device__ __forceinline__ bool found(T a) { return a != 0u; }
  static __device__ __forceinline__ void atomic(unsigned* p, T v) { atomicOr(p, v); }
  static __device__ __forceinline__ unsigned bits(T v) { return v; }
  static __device__ __forceinline__ T from_bits(unsigned b) { return b; }
};

template <> struct Semi<SS_SELMAX> {  // (max, *): value of u is its id + 1 if in the frontier
  using T = int;
  static __device__ __forceinline__ T id() { return 0; }
  static __device__ __forceinline__ T op(T a, T b) { return max(a, b); }
  static __device__ __forceinline__ T load(const Dev& d, int km1, int c) {
    return __ldg(d.fx[km1 & 1] + c);
  }
  static __device__ __forceinline__ bool found(T a) { return a != 0; }
  static __device__ __forceinline__ void atomic(unsigned* p, T v) { atomicMax((int*)p, v); }
  static __device__ __forceinline__ unsigned bits(T v) { return (unsigned)v; }
  static __device__ __forceinline__ T from_bits(unsigned b) { return (T)b; }
};

__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }

// Store the C frontier bits of one chunk (bit l = row l) into the bitmap.
template <int C>
__device__ __forceinline__ void store_bits(unsigned* fb, int chunk, unsigned lo, unsigned hi) {
  if (C == 8) reinterpret_cast<unsigned char*>(fb)[chunk] = (unsigned char)lo;
  else if (C == 16) reinterpret_cast<unsigned short*>(fb)[chunk] = (unsigned short)lo;
  else if (C == 32) fb[chunk] = lo;
  else reinterpret_cast<uint2*>(fb)[chunk] = make_uint2(lo, hi);
}

// Combine the 4-bit masks of lanes 0 .. C/4-1 into the chunk's bit words (all lanes call).
template <int C>
__device__ __forceinline__ void gather_bits(unsigned nib, int lane, unsigned* lo, unsigned* hi) {
  constexpr int Q = C / 4;
  if (C <= 32) {
    *lo = __reduce_or_sync(SS_FULL_MASK, lane < Q ? nib << (4 * lane) : 0u);
    *hi = 0u;
  } else {
    *lo = __reduce_or_sync(SS_FULL_MASK, lane < 8 ? nib << (4 * lane) : 0u);
    *hi = __reduce_or_sync(SS_FULL_MASK, (lane >= 8 && lane < 16) ? nib << (4 * (lane - 8)) : 0u);
  }
}

struct Counters {
  unsigned long long nw = 0, deg = 0, slots = 0, act = 0;
};

// Post-process one chunk (Section III-A listing of the frontier update): derive
// f_k, d and p from x_k = acc for rows R0 .. R0+3 owned by this lane (lane < Q),
// write the next SlimWork state, count new vertices.  All lanes of the warp call.
template <int SR, int C>
__device__ __forceinline__ void post_chunk(const Dev& d, int k, int chunk, int lane,
                                           const typename Semi<SR>::T acc[4], Counters& cnt) {
  using S = Semi<SR>;
  constexpr int Q = C / 4;
  const bool own = lane < Q;
  const int R0 = chunk * C + 4 * lane;
  unsigned nib = 0, left = 0;
  if (own) {
    int4 lv = *reinterpret_cast<const int4*>(d.lvl + R0);
    int L[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      bool unvisited = (L[r] == SS_INF);
      bool nw = unvisited && S::found(acc[r]);
      if (nw) nib |= 1u << r;
      else if (unvisited) left = 1;
    }
    if (nib) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (nib >> r & 1u) L[r] = k;
      *reinterpret_cast<int4*>(d.lvl + R0) = make_int4(L[0], L[1], L[2], L[3]);
      int4 dg = *reinterpret_cast<const int4*>(d.rdeg + R0);
      int D[4] = {dg.x, dg.y, dg.z, dg.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (nib >> r & 1u) cnt.deg += (unsigned long long)D[r];
      cnt.nw += __popc(nib);
    }
    if (SR == SS_REAL) {
      float4 f;
      f.x = (nib & 1u) ? acc[0] : 0.0f;
      f.y = (nib & 2u) ? acc[1] : 0.0f;
      f.z = (nib & 4u) ? acc[2] : 0.0f;
      f.w = (nib & 8u) ? acc[3] : 0.0f;
      *reinterpret_cast<float4*>(d.fr[k & 1] + R0) = f;
    } else if (SR == SS_SELMAX) {
      int4 x = make_int4(0, 0, 0, 0);
      if (nib) {
        int4 pm = *reinterpret_cast<const int4*>(d.perm + R0);
        int4 pv = *reinterpret_cast<const int4*>(d.par + R0);
        // p_k = p_{k-1} + not(p_{k-1}) (.) x_k ; frontier carries the vertex ids
        if (nib & 1u) { x.x = pm.x + 1; pv.x = (int)acc[0]; }
        if (nib & 2u) { x.y = pm.y + 1; pv.y = (int)acc[1]; }
        if (nib & 4u) { x.z = pm.z + 1; pv.z = (int)acc[2]; }
        if (nib & 8u) { x.w = pm.w + 1; pv.w = (int)acc[3]; }
        *reinterpret_cast<int4*>(d.par + R0) = pv;
      }
      *reinterpret_cast<int4*>(d.fx[k & 1] + R0) = x;
    }
  }
  if (SR == SS_BOOLEAN) {
    unsigned lo, hi;
    gather_bits<C>(nib, lane, &lo, &hi);
    if (lane == 0) store_bits<C>(d.fb[k & 1], chunk, lo, hi);
  }
  unsigned any_left = __any_sync(SS_FULL_MASK, left);
  if (lane == 0) d.act[chunk] = any_left ? 1 : (SR == SS_TROPICAL ? 0 : 3);
}

// A skipped chunk (SlimWork) carries its values over: its rows are all final, so
// f_k is zero there; clear the parity buffer for the two iterations after the
// chunk's last discovery, then leave it alone.
template <int SR, int C>
__device__ __forceinline__ void carry_chunk(const Dev& d, int k, int chunk, int lane, unsigned char a) {
  if (SR == SS_TROPICAL || a < 2) return;
  constexpr int Q = C / 4;
  const int R0 = chunk * C + 4 * lane;
  if (SR == SS_BOOLEAN) {
    if (lane == 0) store_bits<C>(d.fb[k & 1], chunk, 0u, 0u);
  } else if (SR == SS_REAL) {
    if (lane < Q) *reinterpret_cast<float4*>(d.fr[k & 1] + R0) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    if (lane < Q) *reinterpret_cast<int4*>(d.fx[k & 1] + R0) = make_int4(0, 0, 0, 0);
  }
  if (lane == 0) d.act[chunk] = (a == 3) ? 2 : 0;
}

template <int SR>
__device__ __forceinline__ void acc_quad(const Dev& d, int km1, int4 c, typename Semi<SR>::T acc[4]) {
  using S = Semi<SR>;
  if (c.x >= 0) acc[0] = S::op(acc[0], S::load(d, km1, c.x));
  if (c.y >= 0) acc[1] = S::op(acc[1], S::load(d, km1, c.y));
  if (c.z >= 0) acc[2] = S::op(acc[2], S::load(d, km1, c.z));
  if (c.w >= 0) acc[3] = S::op(acc[3], S::load(d, km1, c.w));
}

constexpr int PULL_THREADS = 256;
constexpr int PULL_UNROLL = 2;

// One frontier expansion x_k = A (x)_S f_{k-1} with fused post-processing.
template <int SR, int C, bool SLIMWORK>
__global__ void __launch_bounds__(PULL_THREADS) k_pull(Dev d) {
  using S = Semi<SR>;
  using T = typename S::T;
  constexpr int Q = C / 4;
  if (d.ctl->done) return;
  const int k = d.ctl->k;
  const int km1 = k - 1;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * PULL_THREADS + threadIdx.x) >> 5;
  const int nw = (gridDim.x * PULL_THREADS) >> 5;
  Counters cnt;
  for (int it = wid; it < d.n_items; it += nw) {
    const int4 item = d.items[it];
    const int chunk = item.x;
    if (SLIMWORK) {
      unsigned char a = d.act[chunk];
      if (a != 1) {
        if (item.y == 0) carry_chunk<SR, C>(d, k, chunk, lane, a);
        continue;
      }
    }
    T acc[4] = {S::id(), S::id(), S::id(), S::id()};
    const int nq = (item.z - item.y) * Q;
    const int4* base = reinterpret_cast<const int4*>(d.col + d.cs[chunk] + (long long)item.y * C);
    int q = lane;
    for (; q + 32 * (PULL_UNROLL - 1) < nq; q += 32 * PULL_UNROLL) {
      int4 c[PULL_UNROLL];
#pragma unroll
      for (int u = 0; u < PULL_UNROLL; ++u) c[u] = ld_stream(base + q + 32 * u);
#pragma unroll
      for (int u = 0; u < PULL_UNROLL; ++u) acc_quad<SR>(d, km1, c[u], acc);
    }
    for (; q < nq; q += 32) acc_quad<SR>(d, km1, ld_stream(base + q), acc);
    // lanes with equal lane mod Q hold partial results of the same rows
#pragma unroll
    for (int off = Q; off < 32; off <<= 1) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (SR == SS_REAL) acc[r] = S::op(acc[r], __shfl_xor_sync(SS_FULL_MASK, acc[r], off));
        else acc[r] = S::op(acc[r], (T)__shfl_xor_sync(SS_FULL_MASK, (int)acc[r], off));
      }
    }
    if (lane == 0) cnt.slots += (unsigned long long)(item.z - item.y) * C;
    if (item.w >= 0) {  // SlimChunk: combine partial rows, the last arriving item post-processes
      unsigned* xa = d.xacc + (size_t)item.w * C + 4 * lane;
      if (lane < Q) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (S::found(acc[r])) S::atomic(xa + r, acc[r]);
        __threadfence();
      }
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        unsigned old = atomicAdd(d.arrive + item.w, 1u);
        last = (old == (unsigned)d.split_n[item.w] - 1u);
      }
      last = __shfl_sync(SS_FULL_MASK, last, 0);
      if (!last) continue;
      __threadfence();
      if (lane < Q) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[r] = S::from_bits(__ldcg(xa + r));
          xa[r] = S::bits(S::id());
        }
      }
      if (lane == 0) d.arrive[item.w] = 0u;
    }
    if (lane == 0) cnt.act += 1;
    post_chunk<SR, C>(d, k, chunk, lane, acc, cnt);
  }
  // warp, then block reduction of the counters; one atomic per block and counter
  __shared__ unsigned long long red[4][PULL_THREADS / 32];
  unsigned long long v[4] = {cnt.nw, cnt.deg, cnt.slots, cnt.act};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(SS_FULL_MASK, v[i], off);
    if (lane == 0) red[i][threadIdx.x >> 5] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long s = 0;
#pragma unroll
    for (int w = 0; w < PULL_THREADS / 32; ++w) s += red[threadIdx.x][w];
    if (s) {
      unsigned long long* dst = threadIdx.x == 0 ? &d.ctl->new_count
                              : threadIdx.x == 1 ? &d.ctl->new_deg
                              : threadIdx.x == 2 ? &d.ctl->slots
                                                 : &d.ctl->active;
      atomicAdd(dst, s);
    }
  }
}

// End of an iteration: record statistics, test convergence, advance k.
__global__ void k_tail(Dev d, int variant) {
  Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  if (k < d.iter_cap) {
    ss_iter_stats s;
    s.frontier = (long long)c->new_count;
    s.frontier_degree = (long long)c->new_deg;
    s.slots = (long long)c->slots;
    s.active_chunks = (long long)c->active;
    s.variant = variant;
    s.reserved = 0;
    d.iters[k] = s;
  }
  c->reached += c->new_count;
  c->reached_deg += c->new_deg;
  c->total_slots += c->slots;
  c->variant = variant;
  if (c->new_count == 0) c->done = 1;
  c->new_count = 0;
  c->new_deg = 0;
  c->slots = 0;
  c->active = 0;
  c->k = k + 1;
}

__global__ void k_init(Dev d, int sr) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long r = t0; r < d.n_pad; r += stride) {
    d.lvl[r] = r < d.n ? SS_INF : SS_PAD_LEVEL;
    if (sr == SS_REAL) { d.fr[0][r] = 0.0f; d.fr[1][r] = 0.0f; }
    if (sr == SS_SELMAX) { d.fx[0][r] = 0; d.fx[1][r] = 0; d.par[r] = 0; }
  }
  if (sr == SS_BOOLEAN) {
    const long long words = ((long long)d.n_pad + 31) / 32;
    for (long long w = t0; w < words; w += stride) { d.fb[0][w] = 0u; d.fb[1][w] = 0u; }
  }
  for (long long i = t0; i < d.n_c; i += stride) d.act[i] = 1;
  const unsigned ident = (sr == SS_TROPICAL) ? (unsigned)SS_INF : 0u;
  for (long long s = t0; s < (long long)d.n_split * d.C; s += stride) d.xacc[s] = ident;
}

__global__ void k_init_root(Dev d, int sr, int root) {
  const int r = d.invperm[root];
  d.lvl[r] = 0;
  if (sr == SS_BOOLEAN) d.fb[0][r >> 5] |= 1u << (r & 31);
  if (sr == SS_REAL) d.fr[0][r] = 1.0f;
  if (sr == SS_SELMAX) { d.fx[0][r] = root + 1; d.par[r] = root + 1; }
  Ctl* c = d.ctl;
  c->k = 1; c->done = 0; c->error = 0; c->variant = -1;
  c->new_count = 0; c->new_deg = 0; c->slots = 0; c->active = 0;
  c->reached = 1; c->reached_deg = (unsigned long long)d.rdeg[r];
  c->total_slots = 0; c->dp_slots = 0;
  ss_iter_stats s;
  s.frontier = 1; s.frontier_degree = d.rdeg[r]; s.slots = 0; s.active_chunks = 0;
  s.variant = -1; s.reserved = 0;
  d.iters[0] = s;
}

// DP transformation (Section II-C): the parent of a row at level L >= 1 is its
// largest-id neighbour at level L-1.  Neighbours are stored in descending
// original id, so each lane's first hit in its column sequence is that lane's
// maximum; lanes stop once their rows are resolved and the group takes the max.
template <int C>
__global__ void __launch_bounds__(PULL_THREADS) k_dp(Dev d) {
  constexpr int Q = C / 4;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * PULL_THREADS + threadIdx.x) >> 5;
  const int nw = (gridDim.x * PULL_THREADS) >> 5;
  unsigned long long my_slots = 0;
  for (int it = wid; it < d.n_items; it += nw) {
    const int4 item = d.items[it];
    const int chunk = item.x;
    const int R0 = chunk * C + 4 * (lane % Q);
    int4 lv = *reinterpret_cast<const int4*>(d.lvl + R0);
    int tgt[4] = {lv.x, lv.y, lv.z, lv.w};
    int best[4];
    bool need = false;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      tgt[r] = (tgt[r] >= 1 && tgt[r] != SS_INF) ? tgt[r] - 1 : -2;
      best[r] = -1;
      need |= tgt[r] >= 0;
    }
    const int nq = (item.z - item.y) * Q;
    const int4* base = reinterpret_cast<const int4*>(d.col + d.cs[chunk] + (long long)item.y * C);
    int q = lane;
    while (__any_sync(SS_FULL_MASK, need && q < nq)) {
      if (need && q < nq) {
        int4 c = ld_stream(base + q);
        int cc[4] = {c.x, c.y, c.z, c.w};
        need = false;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (best[r] < 0 && tgt[r] >= 0) {
            if (cc[r] >= 0 && d.lvl[cc[r]] == tgt[r]) best[r] = d.perm[cc[r]];
            else need = true;
          }
        }
        q += 32;
        my_slots += 4;
      }
    }
#pragma unroll
    for (int off = Q; off < 32; off <<= 1)
#pragma unroll
      for (int r = 0; r < 4; ++r) best[r] = max(best[r], __shfl_xor_sync(SS_FULL_MASK, best[r], off));
    if (lane < Q) {
      if (item.w < 0) {
        *reinterpret_cast<int4*>(d.par + R0) = make_int4(best[0], best[1], best[2], best[3]);
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (best[r] >= 0) atomicMax(d.par + R0 + r, best[r]);
      }
    }
  }
  __shared__ unsigned long long red[PULL_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) my_slots += __shfl_down_sync(SS_FULL_MASK, my_slots, off);
  if (lane == 0) red[threadIdx.x >> 5] = my_slots;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < PULL_THREADS / 32; ++w) s += red[w];
    if (s) atomicAdd(&d.ctl->dp_slots, s);
  }
}

__global__ void k_output(Dev d, int* dist, int* parent, int selmax) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < d.n;
       v += (long long)gridDim.x * blockDim.x) {
    const int r = d.invperm[v];
    const int L = d.lvl[r];
    if (dist) dist[v] = (L == SS_INF) ? -1 : L;
    if (parent) {
      int p;
      if (L == SS_INF) p = -1;
      else if (L == 0) p = (int)v;
      else p = selmax ? d.par[r] - 1 : d.par[r];
      parent[v] = p;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename K>
static int grid_for(K kernel, int num_sms) {
  int blocks = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, PULL_THREADS, 0);
  if (blocks < 1) blocks = 1;
  return blocks * num_sms;
}

template <int SR, int C>
static ss_status launch_pull(const slimsell_graph* h, const Dev& d, bool slimwork, cudaStream_t st) {
  if (slimwork) {
    static int g = 0;
    if (!g) g = grid_for(k_pull<SR, C, true>, h->num_sms);
    k_pull<SR, C, true><<<g, PULL_THREADS, 0, st>>>(d);
  } else {
    static int g = 0;
    if (!g) g = grid_for(k_pull<SR, C, false>, h->num_sms);
    k_pull<SR, C, false><<<g, PULL_THREADS, 0, st>>>(d);
  }
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

template <int SR>
static ss_status launch_pull_c(const slimsell_graph* h, const Dev& d, bool slimwork, cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_pull<SR, 8>(h, d, slimwork, st);
    case 16: return launch_pull<SR, 16>(h, d, slimwork, st);
    case 32: return launch_pull<SR, 32>(h, d, slimwork, st);
    default: return launch_pull<SR, 64>(h, d, slimwork, st);
  }
}

static ss_status launch_iteration(const slimsell_graph* h, const Dev& d, int sr, bool slimwork,
                                  cudaStream_t st) {
  switch (sr) {
    case SS_TROPICAL: return launch_pull_c<SS_TROPICAL>(h, d, slimwork, st);
    case SS_REAL: return launch_pull_c<SS_REAL>(h, d, slimwork, st);
    case SS_BOOLEAN: return launch_pull_c<SS_BOOLEAN>(h, d, slimwork, st);
    default: return launch_pull_c<SS_SELMAX>(h, d, slimwork, st);
  }
}

template <int C>
static ss_status launch_dp_c(const slimsell_graph* h, const Dev& d, cudaStream_t st) {
  static int g = 0;
  if (!g) g = grid_for(k_dp<C>, h->num_sms);
  k_dp<C><<<g, PULL_THREADS, 0, st>>>(d);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

static ss_status launch_dp(const slimsell_graph* h, const Dev& d, cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_dp_c<8>(h, d, st);
    case 16: return launch_dp_c<16>(h, d, st);
    case 32: return launch_dp_c<32>(h, d, st);
    default: return launch_dp_c<64>(h, d, st);
  }
}

}  // namespace ss

extern "C" {

ss_status slimsell_bfs(slimsell_handle h, int32_t root, int32_t semiring, int32_t policy,
                       int32_t* d_dist, int32_t* d_parent, void* stream) {
  using namespace ss;
  set_error("");
  if (!h) {
    set_error("slimsell_bfs: NULL handle");
    return SS_ERR_INVALID;
  }
  if (root < 0 || root >= h->n) {
    set_error("slimsell_bfs: root %d out of range [0, %d)", root, h->n);
    return SS_ERR_INVALID;
  }
  if (semiring < SS_TROPICAL || semiring > SS_SELMAX) {
    set_error("slimsell_bfs: unknown semiring %d", semiring);
    return SS_ERR_INVALID;
  }
  if (policy < SS_V_FULL || policy > SS_V_LEARNED) {
    set_error("slimsell_bfs: unknown policy %d", policy);
    return SS_ERR_INVALID;
  }
  if (policy != SS_V_FULL && policy != SS_V_SLIMWORK) {
    set_error("slimsell_bfs: policy %d not available in this build", policy);
    return SS_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const Dev d = h->dev();
  const bool slimwork = policy == SS_V_SLIMWORK;
  const int grid = 8 * h->num_sms;
  const bool prof = h->profiling != 0;
  double iter_ms = 0.0;
  if (prof) SS_CUDA(cudaEventRecord(h->ev_c, st));

  k_init<<<grid, 256, 0, st>>>(d, semiring);
  k_init_root<<<1, 1, 0, st>>>(d, semiring, root);
  SS_CUDA(cudaGetLastError());

  const long long max_iter = (long long)h->n + 2;
  for (long long it = 0;; ++it) {
    if (it > max_iter) {
      set_error("slimsell_bfs: no convergence after %lld iterations", it);
      return SS_ERR_CUDA;
    }
    if (prof) SS_CUDA(cudaEventRecord(h->ev_a, st));
    ss_status s = launch_iteration(h, d, semiring, slimwork, st);
    if (s != SS_OK) return s;
    if (prof) SS_CUDA(cudaEventRecord(h->ev_b, st));
    k_tail<<<1, 1, 0, st>>>(d, slimwork ? SS_V_SLIMWORK : SS_V_FULL);
    SS_CUDA(cudaGetLastError());
    SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    if (prof) {
      float ms = 0.f;
      SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
      iter_ms += ms;
    }
    if (h->h_ctl->done) break;
  }
  const int iterations = h->h_ctl->k - 1;

  if (d_parent && semiring != SS_SELMAX) {
    SS_CUDA(cudaMemsetAsync(h->par, 0xff, sizeof(int) * (size_t)h->n_pad, st));
    ss_status s = launch_dp(h, d, st);
    if (s != SS_OK) return s;
  }
  if (d_dist || d_parent) {
    k_output<<<grid, 256, 0, st>>>(d, d_dist, d_parent, semiring == SS_SELMAX);
    SS_CUDA(cudaGetLastError());
  }
  if (prof) SS_CUDA(cudaEventRecord(h->ev_d, st));
  SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  const Ctl& c = *h->h_ctl;
  h->last.iterations = iterations;
  h->last.semiring = semiring;
  h->last.reached = (long long)c.reached;
  h->last.reached_degree = (long long)c.reached_deg;
  h->last.slots = (long long)c.total_slots;
  h->last.dp_slots = (long long)c.dp_slots;
  h->last.iter_kernel_ms = iter_ms;
  h->last.total_ms = 0.0;
  if (prof) {
    float ms = 0.f;
    SS_CUDA(cudaEventElapsedTime(&ms, h->ev_c, h->ev_d));
    h->last.total_ms = ms;
  }
  return SS_OK;
}

ss_status slimsell_get_run_stats(slimsell_handle h, ss_run_stats* out, ss_iter_stats* h_iters,
                                 int32_t cap) {
  if (!h || !out) {
    ss::set_error("slimsell_get_run_stats: NULL argument");
    return SS_ERR_INVALID;
  }
  *out = h->last;
  if (h_iters && cap > 0) {
    int cnt = h->last.iterations + 1;
    if (cnt > cap) cnt = cap;
    if (cnt > h->iter_cap) cnt = h->iter_cap;
    SS_CUDA(cudaMemcpy(h_iters, h->iters, sizeof(ss_iter_stats) * (size_t)cnt, cudaMemcpyDeviceToHost));
  }
  return SS_OK;
}

ss_status slimsell_set_profiling(slimsell_handle h, int32_t on) {
  if (!h) {
    ss::set_error("slimsell_set_profiling: NULL handle");
    return SS_ERR_INVALID;
  }
  h->profiling = on ? 1 : 0;
  return SS_OK;
}

}  // extern "C"
