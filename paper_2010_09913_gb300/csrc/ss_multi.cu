// Multi-source BFS: the boolean semiring of Section III-A run for up to 1024
// sources at once with bit-packed frontiers (an extension beyond the paper).
//
//   F[k&1][r][w]  bit s of word w: row r entered source 64w+s's frontier at level k
//   V[r][w]       visited bits (g_k = not V)
//   x = OR over the row's neighbours u of F[u][w]; new = x & ~V; V |= new;
//   F_next = new; dist[v][64w+s] = k for every new bit.
//
// One thread block handles one work item (chunk i, columns [j0, j1)); thread
// (r, w) = threadIdx.x / W, % W owns word w of row r.  The W threads of a row
// read the same col entry (a broadcast) and gather the W contiguous frontier
// words of the neighbour (one W*8-byte segment).  SlimWork skips chunks whose
// rows have every source visited; split chunks (SlimChunk) combine partial ORs
// with 64-bit atomicOr and the last arriving block post-processes.
//
// The gathers are most of the traffic (W*8 bytes per slot), so they are
// skipped where they cannot matter: a one-bit-per-vertex summary of the
// frontier (bit u set iff some source has u in its frontier, kept in the
// single-source frontier bitmaps fb[], unused here) is tested first, and a
// thread whose 64 sources have all visited its row gathers nothing.
//
// Parents (optional) come from a separate pass after each level: a row's
// neighbours are stored in descending original id, so for each source that
// the row gained at level k, the first neighbour in storage order that was in
// that source's level-(k-1) frontier is its largest-id parent.  The pass
// reads F[(k-1)&1] and the summary bitmap of level k-1, both still intact
// until level k+1 overwrites them.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "ss_device.cuh"

namespace ss {

#ifndef SS_MULTI_BATCH
#define SS_MULTI_BATCH 4
#endif
constexpr int MULTI_BATCH = SS_MULTI_BATCH;  // columns per thread in flight
#ifndef SS_MULTI_BLOCKS_PER_SM
#define SS_MULTI_BLOCKS_PER_SM 0  // resident blocks per SM (0: as many as fit)
#endif

// Distances of the new sources (bits of nb) of one 64-source word, in 16-byte
// groups of 4: a group with no earlier discovery (bits of vold) still holds -1
// everywhere and is written whole; otherwise it is read first.  Kept out of line
// so that the gather loop's register allocation does not depend on it.
__device__ __noinline__ void write_levels_vec(int* out, unsigned long long nb, unsigned long long vold,
                                             int level) {
  for (int gi = 0; gi < 16; ++gi) {
    const unsigned ng = (unsigned)(nb >> (4 * gi)) & 0xFu;
    if (!ng) continue;
    int4* q = reinterpret_cast<int4*>(out) + gi;
    int4 v = ((unsigned)(vold >> (4 * gi)) & 0xFu) ? *q : make_int4(-1, -1, -1, -1);
    if (ng & 1u) v.x = level;
    if (ng & 2u) v.y = level;
    if (ng & 4u) v.z = level;
    if (ng & 8u) v.w = level;
    *q = v;
  }
}

// The C summary bits of one chunk (bit l = row l) into the bitmap.
template <int C>
__device__ __forceinline__ void store_summary(unsigned* fa, int chunk, unsigned lo, unsigned hi) {
  if (C == 8) reinterpret_cast<unsigned char*>(fa)[chunk] = (unsigned char)lo;
  else if (C == 16) reinterpret_cast<unsigned short*>(fa)[chunk] = (unsigned short)lo;
  else if (C == 32) fa[chunk] = lo;
  else reinterpret_cast<uint2*>(fa)[chunk] = make_uint2(lo, hi);
}

template <int C, int W, bool SLIMWORK>
__global__ void __launch_bounds__(C * W) k_multi_pull(MultiDev m, IterLaunch il) {
  constexpr int T = C * W;
  const Dev& d = m.d;
  Ctl* c = d.ctl;
  if (c->done) return;
  const int level = c->k;
  const int tid = threadIdx.x, r = tid / W, w = tid % W;
  const unsigned long long* Fp = m.F[(level - 1) & 1];
  unsigned long long* Fn = m.F[level & 1];
  const unsigned* FAp = d.fb[(level - 1) & 1];  // frontier summary, one bit per row
  unsigned* FAn = d.fb[level & 1];
  __shared__ int s_flag;
  __shared__ unsigned s_fa[2];
  unsigned long long nw = 0, deg = 0, slots = 0, act = 0;
  unsigned maxdeg = 0;
  __shared__ unsigned long long s_rowdeg;  // degree sum of the block's rows that gained a source
  if (tid == 0) s_rowdeg = 0ull;
  for (int it = blockIdx.x; it < d.n_items; it += gridDim.x) {
    const int4 item = d.items[it];
    const int chunk = item.x;
    const long long row = (long long)chunk * C + r;
    if (SLIMWORK) {
      const int a = d.act[chunk];
      __syncthreads();  // every thread has read the state before it may change
      if (a != 1) {
        if (a >= 2 && item.y == 0) {
          Fn[row * W + w] = 0ull;  // f_k is zero on a finished chunk
          if (tid == 0) {
            store_summary<C>(FAn, chunk, 0u, 0u);
            d.act[chunk] = (a == 3) ? 2 : 0;
          }
        }
        continue;
      }
    }
    const long long start = d.cs[chunk] + (long long)item.y * C;
    const int ncol = item.z - item.y;
    const unsigned long long vold0 = m.V[row * W + w];
    const bool want = vold0 != ~0ull;  // some of this word's sources still miss the row
    unsigned long long acc = 0ull;
    int j = 0;
    for (; j + MULTI_BATCH <= ncol; j += MULTI_BATCH) {
      int cc[MULTI_BATCH];
#pragma unroll
      for (int q = 0; q < MULTI_BATCH; ++q) cc[q] = __ldcs(d.col + start + (long long)(j + q) * C + r);
      unsigned hit[MULTI_BATCH];
#pragma unroll
      for (int q = 0; q < MULTI_BATCH; ++q)
        hit[q] = (want && cc[q] >= 0) ? (__ldg(FAp + (cc[q] >> 5)) >> (cc[q] & 31)) & 1u : 0u;
#pragma unroll
      for (int q = 0; q < MULTI_BATCH; ++q)
        if (hit[q]) acc |= __ldg(Fp + (long long)cc[q] * W + w);
    }
    for (; j < ncol; ++j) {
      const int cc = __ldcs(d.col + start + (long long)j * C + r);
      if (want && cc >= 0 && ((__ldg(FAp + (cc >> 5)) >> (cc & 31)) & 1u))
        acc |= __ldg(Fp + (long long)cc * W + w);
    }
    if (tid == 0) slots += (unsigned long long)ncol * C;
    if (item.w >= 0) {  // SlimChunk: OR the partial rows, last block to arrive post-processes
      unsigned long long* xa = m.xacc + ((size_t)item.w * C + r) * W + w;
      if (acc) atomicOr(xa, acc);
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const unsigned old = atomicAdd(d.arrive + item.w, 1u);
        s_flag = (old == (unsigned)d.split_n[item.w] - 1u);
      }
      __syncthreads();
      if (!s_flag) continue;
      __threadfence();
      acc = __ldcg(xa);
      *xa = 0ull;
      if (tid == 0) d.arrive[item.w] = 0u;
    }
    if (tid == 0) s_fa[0] = s_fa[1] = 0u;
    __syncthreads();
    const unsigned long long vold = vold0;
    const unsigned long long nb = acc & ~vold;
    if (nb) atomicOr(&s_fa[r >> 5], 1u << (r & 31));
    if (nb) {
      m.V[row * W + w] = vold | nb;
      const int pc = __popcll(nb);
      const int dv = d.rdeg[row];
      nw += (unsigned long long)pc;
      deg += (unsigned long long)pc * (unsigned long long)dv;
      maxdeg = max(maxdeg, (unsigned)dv);
      if (m.dist) {
        int* out = m.dist + (long long)d.perm[row] * m.k + 64 * w;
        if (m.vec_dist) {
          write_levels_vec(out, nb, vold, level);
        } else {
          unsigned long long b = nb;
          while (b) {
            const int s = __ffsll((long long)b) - 1;
            b &= b - 1;
            out[s] = level;
          }
        }
      }
    }
    Fn[row * W + w] = nb;
    const int left = __syncthreads_or((vold | nb) != ~0ull);
    if (w == 0 && ((s_fa[r >> 5] >> (r & 31)) & 1u)) atomicAdd(&s_rowdeg, (unsigned long long)d.rdeg[row]);
    if (tid == 0) {
      store_summary<C>(FAn, chunk, s_fa[0], s_fa[1]);
      d.act[chunk] = left ? 1 : 3;
      act += 1;
    }
  }
  // degree sum of the rows that gained a source, each row counted once (the
  // parents pass picks its direction from it)
  __syncthreads();
  if (tid == 0 && s_rowdeg) {
    atomicAdd(&c->new_rowdeg, s_rowdeg);
    __threadfence();  // before this block counts itself done
  }
  finish_iteration_block<T>(d, nw, deg, slots, act, maxdeg, il);
}

__global__ void k_multi_init(MultiDev m, int W) {
  const Dev& d = m.d;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long words = (long long)d.n_pad * W;
  // padding rows and sources beyond k count as visited
  for (long long i = t0; i < words; i += stride) {
    const long long r = i / W;
    const int w = (int)(i % W);
    unsigned long long v = 0ull;
    if (r >= d.n) {
      v = ~0ull;
    } else {
      const int lo = 64 * w;  // sources lo .. lo+63; those >= k never exist
      if (lo >= m.k) v = ~0ull;
      else if (m.k - lo < 64) v = ~0ull << (m.k - lo);
    }
    m.V[i] = v;
    m.F[0][i] = 0ull;
    m.F[1][i] = 0ull;
  }
  for (long long i = t0; i < d.n_c; i += stride) d.act[i] = 1;
  for (long long s = t0; s < (long long)d.n_split * d.C * W; s += stride) m.xacc[s] = 0ull;
  for (long long i = t0; i < d.fb_words; i += stride) {
    d.fb[0][i] = 0u;
    d.fb[1][i] = 0u;
  }
}

__global__ void k_multi_roots(MultiDev m, int W, int* parent) {
  const Dev& d = m.d;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m.k; s += gridDim.x * blockDim.x) {
    const int v = m.roots[s];
    const long long r = d.invperm[v];
    const unsigned long long bit = 1ull << (s & 63);
    atomicOr(m.V + r * W + s / 64, bit);
    atomicOr(m.F[0] + r * W + s / 64, bit);
    atomicOr(d.fb[0] + (r >> 5), 1u << (r & 31));
    if (m.dist) m.dist[(long long)v * m.k + s] = 0;
    if (parent) parent[(long long)v * m.k + s] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl* c = d.ctl;
    unsigned long long rd = 0;
    for (int s = 0; s < m.k; ++s) rd += (unsigned long long)d.rdeg[d.invperm[m.roots[s]]];
    c->k = 1; c->done = 0; c->error = 0; c->variant = -1;
    c->new_count = 0; c->new_deg = 0; c->slots = 0; c->active = 0;
    c->reached = (unsigned long long)m.k; c->reached_deg = rd;
    c->total_slots = 0; c->dp_slots = 0; c->blocks_done = 0;
    c->prev_variant = -1; c->prev_slots = 0; c->prev_new = (unsigned long long)m.k; c->prev_deg = rd;
    c->prev2_new = 0; c->prev_active = 0; c->new_maxdeg = 0; c->prev_maxdeg = 0; c->units = 0; c->bunits = 0;
    c->loop_guard = 0;
    for (int v = 0; v < N_VARIANTS; ++v) c->variant_count[v] = 0;
    c->list_level = -1; c->list_prev_ok = 0; c->qlen[0] = c->qlen[1] = 0; c->qprep = 0;
    c->new_rowdeg = 0;
    c->prev_rowdeg = rd;  // the roots' rows (a repeated root counted again: an upper bound)
    ss_iter_stats st;
    st.frontier = m.k; st.frontier_degree = (long long)rd; st.slots = 0; st.active_chunks = 0;
    st.variant = -1; st.kernel_ns = 0;
    d.iters[0] = st;
  }
}

// Parents of the sources each row gained at `level`: (row, w) walks the row's
// neighbours in storage order (descending original id) and gives each new
// source of word w the first neighbour found in its frontier of level-1,
// stopping once every new source has one.  Each lane first walks its own row
// for up to MULTI_PAR_SHORT neighbours; rows still unresolved then are walked
// by the whole warp, 32 neighbours per step, the candidates taken in lane
// (= storage) order.  Plain stores: one lane owns each (row, word) entry.
constexpr int MULTI_PAR_SHORT = 32;
// The parents pass pushes from the previous frontier while the run grows and
// that frontier's rows carry at most nnz / MULTI_PAR_PUSH_SHARE edges.
#ifndef SS_MULTI_PAR_PUSH_SHARE
#define SS_MULTI_PAR_PUSH_SHARE 2
#endif
constexpr unsigned long long MULTI_PAR_PUSH_SHARE = SS_MULTI_PAR_PUSH_SHARE;

__global__ void __launch_bounds__(256) k_multi_parents(MultiDev m, int W, int lgW, int level, int* parent) {
  const Dev& d = m.d;
  const unsigned long long* Fp = m.F[(level - 1) & 1];
  const unsigned long long* Fn = m.F[level & 1];
  const unsigned* FAp = d.fb[(level - 1) & 1];
  const long long words = (long long)d.n_pad << lgW;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i0 = warp0 * 32; i0 < words; i0 += nwarps * 32) {
    const long long i = i0 + lane;
    unsigned long long rem = i < words ? Fn[i] : 0ull;
    const long long row = i >> lgW;
    const int w = (int)(i & (W - 1));
    const int v = rem ? d.perm[row] : -1;
    if (v < 0) rem = 0ull;  // padding rows never gain a source
    long long base = 0;
    int len = 0, j = 0;
    int* prow = nullptr;
    if (rem) {
      prow = parent + (long long)v * m.k + 64 * w;
      const long long chunk = row / d.C;
      base = d.cs[chunk] + (row - chunk * d.C);
      len = d.rdeg[row];  // the row's neighbours come first, padding after
      for (; j < len && j < MULTI_PAR_SHORT && rem; ++j) {
        const int u = __ldg(d.col + base + (long long)j * d.C);
        if (!((__ldg(FAp + (u >> 5)) >> (u & 31)) & 1u)) continue;
        unsigned long long f = __ldg(Fp + ((long long)u << lgW) + w) & rem;
        if (!f) continue;
        rem &= ~f;
        const int pu = __ldg(d.perm + u);
        while (f) {
          prow[__ffsll((long long)f) - 1] = pu;
          f &= f - 1;
        }
      }
    }
    unsigned pend = __ballot_sync(SS_FULL_MASK, rem != 0ull);
    while (pend) {  // long rows, one at a time, by the whole warp
      const int l = __ffs(pend) - 1;
      pend &= pend - 1;
      unsigned long long rl = __shfl_sync(SS_FULL_MASK, rem, l);
      const long long bl = __shfl_sync(SS_FULL_MASK, base, l);
      const int nl = __shfl_sync(SS_FULL_MASK, len, l);
      const int jl = __shfl_sync(SS_FULL_MASK, j, l);
      const int wl = __shfl_sync(SS_FULL_MASK, w, l);
      int* const pl = reinterpret_cast<int*>(
          __shfl_sync(SS_FULL_MASK, reinterpret_cast<unsigned long long>(prow), l));
      for (int jj = jl; jj < nl && rl; jj += 32) {
        const int jx = jj + lane;
        unsigned long long f = 0ull;
        int u = 0;
        if (jx < nl) {
          u = __ldg(d.col + bl + (long long)jx * d.C);
          if ((__ldg(FAp + (u >> 5)) >> (u & 31)) & 1u) f = __ldg(Fp + ((long long)u << lgW) + wl) & rl;
        }
        unsigned cand = __ballot_sync(SS_FULL_MASK, f != 0ull);
        const int pu = f ? __ldg(d.perm + u) : -1;
        while (cand) {  // lane order is storage order
          const int c2 = __ffs(cand) - 1;
          cand &= cand - 1;
          const unsigned long long fc = __shfl_sync(SS_FULL_MASK, f, c2) & rl;
          if (!fc) continue;
          rl &= ~fc;
          if (lane == c2) {
            unsigned long long b = fc;
            while (b) {
              pl[__ffsll((long long)b) - 1] = pu;
              b &= b - 1;
            }
          }
        }
      }
    }
  }
}

// Parents of the sources gained at `level`, pushed from the frontier of level
// - 1 (for levels whose frontier rows carry few edges).  k_multi_par_expand
// turns every row u of that frontier (summary bit set) into units of
// PUSH_UNIT neighbours; in k_multi_par_scatter one warp takes a unit and its
// lanes walk the unit's neighbours v: each source s in F[level][v] &
// F[level-1][u] has u one level closer to s than v, and atomicMax keeps the
// largest original id over all such u (parents start at -1).
__global__ void __launch_bounds__(256) k_multi_par_expand(MultiDev m, int level) {
  const Dev& d = m.d;
  const unsigned* FAp = d.fb[(level - 1) & 1];
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long words = ((long long)d.n_pad + 31) / 32;
  const long long wstride = stride & ~31LL;  // whole warps walk the summary together
  for (long long i0 = t0 - lane; i0 < words; i0 += wstride) {
    const long long i = i0 + lane;
    unsigned bits = i < words ? FAp[i] : 0u;
    while (__any_sync(SS_FULL_MASK, bits != 0u)) {
      int u = -1;
      if (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        u = (int)(i * 32 + b);
      }
      emit_units(d, u, lane);
    }
  }
}

__global__ void __launch_bounds__(256) k_multi_par_scatter(MultiDev m, int W, int lgW, int level,
                                                           int* parent) {
  const Dev& d = m.d;
  const unsigned long long* Fp = m.F[(level - 1) & 1];
  const unsigned long long* Fn = m.F[level & 1];
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nunits = min((long long)d.ctl->units, d.units_cap);
  for (long long ui = wid; ui < nunits; ui += nw) {
    const int2 un = d.units[ui];
    const long long u = un.x;
    const int pu = __ldg(d.perm + u);
    const int end = min(__ldg(d.rdeg + u), un.y + PUSH_UNIT);
    const long long chunk = u / d.C;
    const long long base = __ldg(d.cs + chunk) + (u - chunk * d.C);
    for (int ww = 0; ww < W; ++ww) {
      const unsigned long long fu = __ldg(Fp + (u << lgW) + ww);
      if (!fu) continue;
      for (int j = un.y + lane; j < end; j += 32) {
        const int v = __ldg(d.col + base + (long long)j * d.C);
        unsigned long long g = __ldcg(Fn + ((long long)v << lgW) + ww) & fu;
        if (!g) continue;
        int* prow = parent + (long long)__ldg(d.perm + v) * m.k + 64 * ww;
        while (g) {
          atomicMax(prow + (__ffsll((long long)g) - 1), pu);
          g &= g - 1;
        }
      }
    }
  }
}

template <int C, int W>
static ss_status launch_multi_cw(const slimsell_graph* h, const MultiDev& m, bool slimwork,
                                 const IterLaunch& il, cudaStream_t st) {
  if constexpr (C * W < 32) {
    set_error("slimsell_bfs_multi: C * ceil(k / 64) must be at least 32");
    return SS_ERR_UNSUPPORTED;
  } else {
    static int grid[64][2];  // per device (zero: not measured yet)
    int& g = grid[h->device & 63][slimwork ? 1 : 0];
    if (!g) {
      int b = 0;
      if (slimwork) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_multi_pull<C, W, true>, C * W, 0);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_multi_pull<C, W, false>, C * W, 0);
      if (SS_MULTI_BLOCKS_PER_SM > 0) b = std::min(b, SS_MULTI_BLOCKS_PER_SM);
      g = (b > 0 ? b : 1) * h->num_sms;
    }
    if (slimwork) k_multi_pull<C, W, true><<<g, C * W, 0, st>>>(m, il);
    else k_multi_pull<C, W, false><<<g, C * W, 0, st>>>(m, il);
    SS_CUDA(cudaGetLastError());
    return SS_OK;
  }
}

template <int C>
static ss_status launch_multi_c(const slimsell_graph* h, const MultiDev& m, int W, bool slimwork,
                                const IterLaunch& il, cudaStream_t st) {
  switch (W) {
    case 1: return launch_multi_cw<C, 1>(h, m, slimwork, il, st);
    case 2: return launch_multi_cw<C, 2>(h, m, slimwork, il, st);
    case 4: return launch_multi_cw<C, 4>(h, m, slimwork, il, st);
    case 8: return launch_multi_cw<C, 8>(h, m, slimwork, il, st);
    default: return launch_multi_cw<C, 16>(h, m, slimwork, il, st);
  }
}

static ss_status launch_multi(const slimsell_graph* h, const MultiDev& m, int W, bool slimwork,
                              const IterLaunch& il, cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_multi_c<8>(h, m, W, slimwork, il, st);
    case 16: return launch_multi_c<16>(h, m, W, slimwork, il, st);
    case 32: return launch_multi_c<32>(h, m, W, slimwork, il, st);
    default: return launch_multi_c<64>(h, m, W, slimwork, il, st);
  }
}

// Multi-source scratch, grown on demand and kept with the handle.
static ss_status ensure_multi_scratch(slimsell_graph* h, int W) {
  if (h->multi_w >= W) return SS_OK;
  void* ptrs[] = {h->mF[0], h->mF[1], h->mV, h->mxacc, h->mroots};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->mF[0] = h->mF[1] = h->mV = h->mxacc = nullptr;
  h->mroots = nullptr;
  h->multi_w = 0;
  const size_t words = (size_t)h->n_pad * W;
  ss_status s;
  for (int b = 0; b < 2; ++b)
    if ((s = dmalloc(h, (void**)&h->mF[b], sizeof(unsigned long long) * words)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->mV, sizeof(unsigned long long) * words)) != SS_OK) return s;
  const size_t ns = (size_t)(h->n_split > 0 ? h->n_split : 1) * h->C * W;
  if ((s = dmalloc(h, (void**)&h->mxacc, sizeof(unsigned long long) * ns)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->mroots, sizeof(int) * 1024)) != SS_OK) return s;
  h->multi_w = W;
  return SS_OK;
}

// Level-by-level multi-source BFS for the passes built on it (betweenness
// centrality): seeds k sources (device ids, checked by the caller) and returns
// the view of the handle's multi-source state; multi_level then runs one level
// (SlimWork pull) and reports whether it discovered nothing.  The frontier words
// of level L are m->F[L & 1] (W words per row) until level L + 2 overwrites them.
// Optional events are recorded around the level's kernel.
ss_status multi_start(slimsell_graph* h, const int32_t* d_roots, int k, cudaStream_t st, MultiDev* m,
                      int* W_out) {
  int W = 1;
  while (64 * W < k) W *= 2;
  while (h->C * W < 32) W *= 2;
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
  h->pending = 0;
  ss_status s = ensure_multi_scratch(h, W);
  if (s != SS_OK) return s;
  SS_CUDA(cudaMemcpyAsync(h->mroots, d_roots, sizeof(int) * (size_t)k, cudaMemcpyDeviceToDevice, st));
  m->d = h->dev();
  m->d.reach_cap = (unsigned long long)h->n * (unsigned long long)k;
  m->F[0] = h->mF[0];
  m->F[1] = h->mF[1];
  m->V = h->mV;
  m->xacc = h->mxacc;
  m->dist = nullptr;
  m->vec_dist = 0;
  m->roots = h->mroots;
  m->k = k;
  k_multi_init<<<8 * h->num_sms, 256, 0, st>>>(*m, W);
  k_multi_roots<<<(k + 255) / 256, 256, 0, st>>>(*m, W, nullptr);
  SS_CUDA(cudaGetLastError());
  *W_out = W;
  return SS_OK;
}

ss_status multi_level(slimsell_graph* h, const MultiDev& m, int W, cudaStream_t st, bool* done,
                      cudaEvent_t before, cudaEvent_t after) {
  if (before) SS_CUDA(cudaEventRecord(before, st));
  ss_status s = launch_multi(h, m, W, true, IterLaunch{SS_V_SLIMWORK, 0, 0}, st);
  if (s != SS_OK) return s;
  if (after) SS_CUDA(cudaEventRecord(after, st));
  SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  if (h->h_ctl->error) {
    set_error("multi-source BFS: device error flags %d", h->h_ctl->error);
    return SS_ERR_CUDA;
  }
  *done = h->h_ctl->done != 0;
  return SS_OK;
}

}  // namespace ss

extern "C" ss_status slimsell_bfs_multi(slimsell_handle h, const int32_t* d_roots, int32_t k,
                                        int32_t policy, int32_t* d_dist, void* stream) {
  return slimsell_bfs_multi_parents(h, d_roots, k, policy, d_dist, nullptr, stream);
}

extern "C" ss_status slimsell_bfs_multi_parents(slimsell_handle h, const int32_t* d_roots, int32_t k,
                                                int32_t policy, int32_t* d_dist, int32_t* d_parent,
                                                void* stream) {
  using namespace ss;
  set_error("");
  if (!h || !d_roots) {
    set_error("slimsell_bfs_multi: NULL argument");
    return SS_ERR_INVALID;
  }
  h->values_semiring = -1;
  if (k < 1 || k > 1024) {
    set_error("slimsell_bfs_multi: k must be in [1, 1024] (got %d)", k);
    return SS_ERR_INVALID;
  }
  if (policy != SS_V_FULL && policy != SS_V_SLIMWORK) {
    set_error("slimsell_bfs_multi: policy must be SS_V_FULL or SS_V_SLIMWORK");
    return SS_ERR_INVALID;
  }
  int W = 1;
  while (64 * W < k) W *= 2;
  while (h->C * W < 32) W *= 2;  // a block needs a full warp; extra words hold no source
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> roots((size_t)k);
  SS_CUDA(cudaMemcpyAsync(roots.data(), d_roots, sizeof(int) * (size_t)k, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  for (int s = 0; s < k; ++s)
    if (roots[(size_t)s] < 0 || roots[(size_t)s] >= h->n) {
      set_error("slimsell_bfs_multi: root %d of source %d out of range", roots[(size_t)s], s);
      return SS_ERR_INVALID;
    }
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
  h->pending = 0;
  ss_status s = ensure_multi_scratch(h, W);
  if (s != SS_OK) return s;
  SS_CUDA(cudaMemcpyAsync(h->mroots, d_roots, sizeof(int) * (size_t)k, cudaMemcpyDeviceToDevice, st));
  MultiDev m;
  m.d = h->dev();
  m.d.reach_cap = (unsigned long long)h->n * (unsigned long long)k;
  m.F[0] = h->mF[0];
  m.F[1] = h->mF[1];
  m.V = h->mV;
  m.xacc = h->mxacc;
  m.dist = d_dist;
  m.vec_dist = (k % 4 == 0) && ((reinterpret_cast<uintptr_t>(d_dist) & 15u) == 0);
  m.roots = h->mroots;
  m.k = k;
  const bool prof = h->profiling != 0;
  h->iter_ns.clear();
  double iter_ms = 0.0;
  if (prof) SS_CUDA(cudaEventRecord(h->ev_c, st));
  if (d_dist) SS_CUDA(cudaMemsetAsync(d_dist, 0xff, sizeof(int) * (size_t)h->n * (size_t)k, st));
  if (d_parent) SS_CUDA(cudaMemsetAsync(d_parent, 0xff, sizeof(int) * (size_t)h->n * (size_t)k, st));
  k_multi_init<<<8 * h->num_sms, 256, 0, st>>>(m, W);
  k_multi_roots<<<(k + 255) / 256, 256, 0, st>>>(m, W, d_parent);
  int lgW = 0;
  while ((1 << lgW) < W) ++lgW;
  SS_CUDA(cudaGetLastError());
  if (d_parent) {  // the first frontier's edges (the roots' rows), for the parents pass
    SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
  }
  const IterLaunch il{policy, 0, 0};
  const long long max_iter = (long long)h->n + 2;
  for (long long it = 0;; ++it) {
    if (it > max_iter) {
      set_error("slimsell_bfs_multi: no convergence after %lld iterations", it);
      return SS_ERR_CUDA;
    }
    if (prof) SS_CUDA(cudaEventRecord(h->ev_a, st));
    s = launch_multi(h, m, W, policy == SS_V_SLIMWORK, il, st);
    if (s != SS_OK) return s;
    if (d_parent) {  // parents of the sources gained at this level
      // push from the previous frontier while the run grows and that frontier's
      // rows carry at most 1 / MULTI_PAR_PUSH_SHARE of the edges (the gaining
      // rows would have to search deep into their rows for it); once the
      // frontiers are dense or shrinking, the gaining rows find their parents
      // within a few neighbours and walk (measured on Kronecker 22, k = 64 ..
      // 1024: the push wins levels 1 and 2 by 7-70x, the walk every later level)
      const Ctl& hc = *h->h_ctl;  // counters read after the previous level
      const bool growing = hc.prev_new >= hc.prev2_new;
      if (growing && hc.prev_rowdeg * MULTI_PAR_PUSH_SHARE <= (unsigned long long)h->nnz) {
        SS_CUDA(cudaMemsetAsync(&h->ctl->units, 0, sizeof(unsigned long long), st));
        k_multi_par_expand<<<8 * h->num_sms, 256, 0, st>>>(m, (int)(it + 1));
        k_multi_par_scatter<<<8 * h->num_sms, 256, 0, st>>>(m, W, lgW, (int)(it + 1), d_parent);
      } else
        k_multi_parents<<<8 * h->num_sms, 256, 0, st>>>(m, W, lgW, (int)(it + 1), d_parent);
      SS_CUDA(cudaGetLastError());
    }
    if (prof) SS_CUDA(cudaEventRecord(h->ev_b, st));
    SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    if (prof) {
      float ms = 0.f;
      SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
      iter_ms += ms;
      h->iter_ns.push_back((int)(ms * 1.0e6f));
    }
    if (h->h_ctl->done) break;
  }
  if (prof) SS_CUDA(cudaEventRecord(h->ev_d, st));
  SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaEventRecord(h->ev_done, st));
  h->last.semiring = SS_BOOLEAN;
  h->last.iter_kernel_ms = iter_ms;
  h->last.total_ms = 0.0;
  h->pending = 1;
  ss_run_stats tmp;
  return slimsell_get_run_stats(h, &tmp, nullptr, 0);
}
