// Compacted-frontier push iteration on the SlimSell layout (the direction-
// optimising work avoidance that Section V calls orthogonal to SlimSell and
// implementable on top of it).  It computes exactly what the pull iteration
// computes -- new rows, their largest-id frontier neighbour, the real-semiring
// sum of frontier values -- by scattering from the frontier instead of
// gathering into every row:
//
//   k_push_expand   clears the touched map and turns each level-(k-1) vertex
//                   (read from the frontier bitmap) into work units of
//                   PUSH_UNIT neighbours;
//   k_push_scatter  one warp per unit reads the vertex's row (column-major, so
//                   with stride C) and, for every unvisited neighbour, folds in
//                   the parent by atomicMax, the real value by atomicAdd and a
//                   touched bit by atomicOr (reductions: no result is read);
//   k_push_post     walks the touched words: a touched word becomes the
//                   frontier word of level k (fb[k&1] held level k-2, which is
//                   overwritten), and each touched row gets level k, parent and
//                   value; the scratch is reset and the iteration tail runs.
#include <algorithm>
#include <climits>

#include "ss_device.cuh"

namespace ss {

constexpr int PUSH_UNIT = 256;
constexpr int PUSH_THREADS = 256;

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

__global__ void __launch_bounds__(PUSH_THREADS) k_push_expand(Dev d) {
  const Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long words = ((long long)d.n_pad + 31) / 32;
  for (long long w = t0; w < words; w += stride) d.touched[w] = 0u;
  const long long wstride = stride & ~31LL;  // whole warps walk the bitmap together
  const unsigned* fbm = d.fb[(k - 1) & 1];
  for (long long i0 = t0 - lane; i0 < words; i0 += wstride) {
    const long long i = i0 + lane;
    unsigned bits = i < words ? fbm[i] : 0u;
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

template <int SR, int C>
__global__ void __launch_bounds__(PUSH_THREADS) k_push_scatter(Dev d) {
  const Ctl* c = d.ctl;
  if (c->done) return;
  const long long nunits = min((long long)c->units, d.units_cap);
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_slots = 0;
  for (long long ui = wid; ui < nunits; ui += nw) {
    const int2 un = d.units[ui];
    const int u = un.x;
    const int deg = d.rdeg[u];
    const int chunk = u / C, l = u % C;
    const int* rowp = d.col + d.cs[chunk] + l;
    const int origu = __ldg(d.perm + u);
    const float val = (SR == SS_REAL) ? d.fr[u] : 0.0f;
    const int jend = min(un.y + PUSH_UNIT, deg);
    for (int j = un.y + lane; j < jend; j += 32) {
      const int v = __ldg(rowp + (long long)j * C);
      ++my_slots;
      if (d.lvl[v] == SS_INF) {
        // parents and touched bits only grow, so a stale read can only cause a
        // redundant atomic, never a missed one
        if (*(volatile const int*)(d.pbest + v) < origu) atomicMax(d.pbest + v, origu);
        if (SR == SS_REAL) atomicAdd(d.psum + v, val);
        const unsigned bit = 1u << (v & 31);
        if (!(*(volatile const unsigned*)(d.touched + (v >> 5)) & bit))
          atomicOr(d.touched + (v >> 5), bit);
      }
    }
  }
  __shared__ unsigned long long red[PUSH_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) my_slots += __shfl_down_sync(SS_FULL_MASK, my_slots, off);
  if (lane == 0) red[threadIdx.x >> 5] = my_slots;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < PUSH_THREADS / 32; ++w) s += red[w];
    if (s) atomicAdd(&d.ctl->slots, s);
  }
}

template <int SR>
__global__ void __launch_bounds__(PUSH_THREADS) k_push_post(Dev d, IterLaunch il) {
  const Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  unsigned* fbk = d.fb[k & 1];
  const long long words = ((long long)d.n_pad + 31) / 32;
  unsigned long long nw = 0, deg = 0;
  unsigned maxdeg = 0;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (long long)gridDim.x * blockDim.x) {
    unsigned bits = d.touched[w];
    fbk[w] = bits;  // f_k: exactly the rows first reached now
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int v = (int)(w * 32 + b);
      d.lvl[v] = k;
      d.par[v] = d.pbest[v] + 1;  // largest-id frontier neighbour + 1
      d.pbest[v] = -1;
      if (SR == SS_REAL) {
        d.fr[v] = d.psum[v];
        d.psum[v] = 0.0f;
      }
      const int dv = d.rdeg[v];
      ++nw;
      deg += (unsigned long long)dv;
      maxdeg = max(maxdeg, (unsigned)dv);
    }
  }
  finish_iteration_block<PUSH_THREADS>(d, nw, deg, 0ull, 0ull, maxdeg, il);
}

// ---------------------------------------------------------------------------
// Single-block push for small frontiers: one 1024-thread block runs level after
// level inside one launch (no kernel boundary, no bitmap walk per level).  The
// frontier is a vertex list held in shared memory together with what the
// scatter needs of each vertex (start of its column-major row, original id, the
// prefix sum of degrees), so that a level costs few dependent global round
// trips: the column loads, the level checks, one atomicMax per candidate edge
// (whose old value -1 marks the first discoverer, which appends the vertex),
// then one batch of loads in the post step.  Each thread takes a contiguous run
// of the level's edges (one binary search, then a forward walk).  The control
// block is worked on in shared memory and written back when the kernel ends.
// The block hands back to the iteration loop when the frontier outgrows
// LOCAL_MAX_FRONTIER vertices or LOCAL_MAX_EDGES edges, or after max_levels
// levels, leaving the frontier bitmaps and lists as the grid-wide variants
// and the next launch expect them:
//   fb[(k-1)&1] = level k-1, fb[k&1] = level k-2 (or zero),
//   qlist[(k-1)&1] = level k-1, qlist[k&1] = level k-2 (lengths in qlen).
// ---------------------------------------------------------------------------
constexpr int LOCAL_THREADS = 1024;
constexpr int LOCAL_BATCH = 16;                                  // edges per thread in flight
constexpr int LOCAL_PER_THREAD = LOCAL_MAX_FRONTIER / LOCAL_THREADS;  // frontier entries
constexpr int CTL_WORDS = (int)(sizeof(Ctl) / sizeof(unsigned));
static_assert(sizeof(Ctl) % sizeof(unsigned) == 0, "control block copied as words");
static_assert(LOCAL_MAX_FRONTIER % LOCAL_THREADS == 0, "whole frontier entries per thread");

struct LocalSmem {
  Ctl ctl;                               // working copy of the control block
  long long base[LOCAL_MAX_FRONTIER];    // cs[u / C] + u % C
  int ids[2][LOCAL_MAX_FRONTIER];        // frontier and next lists, by level parity
  int pref[LOCAL_MAX_FRONTIER];          // degrees, then their exclusive prefix
  int orig[LOCAL_MAX_FRONTIER];          // original id (the parent candidate)
  long long wsum[LOCAL_THREADS / 32];
  unsigned long long red[LOCAL_THREADS / 32];
  unsigned redmax[LOCAL_THREADS / 32];
  int nnew, stop;
};
static_assert(sizeof(LocalSmem) <= 227 * 1024, "single-block push shared memory");

// Entry from a bitmap state: list the level-(k-1) rows into qlist[(k-1)&1] and
// clear fb[k&1] (it held level k-2, which the single-block push does not list).
__global__ void __launch_bounds__(PUSH_THREADS) k_push_local_prep(Dev d) {
  Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  if (c->list_level == k - 1) return;  // the previous single-block level left its list
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long words = ((long long)d.n_pad + 31) / 32;
  const unsigned* fbm = d.fb[(k - 1) & 1];
  unsigned* fbk = d.fb[k & 1];
  int* list = d.qlist[(k - 1) & 1];
  for (long long i0 = t0 - lane; i0 < words; i0 += stride & ~31LL) {
    const long long i = i0 + lane;
    unsigned bits = 0u;
    if (i < words) {
      bits = fbm[i];
      fbk[i] = 0u;
    }
    while (__any_sync(SS_FULL_MASK, bits != 0u)) {
      int u = -1;
      if (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        u = (int)(i * 32 + b);
      }
      const unsigned m = __ballot_sync(SS_FULL_MASK, u >= 0);
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&c->qprep, (unsigned long long)__popc(m));
      base = __shfl_sync(SS_FULL_MASK, base, 0);
      if (u >= 0) list[base + __popc(m & ((1u << lane) - 1u))] = u;
    }
  }
}

// End the kernel: write the working control block back and set the loop
// condition (all threads call).
__device__ __forceinline__ void local_exit(LocalSmem& S, Ctl* c, const IterLaunch& il, unsigned cond) {
  __syncthreads();
  const unsigned* src = reinterpret_cast<const unsigned*>(&S.ctl);
  unsigned* dst = reinterpret_cast<unsigned*>(c);
  for (int i = threadIdx.x; i < CTL_WORDS; i += LOCAL_THREADS) dst[i] = src[i];
  if (threadIdx.x == 0 && il.use_cond) cudaGraphSetConditional(il.cond, cond);
}

// Row data of vertex u into frontier slot i.
template <int C>
__device__ __forceinline__ void local_stage(LocalSmem& S, const Dev& d, int i, int u, int deg) {
  S.pref[i] = deg;
  S.base[i] = __ldg(d.cs + u / C) + (u % C);
  S.orig[i] = __ldg(d.perm + u);
}

extern __shared__ __align__(16) unsigned char ss_local_smem[];

template <int SR, int C>
__global__ void __launch_bounds__(LOCAL_THREADS, 1) k_push_local(Dev d, IterLaunch il, int max_levels) {
  constexpr int BATCH = (SR == SS_REAL) ? LOCAL_BATCH / 2 : LOCAL_BATCH;  // registers
  LocalSmem& S = *reinterpret_cast<LocalSmem*>(ss_local_smem);
  Ctl* c = d.ctl;
  if (c->done) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(c);
    unsigned* dst = reinterpret_cast<unsigned*>(&S.ctl);
    for (int i = tid; i < CTL_WORDS; i += LOCAL_THREADS) dst[i] = src[i];
  }
  __syncthreads();
  int k = S.ctl.k;
  // the frontier list (level k-1): left by the previous launch, or just listed by
  // k_push_local_prep (which also cleared fb[k&1])
  const bool have_list = S.ctl.list_level == k - 1;
  int nf = (int)min(have_list ? S.ctl.qlen[(k - 1) & 1] : S.ctl.qprep, (unsigned long long)INT_MAX);
  if (nf > LOCAL_MAX_FRONTIER) {  // the decide kernel never sends a frontier this large
    if (tid == 0) {
      S.ctl.error |= 8;
      S.ctl.done = 1;
    }
    local_exit(S, c, il, 0u);
    return;
  }
  int cur = (k - 1) & 1;  // S.ids[cur] holds the frontier
  {
    const int* gl = d.qlist[(k - 1) & 1];
    for (int i = tid; i < nf; i += LOCAL_THREADS) {
      const int u = gl[i];
      S.ids[cur][i] = u;
      local_stage<C>(S, d, i, u, __ldg(d.rdeg + u));
    }
    // level k-2 words of fb[k&1], through the list the previous launch left
    const int n2 = (have_list && S.ctl.list_prev_ok) ? (int)S.ctl.qlen[k & 1] : 0;
    const int* g2 = d.qlist[k & 1];
    unsigned* fbk = d.fb[k & 1];
    for (int i = tid; i < n2; i += LOCAL_THREADS) fbk[g2[i] >> 5] = 0u;
  }
  if (tid == 0 && !have_list) S.ctl.qlen[(k - 1) & 1] = (unsigned long long)nf;
  __syncthreads();
  int clear_n = 0;  // level k-2 entries of S.ids[cur ^ 1] to clear (after the first level)
  for (int lev = 0;; ++lev) {
    const bool give_back = lev >= max_levels || nf > LOCAL_MAX_FRONTIER;
    long long E = 0;
    if (!give_back) {  // exclusive prefix of the frontier degrees, in place
      int dg[LOCAL_PER_THREAD];
      long long sum = 0;
#pragma unroll
      for (int q = 0; q < LOCAL_PER_THREAD; ++q) {
        const int i = tid * LOCAL_PER_THREAD + q;
        dg[q] = (i < nf) ? S.pref[i] : 0;
        sum += dg[q];
      }
      long long incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(SS_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) S.wsum[wid] = incl;
      if (tid == 0) S.nnew = 0;
      __syncthreads();
      if (wid == 0) {
        long long w = S.wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long t = __shfl_up_sync(SS_FULL_MASK, w, o);
          if (lane >= o) w += t;
        }
        S.wsum[lane] = w;
      }
      __syncthreads();
      E = S.wsum[LOCAL_THREADS / 32 - 1];
      if (E <= LOCAL_MAX_EDGES) {  // then every prefix fits in int
        long long run = (wid > 0 ? S.wsum[wid - 1] : 0LL) + incl - sum;
#pragma unroll
        for (int q = 0; q < LOCAL_PER_THREAD; ++q) {
          const int i = tid * LOCAL_PER_THREAD + q;
          if (i < nf) S.pref[i] = (int)run;
          run += dg[q];
        }
      }
    }
    const bool too_many = E > LOCAL_MAX_EDGES;
    if (give_back || (lev > 0 && too_many)) {  // hand the level-(k-1) list back
      if (tid == 0) {
        S.ctl.list_level = k - 1;
        S.ctl.list_prev_ok = 1;
      }
      local_exit(S, c, il, 1u);
      return;
    }
    if (too_many) {  // first level: the decide kernel never sends this many edges
      if (tid == 0) {
        S.ctl.error |= 8;
        S.ctl.done = 1;
      }
      local_exit(S, c, il, 0u);
      return;
    }
    const int nxt = cur ^ 1;
    unsigned* fbk = d.fb[k & 1];
    int* gnew = d.qlist[k & 1];
    for (int i = tid; i < clear_n; i += LOCAL_THREADS) fbk[S.ids[nxt][i] >> 5] = 0u;
    __syncthreads();  // prefix complete; the level k-2 list consumed
    // ---- scatter: each thread a contiguous run of at most BATCH edges per pass ----
    const int Ei = (int)E;
    for (int e0 = 0; e0 < Ei; e0 += LOCAL_THREADS * BATCH) {
      const int per = min(BATCH, (Ei - e0 + LOCAL_THREADS - 1) / LOCAL_THREADS);
      const int ea = e0 + tid * per;
      const int eb = min(ea + per, Ei);
      int i = 0;
      if (ea < eb) {  // largest i with pref[i] <= ea
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (S.pref[mid] <= ea) lo = mid;
          else hi = mid - 1;
        }
        i = lo;
      }
      int src[BATCH], v[BATCH];
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        const int e = ea + q;
        src[q] = -1;
        v[q] = -1;
        if (e < eb) {
          while (i + 1 < nf && S.pref[i + 1] <= e) ++i;
          src[q] = i;
          v[q] = __ldg(d.col + S.base[i] + (long long)(e - S.pref[i]) * C);
        }
      }
      // values written by this block earlier in the kernel are read past L1
      float fu[BATCH];
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        if (v[q] >= 0 && __ldcg(d.lvl + v[q]) != SS_INF) v[q] = -1;
        if (SR == SS_REAL) fu[q] = (v[q] >= 0) ? __ldcg(d.fr + S.ids[cur][src[q]]) : 0.0f;
      }
      // all atomics of the batch in flight before any result is used
      int old[BATCH];
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        old[q] = 0;
        if (v[q] >= 0) {
          if (SR == SS_REAL) atomicAdd(d.psum + v[q], fu[q]);
          old[q] = atomicMax(d.pbest + v[q], S.orig[src[q]]);
        }
      }
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        if (v[q] >= 0 && old[q] < 0) {  // first discoverer appends the vertex
          const int idx = atomicAdd(&S.nnew, 1);
          gnew[idx] = v[q];
          if (idx < LOCAL_MAX_FRONTIER) S.ids[nxt][idx] = v[q];
        }
      }
    }
    __syncthreads();
    // ---- post: the new level's rows, and their data for the next level ----
    const int nnew = S.nnew;
    unsigned long long nd = 0;
    unsigned md = 0;
    for (int i0 = 0; i0 < nnew; i0 += 4 * LOCAL_THREADS) {
      int vv[4], pb[4], dv[4], og[4];
      long long cs[4];
      float fv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * LOCAL_THREADS + tid;
        vv[q] = -1;
        if (i < nnew) vv[q] = (i < LOCAL_MAX_FRONTIER) ? S.ids[nxt][i] : __ldcg(gnew + i);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // every load of the batch before any store
        if (vv[q] >= 0) {
          pb[q] = __ldcg(d.pbest + vv[q]);
          dv[q] = __ldg(d.rdeg + vv[q]);
          cs[q] = __ldg(d.cs + vv[q] / C);
          og[q] = __ldg(d.perm + vv[q]);
          fv[q] = (SR == SS_REAL) ? __ldcg(d.psum + vv[q]) : 0.0f;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (vv[q] < 0) continue;
        const int x = vv[q];
        d.lvl[x] = k;
        d.par[x] = pb[q] + 1;  // largest-id frontier neighbour + 1
        d.pbest[x] = -1;
        if (SR == SS_REAL) {
          d.fr[x] = fv[q];
          d.psum[x] = 0.0f;
        }
        atomicOr(fbk + (x >> 5), 1u << (x & 31));
        nd += (unsigned long long)dv[q];
        md = max(md, (unsigned)dv[q]);
        const int i = i0 + q * LOCAL_THREADS + tid;
        if (i < LOCAL_MAX_FRONTIER) {
          S.pref[i] = dv[q];
          S.base[i] = cs[q] + (x % C);
          S.orig[i] = og[q];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nd += __shfl_down_sync(SS_FULL_MASK, nd, o);
    md = __reduce_max_sync(SS_FULL_MASK, md);
    if (lane == 0) {
      S.red[wid] = nd;
      S.redmax[wid] = md;
    }
    __syncthreads();
    if (tid == 0) {
      unsigned long long td = 0;
      unsigned tm = 0;
      for (int w = 0; w < LOCAL_THREADS / 32; ++w) {
        td += S.red[w];
        tm = max(tm, S.redmax[w]);
      }
      S.ctl.qlen[k & 1] = (unsigned long long)nnew;
      const bool stop = advance_level(d, &S.ctl, k, (unsigned long long)nnew, td,
                                      (unsigned long long)E, 0ull, tm, VAR_PUSH_LOCAL);
      S.ctl.list_level = k;
      S.ctl.list_prev_ok = 1;
      S.stop = stop ? 1 : 0;
    }
    __syncthreads();
    if (S.stop) {
      local_exit(S, c, il, 0u);
      return;
    }
    clear_n = nf;  // level k-1 is level (k+1)-2
    nf = nnew;
    cur = nxt;
    ++k;
  }
}

template <int SR, int C>
static ss_status launch_push_local_c(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                                     int max_levels, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    SS_CUDA(cudaFuncSetAttribute(k_push_local<SR, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(LocalSmem)));
    configured = true;
  }
  k_push_local_prep<<<vertex_grid(h, 32 * PUSH_THREADS), PUSH_THREADS, 0, st>>>(d);
  k_push_local<SR, C><<<1, LOCAL_THREADS, sizeof(LocalSmem), st>>>(d, il, max_levels);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

template <int SR>
static ss_status launch_push_local_sr(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                                      int max_levels, cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_push_local_c<SR, 8>(h, d, il, max_levels, st);
    case 16: return launch_push_local_c<SR, 16>(h, d, il, max_levels, st);
    case 32: return launch_push_local_c<SR, 32>(h, d, il, max_levels, st);
    default: return launch_push_local_c<SR, 64>(h, d, il, max_levels, st);
  }
}

ss_status launch_push_local(const slimsell_graph* h, const Dev& d, int sr, const IterLaunch& il,
                            int max_levels, cudaStream_t st) {
  switch (sr) {
    case SS_TROPICAL: return launch_push_local_sr<SS_TROPICAL>(h, d, il, max_levels, st);
    case SS_REAL: return launch_push_local_sr<SS_REAL>(h, d, il, max_levels, st);
    case SS_BOOLEAN: return launch_push_local_sr<SS_BOOLEAN>(h, d, il, max_levels, st);
    default: return launch_push_local_sr<SS_SELMAX>(h, d, il, max_levels, st);
  }
}

template <int SR, int C>
static ss_status launch_push_c(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                               cudaStream_t st) {
  // grids follow the graph size: bitmap words for expand/post, possible units for scatter
  const int gw = vertex_grid(h, 32 * PUSH_THREADS);
  const long long units = (long long)h->n_pad + h->nnz / PUSH_UNIT;
  const int gs = (int)std::max(1LL, std::min((long long)8 * h->num_sms, (units + 7) / 8));
  k_push_expand<<<gw, PUSH_THREADS, 0, st>>>(d);
  k_push_scatter<SR, C><<<gs, PUSH_THREADS, 0, st>>>(d);
  k_push_post<SR><<<gw, PUSH_THREADS, 0, st>>>(d, il);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

template <int SR>
static ss_status launch_push_sr(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                                cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_push_c<SR, 8>(h, d, il, st);
    case 16: return launch_push_c<SR, 16>(h, d, il, st);
    case 32: return launch_push_c<SR, 32>(h, d, il, st);
    default: return launch_push_c<SR, 64>(h, d, il, st);
  }
}

ss_status launch_push(const slimsell_graph* h, const Dev& d, int sr, const IterLaunch& il,
                      cudaStream_t st) {
  switch (sr) {
    case SS_TROPICAL: return launch_push_sr<SS_TROPICAL>(h, d, il, st);
    case SS_REAL: return launch_push_sr<SS_REAL>(h, d, il, st);
    case SS_BOOLEAN: return launch_push_sr<SS_BOOLEAN>(h, d, il, st);
    default: return launch_push_sr<SS_SELMAX>(h, d, il, st);
  }
}

}  // namespace ss
