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

#include <cooperative_groups.h>

#include "ss_device.cuh"

namespace ss {

namespace cg = cooperative_groups;

constexpr int PUSH_THREADS = 256;

// The frontier bits of one chunk (bit l = row l of the chunk) in a 64-bit word.
template <int C>
__device__ __forceinline__ unsigned long long chunk_bits(const unsigned* fb, long long chunk) {
  if (C == 8) return reinterpret_cast<const unsigned char*>(fb)[chunk];
  if (C == 16) return reinterpret_cast<const unsigned short*>(fb)[chunk];
  if (C == 32) return fb[chunk];
  const uint2 v = reinterpret_cast<const uint2*>(fb)[chunk];
  return ((unsigned long long)v.y << 32) | v.x;
}

// Emit the block units (chunk, first column) of chunk i, warp-aggregated; all
// lanes call, lanes with i < 0 emit nothing.
template <int C>
__device__ __forceinline__ void emit_block_units(const Dev& d, long long i, int lane) {
  constexpr int COLS = PUSH_BLOCK_SLOTS / C;
  const int cl = (i >= 0) ? d.cl[i] : 0;
  const unsigned nu = (unsigned)((cl + COLS - 1) / COLS);
  unsigned incl = nu;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(SS_FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned total = __shfl_sync(SS_FULL_MASK, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(&d.ctl->bunits, (unsigned long long)total);
  base = __shfl_sync(SS_FULL_MASK, base, 31);
  const unsigned long long first = base + incl - nu;
  if (first + nu > (unsigned long long)d.bunits_cap) {  // cannot happen: the capacity covers every chunk
    if (nu) atomicOr(&d.ctl->error, 2);
    return;
  }
  for (unsigned q = 0; q < nu; ++q) d.bunits[first + q] = make_int2((int)i, (int)(q * COLS));
}

// The frontier f_{k-1} as work: walked one chunk (one block of C rows, the
// layout's own block size) per lane.  With push_blocks on, a chunk whose block
// holds at least C/4 frontier rows (all non-empty blocks with push_blocks = 2)
// becomes block units that read whole columns of the chunk with coalesced
// loads, the block-sparse frontier; the rows of sparser blocks become vertex
// units that read one row each (stride C).  Also clears the touched map.
template <int C>
__global__ void __launch_bounds__(PUSH_THREADS) k_push_expand(Dev d) {
  const Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long words = ((long long)d.n_pad + 31) / 32;
  for (long long w = t0; w < words; w += stride) d.touched[w] = 0u;
  const long long wstride = stride & ~31LL;  // whole warps walk the chunks together
  const unsigned* fbm = d.fb[(k - 1) & 1];
  for (long long i0 = t0 - lane; i0 < d.n_c; i0 += wstride) {
    const long long i = i0 + lane;
    unsigned long long bits = i < d.n_c ? chunk_bits<C>(fbm, i) : 0ull;
    const int pc = __popcll(bits);
    const bool block = bits && (d.push_blocks == 2 || (d.push_blocks == 1 && pc >= C / 4));
    if (__any_sync(SS_FULL_MASK, block)) emit_block_units<C>(d, block ? i : -1, lane);
    if (block) bits = 0ull;
    while (__any_sync(SS_FULL_MASK, bits != 0ull)) {
      int u = -1;
      if (bits) {
        const int b = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        u = (int)(i * C + b);
      }
      emit_units(d, u, lane);
    }
  }
}

// Fold the frontier row (original id origu, real value val) into neighbour v
// when v is unvisited.
template <int SR>
__device__ __forceinline__ void push_fold(const Dev& d, int v, int origu, float val) {
  if (d.lvl[v] == SS_INF) {
    // parents and touched bits only grow, so a stale read can only cause a
    // redundant atomic, never a missed one
    if (*(volatile const int*)(d.pbest + v) < origu) atomicMax(d.pbest + v, origu);
    if (SR == SS_REAL) atomicAdd(d.psum + v, val);
    const unsigned bit = 1u << (v & 31);
    if (!(*(volatile const unsigned*)(d.touched + (v >> 5)) & bit)) atomicOr(d.touched + (v >> 5), bit);
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
      push_fold<SR>(d, v, origu, val);
    }
  }
  // block units: columns [j0, j0 + COLS) of a chunk whose frontier block is
  // dense, read as 16-byte quads (lane l meets rows 4 (l mod C/4) .. + 3 in
  // every column); only the block's frontier rows fold their neighbours in
  {
    constexpr int Q = C / 4;
    constexpr int COLS = PUSH_BLOCK_SLOTS / C;
    const long long nb = min((long long)c->bunits, d.bunits_cap);
    const unsigned* fbm = d.fb[(c->k - 1) & 1];
    const int lq = lane % Q;
    for (long long bi = wid; bi < nb; bi += nw) {
      const int2 un = d.bunits[bi];
      const long long chunk = un.x;
      const unsigned mb = (unsigned)(chunk_bits<C>(fbm, chunk) >> (4 * lq)) & 0xFu;
      const int ncols = min(COLS, d.cl[chunk] - un.y);
      if (lane == 0) my_slots += (unsigned long long)ncols * C;
      if (!mb) continue;  // none of this lane's rows is in the frontier
      const long long r0 = chunk * C + 4 * lq;
      int origs[4];
      float vals[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        origs[r] = (mb >> r & 1u) ? __ldg(d.perm + r0 + r) : -1;
        vals[r] = (SR == SS_REAL && (mb >> r & 1u)) ? d.fr[r0 + r] : 0.0f;
      }
      const int4* base = reinterpret_cast<const int4*>(d.col + d.cs[chunk] + (long long)un.y * C) + lq;
      for (int j = lane / Q; j < ncols; j += 32 / Q) {
        const int4 q = __ldcs(base + (long long)j * Q);
        const int cc[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if ((mb >> r & 1u) && cc[r] >= 0) push_fold<SR>(d, cc[r], origs[r], vals[r]);
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
      d.pbest[v] = SS_PBEST_VISITED;
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
// Cluster push for small frontiers: one thread-block cluster (16 CTAs of 1024
// threads where the device can place it, else 8) runs level after level inside
// one launch, with no kernel boundary and no bitmap walk per level.  The
// frontier is a vertex list; each CTA holds an equal share of it in shared
// memory with, per entry, what the scatter needs (start of the row's edges in
// col, edge count, original id).  The first level's share is loaded from the
// global list; later shares are written straight into the owning CTA's shared
// memory by the CTAs that discover the vertices (distributed shared memory),
// rows longer than LOCAL_UNIT edges being cut into units spread round-robin
// over the cluster.  Per level a CTA scatters over its share's edges (each
// thread a contiguous run: one binary search, then a forward walk) and claims
// each candidate with one atomicMax on its parent slot: the old value -1 makes
// this CTA the vertex's owner, visited vertices hold SS_PBEST_VISITED (no id
// is larger, so their slot never changes), and the slot ends with the largest
// id among the frontier neighbours, the parent.  Two hardware cluster barriers
// per level order the scatter before the post step (which reads the final
// parents) and the post step before the next level; per-CTA counts and
// statistics reach every CTA through distributed shared memory.  Spreading the
// random accesses over many SMs is what makes a level cheap: one SM's L1
// serves about one uncoalesced line per clock.  Every CTA keeps a copy of the
// control block in shared memory, updated identically from the cluster totals,
// so all CTAs take the same exits; CTA 0 writes it back at the end.
// The cluster hands back to the iteration loop when the frontier outgrows
// d.local_max_nf vertices or d.local_max_e edges, or after max_levels levels,
// leaving the bitmaps and lists as the grid-wide variants and the next launch
// expect them:
//   fb[(k-1)&1] = level k-1, fb[k&1] = level k-2 (or zero),
//   qlist/qdeg/qbase/qorig[(k-1)&1] = level k-1, qlist[k&1] = level k-2 (lengths in qlen).
// ---------------------------------------------------------------------------
constexpr int LOCAL_THREADS = 1024;
constexpr int LOCAL_BATCH = 16;     // candidate edges per thread in flight
constexpr int LOCAL_NEWCAP = 8192;  // new vertices per CTA kept in shared memory
constexpr int LOCAL_POST = 2;       // new vertices per thread in flight in the post step
constexpr int LOCAL_UNIT = 1024;    // edges of one slice entry; longer rows become several units
constexpr int LOCAL_HUBCAP = 256;   // extra slice entries per CTA for the units of long rows
constexpr int LOCAL_SLOTS = SS_LOCAL_SLICE + LOCAL_HUBCAP;
constexpr int LOCAL_PER_THREAD = (LOCAL_SLOTS + LOCAL_THREADS - 1) / LOCAL_THREADS;
constexpr int CTL_WORDS = (int)(sizeof(Ctl) / sizeof(unsigned));
static_assert(sizeof(Ctl) % sizeof(unsigned) == 0, "control block copied as words");
static_assert(SS_LOCAL_SLICE % LOCAL_THREADS == 0, "whole frontier entries per thread");
static_assert(SS_LOCAL_CLUSTER_MAX * SS_LOCAL_EDGES_PER_CTA / LOCAL_UNIT <= LOCAL_HUBCAP,
              "the units of the largest frontier fit one CTA");

struct LocalPub {             // what each CTA tells every CTA of the cluster about a level
  int nsm;                    // new vertices it holds in shared memory
  int novf;                   // new vertices it put in the overflow list
  unsigned md;                // largest degree of the vertices it posted
  int drop;                   // a unit of a long row found no room (the next level goes back)
  unsigned long long nd;      // their degree sum
};

// A CTA's slice of the frontier: entries 0 .. ns-1 are its equal share of the
// vertex list (each with at most LOCAL_UNIT of its edges), then `hubn` units
// carrying further LOCAL_UNIT-edge pieces of long rows, appended by any CTA.
struct LocalSmem {
  Ctl ctl;                             // this CTA's copy of the control block
  long long base[LOCAL_SLOTS];         // start of the entry's first edge in col
  int pref[LOCAL_SLOTS];               // edge counts, then their exclusive prefix
  int orig[LOCAL_SLOTS];               // original ids (parent candidates)
  int sid[2][LOCAL_SLOTS];             // vertex ids, by level parity
  int nid[LOCAL_NEWCAP];               // vertices this CTA discovered
  long long wsum[LOCAL_THREADS / 32];
  unsigned long long red[LOCAL_THREADS / 32];
  unsigned redmax[LOCAL_THREADS / 32];
  LocalPub all[2][SS_LOCAL_CLUSTER_MAX];  // written by every CTA of the cluster, by level parity
  int nnew, novf, es, hubn, drop;
};
static_assert(sizeof(LocalSmem) <= 227 * 1024, "cluster push shared memory");

// Entry from a bitmap state: list the level-(k-1) rows into qlist[(k-1)&1] and
// clear fb[k&1] (it held level k-2, which the cluster push does not list).
__global__ void __launch_bounds__(PUSH_THREADS) k_push_local_prep(Dev d) {
  Ctl* c = d.ctl;
  if (c->done) return;
  const int k = c->k;
  if (c->list_level == k - 1) return;  // the previous cluster-push level left its list
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
      // the decide kernel sends only frontiers that fit the list
      const unsigned long long at = base + __popc(m & ((1u << lane) - 1u));
      if (u >= 0 && at < (unsigned long long)d.n_pad) list[at] = u;
    }
  }
}

// End the kernel: no CTA leaves while another may still read its shared memory;
// CTA 0 writes its control block back and sets the loop condition.
__device__ __forceinline__ void local_exit(LocalSmem& S, Ctl* c, const IterLaunch& il, unsigned cond,
                                           cg::cluster_group& cl) {
  cl.sync();
  if (cl.block_rank() != 0) return;
  const unsigned* src = reinterpret_cast<const unsigned*>(&S.ctl);
  unsigned* dst = reinterpret_cast<unsigned*>(c);
  for (int i = threadIdx.x; i < CTL_WORDS; i += LOCAL_THREADS) dst[i] = src[i];
  if (threadIdx.x == 0 && il.use_cond) cudaGraphSetConditional(il.cond, cond);
}

// Entry `slot` of CTA `owner`'s slice (parity p) gets vertex x's first edges; the
// rest of a row longer than LOCAL_UNIT goes in LOCAL_UNIT-edge units to the
// following CTAs in turn, appended after their shares (ns_of(o) entries).
template <int C, typename NsOf>
__device__ __forceinline__ void place_entry(LocalSmem& S, cg::cluster_group& cl, int G, int owner, int slot,
                                            int p, int x, long long bx, int dv, int og, NsOf ns_of) {
  LocalSmem* R = cl.map_shared_rank(&S, owner);
  R->sid[p][slot] = x;
  R->pref[slot] = min(dv, LOCAL_UNIT);
  R->base[slot] = bx;
  R->orig[slot] = og;
  int o = owner;
  for (int j0 = LOCAL_UNIT; j0 < dv; j0 += LOCAL_UNIT) {
    o = (o + 1 == G) ? 0 : o + 1;
    LocalSmem* T = cl.map_shared_rank(&S, o);
    const int at = ns_of(o) + atomicAdd(&T->hubn, 1);
    if (at >= LOCAL_SLOTS) {  // no room: the cluster hands this level back instead
      S.drop = 1;
      continue;
    }
    T->sid[p][at] = x;
    T->pref[at] = min(dv - j0, LOCAL_UNIT);
    T->base[at] = bx + (long long)j0 * C;
    T->orig[at] = og;
  }
}

extern __shared__ __align__(16) unsigned char ss_local_smem[];

// CTA r's first entry of a list of `total` entries split into G = 2^lg equal
// shares (every list here has fewer than 2^27 entries, so 32 bits hold total * G).
__device__ __forceinline__ long long share(long long total, int r, int lg) {
  return (long long)(((unsigned)total * (unsigned)r) >> lg);
}

// The CTA whose share holds list entry `at` (0 <= at < total).
__device__ __forceinline__ int share_owner(long long at, long long total, int lg) {
  const int G = 1 << lg;
  int r = (int)(((unsigned)at << lg) / (unsigned)total);
  while (r + 1 < G && share(total, r + 1, lg) <= at) ++r;
  while (r > 0 && share(total, r, lg) > at) --r;
  return r;
}

// Selector features of the iterations after levels k0 .. k1 run in this launch
// (the decide kernel did not run before them), from the per-level totals the
// launch recorded; rank 0's threads, one level each, when the launch ends.
__device__ __forceinline__ void local_features(const Dev& d, LocalSmem& S, cg::cluster_group& cl, int k0,
                                               int k1) {
  __syncthreads();  // the last level's totals are in place
  if (cl.block_rank() != 0) return;
  for (int k = k0 + (int)threadIdx.x; k <= k1 && k + 1 < d.iter_cap; k += LOCAL_THREADS) {
    const unsigned long long* ls = d.lstat + (size_t)k * SS_LSTAT;
    float f[SS_SELECTOR_FEATURES];
    features_of(d, k + 1, ls[0], ls[1], ls[4], ls[5], (unsigned)ls[2], ls[6], f);
    store_features(d, k + 1, f);
  }
}

// One scatter pass of the cluster push: thread tid takes edges [ea, ea + per) of
// the slice (per <= B), finds their rows by one binary search and a forward walk,
// loads the neighbours, and claims each with one atomicMax (all B in flight
// before any result is used); one atomicMax both claims a vertex (old value -1),
// keeps the largest-id parent and tells visited vertices apart (their slot holds
// SS_PBEST_VISITED, which no id exceeds).
template <int SR, int C, int B>
__device__ __forceinline__ void local_scatter(const Dev& d, LocalSmem& S, int p0, int p1, int ns, int e0,
                                              int per, int Es, int tid) {
  const int* sid = S.sid[p1];
  const int ea = e0 + tid * per;
  const int eb = min(ea + per, Es);
  int i = 0;
  if (ea < eb) {  // largest i with pref[i] <= ea
    int lo_ = 0, hi_ = ns - 1;
    while (lo_ < hi_) {
      const int mid = (lo_ + hi_ + 1) >> 1;
      if (S.pref[mid] <= ea) lo_ = mid;
      else hi_ = mid - 1;
    }
    i = lo_;
  }
  int src[B], v[B];
  float fu[B];  // real semiring: the source's value, loaded with the neighbour
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int e = ea + q;
    src[q] = -1;
    v[q] = -1;
    fu[q] = 0.0f;
    if (e < eb) {
      while (i + 1 < ns && S.pref[i + 1] <= e) ++i;
      src[q] = i;
      v[q] = __ldg(d.col + S.base[i] + (long long)(e - S.pref[i]) * C);
      if (SR == SS_REAL) fu[q] = __ldcg(d.fr + sid[i]);  // written during this launch: past L1
    }
  }
  int old[B];
#pragma unroll
  for (int q = 0; q < B; ++q) {
    old[q] = SS_PBEST_VISITED;
    if (v[q] >= 0) old[q] = atomicMax(d.pbest + v[q], S.orig[src[q]]);
  }
  if (SR == SS_REAL) {
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (old[q] != SS_PBEST_VISITED) atomicAdd(d.psum + v[q], fu[q]);
  }
#pragma unroll
  for (int q = 0; q < B; ++q) {
    if (old[q] < 0) {  // first discoverer: this CTA owns the vertex
      const int idx = atomicAdd(&S.nnew, 1);
      if (idx < LOCAL_NEWCAP) {
        S.nid[idx] = v[q];
      } else {  // past this CTA's list (skewed slices): the shared overflow list
        atomicAdd(&S.novf, 1);
        const unsigned long long o = atomicAdd(d.qovf_n + p0, 1ull);
        if (o < (unsigned long long)SS_LOCAL_LIST_CAP) d.qovf[o] = v[q];
        else atomicOr(&S.ctl.error, 16);  // cannot happen: new vertices <= E <= cap
      }
    }
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int SR, int C>
__global__ void __launch_bounds__(LOCAL_THREADS, 1) k_push_local(Dev d, IterLaunch il, int max_levels,
                                                                 int time_levels) {
  constexpr int BATCH = (SR == SS_REAL) ? LOCAL_BATCH / 2 : LOCAL_BATCH;  // registers
  LocalSmem& S = *reinterpret_cast<LocalSmem*>(ss_local_smem);
  // per-level timing (profiling): the first level also carries the launch's entry
  unsigned long long t_prev = time_levels ? global_ns() : 0ull;
  cg::cluster_group cl = cg::this_cluster();
  const int G = (int)cl.num_blocks();  // 8 or 16
  const int lg = 31 - __clz(G);
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  Ctl* c = d.ctl;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(c);
    unsigned* dst = reinterpret_cast<unsigned*>(&S.ctl);
    for (int i = tid; i < CTL_WORDS; i += LOCAL_THREADS) dst[i] = src[i];
    if (rank == 0 && tid < 2) d.qovf_n[tid] = 0ull;
    if (tid == 0) {
      S.hubn = 0;
      S.drop = 0;
    }
  }
  cl.sync();  // every CTA holds its copy before CTA 0 can write the block back
  if (S.ctl.done) return;  // the same in every CTA; no shared memory was shared yet
  int k = S.ctl.k;
  const int k0 = k;  // first level of this launch (its features came from the decide kernel)
  const bool have_list = S.ctl.list_level == k - 1;
  long long nf = (long long)(have_list ? S.ctl.qlen[(k - 1) & 1] : S.ctl.qprep);
  long long E = (long long)S.ctl.prev_deg;  // edges of the level-(k-1) frontier
  if (!local_fits(d, (unsigned long long)nf, (unsigned long long)E)) {
    // the decide kernel never sends such a frontier
    if (tid == 0) {
      S.ctl.error |= 8;
      S.ctl.done = 1;
    }
    local_exit(S, c, il, 0u, cl);
    return;
  }
  if (tid == 0 && !have_list) S.ctl.qlen[(k - 1) & 1] = (unsigned long long)nf;
  // the first slice comes from the global list (its per-vertex data listed too, or
  // gathered), and the level k-2 words to clear from the list the previous launch
  // left; later slices arrive in shared memory from the CTAs that found them
  {
    const int p1 = (k - 1) & 1;
    const long long lo = share(nf, rank, lg);
    const int ns = (int)(share(nf, rank + 1, lg) - lo);
    auto ns_of = [&](int o) { return (int)(share(nf, o + 1, lg) - share(nf, o, lg)); };
    for (int i = tid; i < ns; i += LOCAL_THREADS) {
      const int u = __ldcg(d.qlist[p1] + lo + i);
      int dv, og;
      long long bx;
      if (have_list) {
        dv = __ldcg(d.qdeg[p1] + lo + i);
        bx = __ldcg(d.qbase[p1] + lo + i);
        og = __ldcg(d.qorig[p1] + lo + i);
      } else {
        dv = __ldg(d.rdeg + u);
        bx = __ldg(d.cs + u / C) + (u % C);
        og = __ldg(d.perm + u);
      }
      place_entry<C>(S, cl, G, rank, i, p1, u, bx, dv, og, ns_of);
    }
    const long long n2 = (have_list && S.ctl.list_prev_ok) ? (long long)S.ctl.qlen[k & 1] : 0;
    const long long lo2 = share(n2, rank, lg), hi2 = share(n2, rank + 1, lg);
    unsigned* fbk = d.fb[k & 1];
    for (long long i = lo2 + tid; i < hi2; i += LOCAL_THREADS) fbk[__ldcg(d.qlist[k & 1] + i) >> 5] = 0u;
  }
  cl.sync();  // the first slices, with the units of long rows, are in place
  int ns_prev = 0;  // entries of S.sid[k&1]: this CTA's slice of level k-2 (after the first level)
  unsigned long long reached = S.ctl.reached;  // every thread tracks the stop condition
  unsigned long long reached_deg = S.ctl.reached_deg;
  for (int lev = 0;; ++lev) {
    if (lev > 0 && (lev >= max_levels || !local_fits(d, (unsigned long long)nf, (unsigned long long)E))) {
      local_features(d, S, cl, k0, k - 1);
      if (tid == 0) {  // hand the level-(k-1) list back
        S.ctl.list_level = k - 1;
        S.ctl.list_prev_ok = 1;
      }
      local_exit(S, c, il, 1u, cl);
      return;
    }
    const int p1 = (k - 1) & 1, p0 = k & 1;
    unsigned* fbk = d.fb[p0];
    const int nsv = (int)(share(nf, rank + 1, lg) - share(nf, rank, lg));  // vertices
    const int ns = nsv + S.hubn;  // slice entries: vertices, then units of long rows
    for (int i = tid; i < ns_prev; i += LOCAL_THREADS) fbk[S.sid[p0][i] >> 5] = 0u;  // level k-2
    if (tid == 0) {
      S.nnew = 0;
      S.novf = 0;
    }
    // ---- exclusive prefix of the slice's degrees, in place (slice edges <= E <= d.local_max_e) ----
    if (ns <= 8 * 32) {  // small slice: one warp
      if (wid == 0) {
        int dg[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = lane * 8 + q;
          dg[q] = (i < ns) ? S.pref[i] : 0;
          sum += dg[q];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(SS_FULL_MASK, incl, o);
          if (lane >= o) incl += t;
        }
        int run = incl - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = lane * 8 + q;
          if (i < ns) S.pref[i] = run;
          run += dg[q];
        }
        if (lane == 31) S.es = incl;
      }
    } else {
      int dg[LOCAL_PER_THREAD], sum = 0;
#pragma unroll
      for (int q = 0; q < LOCAL_PER_THREAD; ++q) {
        const int i = tid * LOCAL_PER_THREAD + q;
        dg[q] = (i < ns) ? S.pref[i] : 0;
        sum += dg[q];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(SS_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) S.wsum[wid] = incl;
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
      int run = (wid > 0 ? (int)S.wsum[wid - 1] : 0) + incl - sum;
#pragma unroll
      for (int q = 0; q < LOCAL_PER_THREAD; ++q) {
        const int i = tid * LOCAL_PER_THREAD + q;
        if (i < ns) S.pref[i] = run;
        run += dg[q];
      }
      if (tid == LOCAL_THREADS - 1) S.es = (int)S.wsum[LOCAL_THREADS / 32 - 1];
    }
    __syncthreads();
    const int Es = S.es;
    // ---- scatter: each thread a contiguous run of at most BATCH edges per pass
    // (a 4-edge batch when that covers the slice: fewer idle unrolled steps) ----
    for (int e0 = 0; e0 < Es; e0 += LOCAL_THREADS * BATCH) {
      const int per = min(BATCH, (Es - e0 + LOCAL_THREADS - 1) / LOCAL_THREADS);
      if (per <= 4)
        local_scatter<SR, C, 4>(d, S, p0, p1, ns, e0, per, Es, tid);
      else
        local_scatter<SR, C, BATCH>(d, S, p0, p1, ns, e0, per, Es, tid);
    }
    __syncthreads();
    if (tid < G) {  // tell every CTA how many vertices this one found
      LocalPub* dst = &cl.map_shared_rank(&S, tid)->all[p0][rank];
      dst->nsm = min(S.nnew, LOCAL_NEWCAP);
      dst->novf = S.novf;
    }
    if (rank == 0 && tid == 0) d.qovf_n[p1] = 0ull;  // the next level's overflow counter
    if (tid == 0) {  // units for the next level are appended after this barrier
      S.hubn = 0;
      S.drop = 0;
    }
    cl.sync();  // #1: every scatter is done, so parents and sums are final
    // ---- list positions (every warp alike): this CTA's list, then its share of the overflow ----
    long long tot, novf, off;
    {
      const int nr = lane < G ? S.all[p0][lane].nsm : 0;
      const int vr = lane < G ? S.all[p0][lane].novf : 0;
      novf = (long long)__reduce_add_sync(SS_FULL_MASK, (unsigned)vr);
      const long long cntr = nr + (lane < G ? share(novf, lane + 1, lg) - share(novf, lane, lg) : 0);
      long long incl = cntr;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(SS_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
      }
      tot = __shfl_sync(SS_FULL_MASK, incl, 31);
      off = __shfl_sync(SS_FULL_MASK, incl - cntr, rank);
    }
    const int nsm = S.all[p0][rank].nsm;
    const long long olo = share(novf, rank, lg);
    const int cnt = nsm + (int)(share(novf, rank + 1, lg) - olo);
    // the next slices are filled only for a frontier the cluster will likely take:
    // past local_max_e / 4 vertices its edges almost surely outgrow the cluster
    const bool next_here = local_fits(d, (unsigned long long)tot, 0ull) && tot <= d.local_max_e / 4;
    // ---- post: level, parent, value, frontier bit and list record of each new vertex;
    // its data also goes straight to the CTA that takes it in the next level ----
    unsigned long long nd = 0;
    unsigned md = 0;
    for (int i0 = 0; i0 < cnt; i0 += LOCAL_POST * LOCAL_THREADS) {
      int vv[LOCAL_POST], pb[LOCAL_POST], dv[LOCAL_POST], og[LOCAL_POST];
      long long csv[LOCAL_POST];
      float fv[LOCAL_POST];
#pragma unroll
      for (int q = 0; q < LOCAL_POST; ++q) {
        const int i = i0 + q * LOCAL_THREADS + tid;
        vv[q] = -1;
        if (i < cnt) vv[q] = (i < nsm) ? S.nid[i] : __ldcg(d.qovf + olo + (i - nsm));
      }
#pragma unroll
      for (int q = 0; q < LOCAL_POST; ++q) {  // every load of the batch before any store
        if (vv[q] >= 0) {
          pb[q] = __ldcg(d.pbest + vv[q]);
          dv[q] = __ldg(d.rdeg + vv[q]);
          csv[q] = __ldg(d.cs + vv[q] / C);
          og[q] = __ldg(d.perm + vv[q]);
          fv[q] = (SR == SS_REAL) ? __ldcg(d.psum + vv[q]) : 0.0f;
        }
      }
#pragma unroll
      for (int q = 0; q < LOCAL_POST; ++q) {
        if (vv[q] < 0) continue;
        const int x = vv[q];
        d.lvl[x] = k;
        d.par[x] = pb[q] + 1;  // largest-id frontier neighbour + 1
        d.pbest[x] = SS_PBEST_VISITED;
        if (SR == SS_REAL) {
          d.fr[x] = fv[q];
          d.psum[x] = 0.0f;
        }
        atomicOr(fbk + (x >> 5), 1u << (x & 31));
        const long long at = off + i0 + q * LOCAL_THREADS + tid;
        const long long bx = csv[q] + (x % C);
        d.qlist[p0][at] = x;
        d.qdeg[p0][at] = dv[q];
        d.qbase[p0][at] = bx;
        d.qorig[p0][at] = og[q];
        if (next_here) {
          const int r = share_owner(at, tot, lg);
          place_entry<C>(S, cl, G, r, (int)(at - share(tot, r, lg)), p0, x, bx, dv[q], og[q],
                         [&](int o) { return (int)(share(tot, o + 1, lg) - share(tot, o, lg)); });
        }
        nd += (unsigned long long)dv[q];
        md = max(md, (unsigned)dv[q]);
      }
    }
    // this CTA's statistics, told to every CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nd += __shfl_down_sync(SS_FULL_MASK, nd, o);
    md = __reduce_max_sync(SS_FULL_MASK, md);
    if (lane == 0) {
      S.red[wid] = nd;
      S.redmax[wid] = md;
    }
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = S.red[lane];
      unsigned m = S.redmax[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(SS_FULL_MASK, w, o);
      m = __reduce_max_sync(SS_FULL_MASK, m);
      if (lane < G) {
        LocalPub* dst = &cl.map_shared_rank(&S, lane)->all[p0][rank];
        dst->nd = w;
        dst->md = m;
        dst->drop = S.drop;
      }
    }
    cl.sync();  // #2: every record, slice and statistic of level k is in place
    // ---- totals (every warp alike) and the stop decision ----
    unsigned long long td = lane < G ? S.all[p0][lane].nd : 0ull;
    unsigned tm = lane < G ? S.all[p0][lane].md : 0u;
    const bool dropped = __any_sync(SS_FULL_MASK, lane < G && S.all[p0][lane].drop != 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) td += __shfl_xor_sync(SS_FULL_MASK, td, o);
    tm = __reduce_max_sync(SS_FULL_MASK, tm);
    reached += (unsigned long long)tot;
    // the same decision advance_level takes on the control block
    const bool stop = tot == 0 || k >= d.n + 1 || reached > d.reach_cap;
    if (tid == 0) {
      S.ctl.qlen[p0] = (unsigned long long)tot;
      advance_level(d, &S.ctl, k, (unsigned long long)tot, td, (unsigned long long)E, 0ull, tm,
                    VAR_PUSH_LOCAL, rank == 0);
      S.ctl.list_level = k;
      S.ctl.list_prev_ok = 1;
      if (time_levels && rank == 0 && k < d.iter_cap) {  // device-side time of this level
        const unsigned long long t = global_ns();
        d.iters[k].kernel_ns = (int)min(t - t_prev, 2000000000ull);
        t_prev = t;
      }
    }
    reached_deg += td;
    if (rank == 0 && wid == LOCAL_THREADS / 32 - 1 && lane < 7 && k < d.iter_cap) {
      // the totals the next level's selector features come from (computed at exit)
      const unsigned long long v = lane == 0 ? (unsigned long long)tot : lane == 1 ? td
                                 : lane == 2 ? (unsigned long long)tm : lane == 3 ? (unsigned long long)E
                                 : lane == 4 ? reached : lane == 5 ? reached_deg : (unsigned long long)nf;
      d.lstat[(size_t)k * SS_LSTAT + lane] = v;
    }
    if (stop) {
      local_features(d, S, cl, k0, k - 1);
      local_exit(S, c, il, 0u, cl);
      return;
    }
    if (!next_here || dropped) {  // the next frontier does not fit: hand back before using it
      local_features(d, S, cl, k0, k);
      ++k;
      if (tid == 0) {
        S.ctl.list_level = k - 1;
        S.ctl.list_prev_ok = 1;
      }
      local_exit(S, c, il, 1u, cl);
      return;
    }
    ns_prev = nsv;  // this level's frontier is level (k+1)-2
    nf = tot;
    E = (long long)td;
    ++k;
  }
}


static int g_local_cluster[64];  // per device: 0 unknown, -1 none fits, else CTAs per cluster

int push_local_cluster_size() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (g_local_cluster[dev] != 0) return g_local_cluster[dev] > 0 ? g_local_cluster[dev] : 0;
  int best = -1;
  for (int G : {SS_LOCAL_CLUSTER_MAX, 8}) {
    auto kern = k_push_local<SS_TROPICAL, 32>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LocalSmem)) !=
        cudaSuccess)
      break;
    if (G > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(LOCAL_THREADS);
    cfg.dynamicSmemBytes = sizeof(LocalSmem);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) {
      best = G;
      break;
    }
  }
  cudaGetLastError();  // a refused size is not an error of a later call
  g_local_cluster[dev] = best;
  return best > 0 ? best : 0;
}

template <int SR, int C>
static ss_status launch_push_local_c(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                                     int max_levels, cudaStream_t st) {
  const int time_levels = h->profiling ? 1 : 0;
  static std::atomic<unsigned long long> configured{0};
  auto kern = k_push_local<SR, C>;
  if (first_on_device(configured)) {
    SS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LocalSmem)));
    SS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  k_push_local_prep<<<vertex_grid(h, 32 * PUSH_THREADS), PUSH_THREADS, 0, st>>>(d);
  SS_CUDA(cudaGetLastError());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d.local_cluster);
  cfg.blockDim = dim3(LOCAL_THREADS);
  cfg.dynamicSmemBytes = sizeof(LocalSmem);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = d.local_cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SS_CUDA(cudaLaunchKernelEx(&cfg, kern, d, il, max_levels, time_levels));
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
  k_push_expand<C><<<gw, PUSH_THREADS, 0, st>>>(d);
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
