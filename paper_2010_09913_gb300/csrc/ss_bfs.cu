// Single-source BFS-SpMV on SlimSell (Section III-A semirings, Section III-B
// SlimSell, Section III-C SlimWork, Section III-D SlimChunk, Section II-C DP).
//
// Vertex state lives in the relabelled row space of the layout:
//   lvl[r]      level of row r (SS_INF while unvisited); this is the distance
//               vector d and, for the tropical semiring, the vector f itself.
//   fb[k&1]     1-bit image of the frontier f_k (the rows that entered at level k),
//               double-buffered by level parity.  Every semiring's f_{k-1} is zero
//               outside this set, so x_k = A (x) f_{k-1} only needs the semiring
//               value of the neighbours whose bit is set:
//                 tropical  f^u + 1 = k          (f^u = k - 1 on the frontier; rows
//                                                 with non-frontier visited neighbours
//                                                 are visited themselves and keep f^v)
//                 boolean   1
//                 real      fr[u], the path count u carried into the frontier
//                 sel-max   id(u) + 1
//   fr[r]       real-semiring value of row r when it entered the frontier.
//   par[r]      parent original id + 1 (0 = none): sel-max p_k, or the DP parent.
//
// Neighbours are stored in descending original id, so the first frontier hit
// of a row (in column order) is its largest-id frontier neighbour: that is the
// sel-max value and, for the other semirings, the DP parent (Section II-C)
// computed on the fly; a separate DP pass after the iterations is also kept.
//
// The bitmap is gathered once per slot.  Random global gathers cost about one
// L1 cycle each, so each block first stages a prefix of the bitmap (the
// degree-sorted hubs, which receive most edges) in shared memory and reads
// the rest through the read-only path.
//
// One warp processes one work item (chunk i, columns [j0, j1)).  Each lane
// loads 16-byte quads of col: a quad is 4 consecutive rows of one column, so
// lane l always meets rows 4*(l mod C/4) .. +3; lanes sharing rows are combined
// with xor-shuffles.  Split chunks (SlimChunk) combine partial rows with
// atomics; the last item of a chunk to arrive runs the post-processing.
#include <algorithm>

#include "ss_device.cuh"

namespace ss {

// Compile-time tunables of the pull kernel (defaults measured best on GB300).
#ifndef SS_PULL_STEP
#define SS_PULL_STEP 4
#endif
#ifndef SS_PULL_STEP_REAL
#define SS_PULL_STEP_REAL 3  // the real semiring also gathers a value per hit
#endif
#ifndef SS_PULL_STEP_SELL
#define SS_PULL_STEP_SELL 2  // Sell-C-sigma loads a value quad beside each column quad
#endif
#ifndef SS_PULL_PREFETCH
#define SS_PULL_PREFETCH 0  // bulk L2 prefetch distance beyond the next step (0: next step only)
#endif
#ifndef SS_PULL_LOAD
#define SS_PULL_LOAD 2  // col loads: 0 evict-first, 1 no-L1 with 256-byte L2 fetches, 2 no-L1
#endif

constexpr int PULL_THREADS = SS_PULL_THREADS;  // one block per SM
#ifndef SS_PULL_SHORT_COLS
#define SS_PULL_SHORT_COLS 4
#endif
constexpr int SHORT_COLS = SS_PULL_SHORT_COLS;  // chunks this short go several per warp

// int4 col loads in flight per lane (4 slots each)
template <int SR, int FMT>
__host__ __device__ constexpr int pull_step() {
  return FMT == SS_FORMAT_SELL ? SS_PULL_STEP_SELL : (SR == SS_REAL ? SS_PULL_STEP_REAL : SS_PULL_STEP);
}
// Bits of the semiring's zero, the value of a Sell-C-sigma padding slot.
template <int SR>
__host__ __device__ constexpr int sell_zero_bits() { return SR == SS_TROPICAL ? 0x7f800000 : 0; }

// A Sell-C-sigma quad read: the slots whose value is the semiring's zero are no
// edges (padding, column 0) and become -1, so the scan treats them as SlimSell
// padding; the values stay in v for the real semiring's multiply.
template <int SR>
__device__ __forceinline__ int4 sell_edges(int4 c, int4 v) {
  constexpr int Z = sell_zero_bits<SR>();
  return make_int4(v.x == Z ? -1 : c.x, v.y == Z ? -1 : c.y, v.z == Z ? -1 : c.z, v.w == Z ? -1 : c.w);
}
// Stage the bitmap prefix only when the previous iteration read at least this
// many slots; below it, reading frontier bits from global memory is cheaper.
constexpr unsigned long long STAGE_MIN_SLOTS = 2ull << 20;

enum { MODE_FULL = 0, MODE_SLIMWORK = 1, MODE_FILTERED = 3 };

// Real semiring: a level whose frontier's degree sum exceeds nnz / HUB_EDGE_SHARE
// stages the values of the HUB_VALUE_ROWS highest-degree rows (64 KB) in shared
// memory, where most of its value gathers land (the top 16 K rows of a
// Kronecker graph of scale 22 receive 40 % of all edge endpoints).
#ifndef SS_HUB_VALUE_ROWS
#define SS_HUB_VALUE_ROWS 16384
#endif
constexpr int HUB_VALUE_ROWS = SS_HUB_VALUE_ROWS;
constexpr unsigned long long HUB_EDGE_SHARE = 16;

__device__ __forceinline__ int4 ld_stream(const int4* p) {
#if SS_PULL_LOAD == 1
  int4 v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
#elif SS_PULL_LOAD == 2
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
#else
  return __ldcs(p);
#endif
}

// Ask the TMA unit to pull [p, p + bytes) into L2 ahead of the warp's loads
// (p 16-byte aligned, bytes a positive multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  if (bytes == 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

constexpr int PREFETCH_BYTES = SS_PULL_PREFETCH;  // col bytes prefetched ahead of each warp

__device__ __forceinline__ int4 shfl_int4(int4 v, int src) {
  return make_int4(__shfl_sync(SS_FULL_MASK, v.x, src), __shfl_sync(SS_FULL_MASK, v.y, src),
                   __shfl_sync(SS_FULL_MASK, v.z, src), __shfl_sync(SS_FULL_MASK, v.w, src));
}

// Shared-memory image of the bitmap: SMEM_GUARD zero words, then the staged
// prefix.  The padding marker c = -1 has c >> 5 = -1 and lands on the last guard
// word, so it needs no branch; vertices past the prefix read the global bitmap.
constexpr int SMEM_GUARD = 4;

__device__ __forceinline__ unsigned frontier_bit(const unsigned* smw, int sbits, const unsigned* gbm,
                                                 int c) {
  const int wi = c >> 5;
  const unsigned w = (c < sbits) ? smw[wi] : __ldg(gbm + wi);
  return (w >> (c & 31)) & 1u;
}

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
  unsigned maxdeg = 0;
};

// Per-row result of one item: best = largest original id among frontier
// neighbours (-1 if none) and, for the real semiring, the sum of their values.
struct RowAcc {
  int best[4];
  float sum[4];
};

// Post-process one chunk (the frontier update of Section III-A): new rows are
// the unvisited rows whose x_k is non-zero; they get level k, a parent and a
// frontier bit; the chunk's SlimWork state is refreshed.  All lanes call.
//
// GROUPED: the warp holds 32 / Q chunks at once, lanes g*Q .. g*Q+Q-1 owning all
// rows of chunk g (own = this lane's group has a chunk); otherwise lanes 0..Q-1
// own the rows of the warp's one chunk.
template <int SR, int C, bool GROUPED = false>
__device__ __forceinline__ void post_chunk(const Dev& d, int k, int chunk, int lane, int4 lv,
                                           const RowAcc& a, Counters& cnt, bool own = true) {
  constexpr int Q = C / 4;
  const int lq = GROUPED ? lane % Q : lane;
  const bool owner = GROUPED ? own : lane < Q;
  const int R0 = chunk * C + 4 * lq;
  unsigned nib = 0, left = 0;
  if (owner) {
    int L[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool unvisited = (L[r] == SS_INF);
      // x_k is non-zero exactly where a row has a frontier neighbour (the real
      // semiring's values are positive path counts), so every semiring tests the hit
      const bool found = a.best[r] >= 0;
      if (unvisited && found) nib |= 1u << r;
      else if (unvisited) left = 1;
    }
    if (nib) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (nib >> r & 1u) {
          L[r] = k;
          d.par[R0 + r] = a.best[r] + 1;  // p_k = p_{k-1} + not(p_{k-1}) (.) x_k / DP parent
          if (SR == SS_REAL) d.fr[R0 + r] = a.sum[r];
        }
      *reinterpret_cast<int4*>(d.lvl + R0) = make_int4(L[0], L[1], L[2], L[3]);
      // the push variants tell visited vertices apart by their pbest slot
      *reinterpret_cast<int4*>(d.pbest + R0) =
          make_int4(L[0] == SS_INF ? -1 : SS_PBEST_VISITED, L[1] == SS_INF ? -1 : SS_PBEST_VISITED,
                    L[2] == SS_INF ? -1 : SS_PBEST_VISITED, L[3] == SS_INF ? -1 : SS_PBEST_VISITED);
      const int4 dg = *reinterpret_cast<const int4*>(d.rdeg + R0);
      const int D[4] = {dg.x, dg.y, dg.z, dg.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (nib >> r & 1u) {
          cnt.deg += (unsigned long long)D[r];
          cnt.maxdeg = max(cnt.maxdeg, (unsigned)D[r]);
        }
      cnt.nw += __popc(nib);
    }
  }
  unsigned lo, hi, any_left;
  if (GROUPED) {  // OR within each group of Q lanes
    lo = (C <= 32 || lq < 8) ? nib << (4 * (lq & 7)) : 0u;
    hi = (C > 32 && lq >= 8) ? nib << (4 * (lq - 8)) : 0u;
    any_left = left;
#pragma unroll
    for (int o = 1; o < Q; o <<= 1) {
      lo |= __shfl_xor_sync(SS_FULL_MASK, lo, o);
      if (C > 32) hi |= __shfl_xor_sync(SS_FULL_MASK, hi, o);
      any_left |= __shfl_xor_sync(SS_FULL_MASK, any_left, o);
    }
  } else {
    gather_bits<C>(nib, lane, &lo, &hi);
    any_left = __any_sync(SS_FULL_MASK, left);
  }
  if (owner && lq == 0) {
    store_bits<C>(d.fb[k & 1], chunk, lo, hi);
    d.act[chunk] = any_left ? 1 : 3;
  }
}

// A skipped chunk (SlimWork) has only final rows, so f_k is zero there; its bits
// in the parity buffer are cleared for the two iterations after its last
// discovery (states 3 and 2), then left alone (state 0).
template <int C>
__device__ __forceinline__ void carry_chunk(const Dev& d, int k, int chunk, int lane, int a) {
  if (a < 2) return;
  if (lane == 0) {
    store_bits<C>(d.fb[k & 1], chunk, 0u, 0u);
    d.act[chunk] = (a == 3) ? 2 : 0;
  }
}

// Scan the slots of one quad: record the first frontier hit per row and, for
// the real semiring, add the values of all hits.
// live: bit r set while row r is unvisited.  Visited rows keep their value, so
// the real semiring gathers frontier values for live rows only, and only in a
// branch taken when a live row of the quad was hit (the full passes of the first
// levels see almost no hits).  Values of rows below sf come from the copy staged
// in shared memory (smf), the others from global memory.  (Skipping the bit
// lookups of rows already hit, for the other semirings, measured slower: the
// predicated lookups cost more issue slots than they save.)
//
// Sell-C-sigma (FMT = SS_FORMAT_SELL): the caller has turned the quad's padding
// into -1 (sell_edges), and the real semiring multiplies the gathered value by
// the slot's matrix value v.  The real semiring over SlimSell takes quad_hits
// and gather_step instead, which gather a whole step's values at once.
template <int SR, int FMT>
__device__ __forceinline__ void scan_quad(const Dev& d, const unsigned* sm, int sbits,
                                          const unsigned* gbm, int4 c, int4 v, int first[4], float sum[4],
                                          unsigned live, const float* smf, int sf) {
  const int cc[4] = {c.x, c.y, c.z, c.w};
  const int vv[4] = {v.x, v.y, v.z, v.w};
  unsigned hit[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) hit[r] = frontier_bit(sm, sbits, gbm, cc[r]);
#pragma unroll
  for (int r = 0; r < 4; ++r) first[r] = (hit[r] && first[r] < 0) ? cc[r] : first[r];
  if (SR == SS_REAL) {
    const unsigned m = (hit[0] | (hit[1] << 1) | (hit[2] << 2) | (hit[3] << 3)) & live;
    if (m) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (m >> r & 1u) {
          const float x = (cc[r] < sf) ? smf[cc[r]] : __ldg(d.fr + cc[r]);
          sum[r] += (FMT == SS_FORMAT_SELL) ? __int_as_float(vv[r]) * x : x;
        }
    }
  }
}


// Real semiring, SlimSell: the frontier hits of one quad (bit r for row r) and
// the first-hit update; the value gathers follow for the whole step at once.
__device__ __forceinline__ unsigned quad_hits(const unsigned* sm, int sbits, const unsigned* gbm, int4 c,
                                              int first[4]) {
  const int cc[4] = {c.x, c.y, c.z, c.w};
  unsigned m = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const unsigned h = frontier_bit(sm, sbits, gbm, cc[r]);
    first[r] = (h && first[r] < 0) ? cc[r] : first[r];
    m |= h << r;
  }
  return m;
}

// Gather and add the values of every live hit of a step's U quads: all loads are
// issued before the first add, so a warp waits once per step, not once per quad
// (Kronecker 22 hub level: 322 -> 278 us; the gathers are latency-bound, and
// staging more hub rows as 8- or 16-bit counts measured no faster).
template <int U>
__device__ __forceinline__ void gather_step(const Dev& d, const int4* c, const unsigned* mm, float sum[4],
                                            const float* smf, int sf) {
  unsigned any = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) any |= mm[u];
  if (!any) return;
  float x[U][4];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int cc[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float v = 0.f;
      if (mm[u] >> r & 1u) v = (cc[r] < sf) ? smf[cc[r]] : __ldg(d.fr + cc[r]);
      x[u][r] = v;
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) sum[r] += x[u][r];
}

extern __shared__ __align__(16) unsigned ss_smem_bits[];

// One frontier expansion x_k = A (x)_S f_{k-1} with fused post-processing.
// Warp w of the grid owns items w, w + W, w + 2W, ... (W = warps in the grid,
// the item list is ordered for that assignment); it reads the descriptors and
// SlimWork states of 32 of them at once (one per lane) and walks the active ones.
template <int SR, int C, int MODE, int FMT>
__global__ void __launch_bounds__(PULL_THREADS, 1) k_pull(Dev d, int variant,
                                                          cudaGraphConditionalHandle cond,
                                                          int use_cond) {
  constexpr int PULL_STEP = pull_step<SR, FMT>();
  const int* colp = (FMT == SS_FORMAT_SELL) ? d.scol : d.col;
  constexpr int Q = C / 4;
  if (d.ctl->done) return;
  const int k = d.ctl->k;
  const int km1 = k - 1;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (PULL_THREADS / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (PULL_THREADS / 32);
  const unsigned* gbm = d.fb[km1 & 1];
  // stage the bitmap prefix of f_{k-1} with asynchronous 16-byte copies
  const int pv = d.ctl->prev_variant;
  const bool light = (pv == VAR_FULL || pv == VAR_SLIMWORK || pv == VAR_FILTERED) &&
                     d.ctl->prev_slots < STAGE_MIN_SLOTS;
  const int sw_all = light ? 0 : d.smem_words;
  // real semiring on a level whose frontier carries a large share of the edges
  // (the hub level of a skewed graph): the last sf words of the staging area
  // hold the values fr of the sf highest-degree rows instead of bitmap words
  const bool hub = SR == SS_REAL && (unsigned long long)d.ctl->prev_deg * HUB_EDGE_SHARE >
                                        (unsigned long long)d.nnz;
  const int sf = hub ? min(HUB_VALUE_ROWS, (sw_all >> 1) & ~3) : 0;
  const int sw = sw_all - sf;  // bitmap words staged (a multiple of 4)
  {
    if (threadIdx.x < SMEM_GUARD) ss_smem_bits[threadIdx.x] = 0u;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(ss_smem_bits + SMEM_GUARD);
    for (int i = threadIdx.x; i < (sw >> 2); i += PULL_THREADS)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbase + 16u * (unsigned)i),
                   "l"(reinterpret_cast<const int4*>(gbm) + i)
                   : "memory");
    const unsigned fbase = sbase + 4u * (unsigned)sw;
    for (int i = threadIdx.x; i < (sf >> 2); i += PULL_THREADS)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(fbase + 16u * (unsigned)i),
                   "l"(reinterpret_cast<const int4*>(d.fr) + i)
                   : "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();
  const unsigned* sm = ss_smem_bits + SMEM_GUARD;
  const float* smf = reinterpret_cast<const float*>(sm + sw);
  const int sbits = sw * 32;
  Counters cnt;
  unsigned long long lane_slots = 0;
  for (long long b0 = wid; b0 < d.n_items; b0 += 32LL * nw) {
    const long long my_it = b0 + (long long)lane * nw;
    int4 my_item = make_int4(0, 0, 0, -1);
    long long my_start = 0;
    int a = 0;
    if (my_it < d.n_items) {
      my_item = d.items[my_it];
      a = (MODE == MODE_FULL) ? 1 : d.act[my_item.x];
      my_start = d.cs[my_item.x] + (long long)my_item.y * C;
    }
    unsigned todo = __ballot_sync(SS_FULL_MASK, a == 1);
    if (MODE != MODE_FULL) {
      unsigned carry = __ballot_sync(SS_FULL_MASK, a >= 2 && my_item.y == 0);
      while (carry) {
        const int src = __ffs(carry) - 1;
        carry &= carry - 1;
        carry_chunk<C>(d, k, __shfl_sync(SS_FULL_MASK, my_item.x, src), lane,
                       __shfl_sync(SS_FULL_MASK, a, src));
      }
    }
    // short whole chunks (at most SHORT_COLS columns, about half of all chunks of a
    // skewed graph) go 32 / Q at a time, one group of Q lanes each
    unsigned shortm = __ballot_sync(SS_FULL_MASK, a == 1 && my_item.w < 0 &&
                                                      my_item.z - my_item.y <= SHORT_COLS);
    todo &= ~shortm;
    while (shortm) {
      constexpr int GROUPS = 32 / Q;
      int mysrc = -1;
#pragma unroll
      for (int g = 0; g < GROUPS; ++g) {
        const int sidx = shortm ? __ffs(shortm) - 1 : -1;
        if (lane / Q == g) mysrc = sidx;
        shortm &= shortm - 1;
      }
      const bool own = mysrc >= 0;
      const int sl = own ? mysrc : 0;
      const int4 item = make_int4(__shfl_sync(SS_FULL_MASK, my_item.x, sl),
                                  __shfl_sync(SS_FULL_MASK, my_item.y, sl),
                                  __shfl_sync(SS_FULL_MASK, my_item.z, sl), -1);
      const long long start = __shfl_sync(SS_FULL_MASK, my_start, sl);
      const int lq = lane % Q;
      const int ncols = own ? item.z - item.y : 0;
      const int chunk = item.x;
      const int4 lv = own ? *reinterpret_cast<const int4*>(d.lvl + chunk * C + 4 * lq)
                          : make_int4(SS_PAD_LEVEL, SS_PAD_LEVEL, SS_PAD_LEVEL, SS_PAD_LEVEL);
      const int L[4] = {lv.x, lv.y, lv.z, lv.w};
      const unsigned live = (L[0] == SS_INF ? 1u : 0u) | (L[1] == SS_INF ? 2u : 0u) |
                            (L[2] == SS_INF ? 4u : 0u) | (L[3] == SS_INF ? 8u : 0u);
      int first[4] = {-1, -1, -1, -1};
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      const int4* base = reinterpret_cast<const int4*>(colp + start) + lq;
      const int4* vbase = reinterpret_cast<const int4*>(d.sval + start) + lq;  // (Sell only)
      int4 c[SHORT_COLS], v[SHORT_COLS];
#pragma unroll
      for (int u = 0; u < SHORT_COLS; ++u) {
        c[u] = (u < ncols) ? ld_stream(base + u * Q) : make_int4(-1, -1, -1, -1);
        if (FMT == SS_FORMAT_SELL) {
          const int4 vq = (u < ncols) ? ld_stream(vbase + u * Q) : make_int4(0, 0, 0, 0);
          c[u] = sell_edges<SR>(c[u], vq);
          v[u] = SR == SS_REAL ? vq : make_int4(0, 0, 0, 0);
        } else {
          v[u] = make_int4(0, 0, 0, 0);
        }
      }
      if constexpr (SR == SS_REAL && FMT == SS_FORMAT_SLIMSELL) {
        unsigned mm[SHORT_COLS];
#pragma unroll
        for (int u = 0; u < SHORT_COLS; ++u)
          mm[u] = (u < ncols) ? quad_hits(sm, sbits, gbm, c[u], first) & live : 0u;
        gather_step<SHORT_COLS>(d, c, mm, sum, smf, sf);
      } else {
#pragma unroll
        for (int u = 0; u < SHORT_COLS; ++u)
          if (u < ncols) scan_quad<SR, FMT>(d, sm, sbits, gbm, c[u], v[u], first, sum, live, smf, sf);
      }
      if (own && lq == 0) {
        cnt.act += 1;
        if (MODE != MODE_FILTERED) cnt.slots += (unsigned long long)ncols * C;
      }
      if (MODE == MODE_FILTERED) lane_slots += 4ull * ncols;
      RowAcc acc;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc.best[r] = (first[r] >= 0 && L[r] == SS_INF) ? __ldg(d.perm + first[r]) : -1;
        acc.sum[r] = sum[r];
      }
      post_chunk<SR, C, true>(d, k, chunk, lane, lv, acc, cnt, own);
    }
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int4 item = shfl_int4(my_item, src);
      const long long start = __shfl_sync(SS_FULL_MASK, my_start, src);
      const int chunk = item.x;
      // L2 prefetch: the head of this item beyond the first step, and of the next item
      if (lane == src) {
        const unsigned bytes = (unsigned)(item.z - item.y) * C * 4u;
        if (bytes > 2048u)
          prefetch_l2(colp + start + 512, min(bytes - 2048u, (unsigned)PREFETCH_BYTES));
      }
      if (todo) {
        const int nxt = __ffs(todo) - 1;
        if (lane == nxt) {
          const unsigned bytes = (unsigned)(my_item.z - my_item.y) * C * 4u;
          prefetch_l2(colp + my_start, min(bytes, (unsigned)PREFETCH_BYTES));
        }
      }
      // levels of this lane's 4 rows (prefetched; only this chunk's post writes them)
      const int4 lv = *reinterpret_cast<const int4*>(d.lvl + chunk * C + 4 * (lane % Q));
      const int L[4] = {lv.x, lv.y, lv.z, lv.w};
      const unsigned live = (L[0] == SS_INF ? 1u : 0u) | (L[1] == SS_INF ? 2u : 0u) |
                            (L[2] == SS_INF ? 4u : 0u) | (L[3] == SS_INF ? 8u : 0u);
      int first[4] = {-1, -1, -1, -1};
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      bool need = true;
      if (MODE == MODE_FILTERED) {  // only unvisited rows are computed
        need = false;
#pragma unroll
        for (int r = 0; r < 4; ++r) need |= (L[r] == SS_INF);
      }
      const int nq = (item.z - item.y) * Q;
      const int4* base = reinterpret_cast<const int4*>(colp + start);
      const int4* vbase = reinterpret_cast<const int4*>(d.sval + start);  // (Sell only)
      for (int q0 = 0; q0 < nq; q0 += 32 * PULL_STEP) {
        if (MODE == MODE_FILTERED) {
          if (!__any_sync(SS_FULL_MASK, need)) break;
          if (!need) continue;
        }
        // keep the prefetch PREFETCH_BYTES ahead inside long items (one lane issues it)
        if (lane == 0) {
          const long long ahead = (long long)(q0 + 32 * PULL_STEP) * 16 + PREFETCH_BYTES;
          const long long total = (long long)nq * 16;
          if (ahead < total) {
            prefetch_l2(reinterpret_cast<const char*>(base) + ahead,
                        (unsigned)min(total - ahead, (long long)(32 * PULL_STEP * 16)));
            if (FMT == SS_FORMAT_SELL)
              prefetch_l2(reinterpret_cast<const char*>(vbase) + ahead,
                          (unsigned)min(total - ahead, (long long)(32 * PULL_STEP * 16)));
          }
        }
        int4 c[PULL_STEP], v[PULL_STEP];
#pragma unroll
        for (int u = 0; u < PULL_STEP; ++u) {
          const int q = q0 + lane + 32 * u;
          c[u] = (q < nq) ? ld_stream(base + q) : make_int4(-1, -1, -1, -1);
          if (FMT == SS_FORMAT_SELL) {
            const int4 vq = (q < nq) ? ld_stream(vbase + q) : make_int4(0, 0, 0, 0);
            c[u] = sell_edges<SR>(c[u], vq);
            v[u] = SR == SS_REAL ? vq : make_int4(0, 0, 0, 0);
          } else {
            v[u] = make_int4(0, 0, 0, 0);
          }
          if (MODE == MODE_FILTERED && q < nq) lane_slots += 4;
        }
        if constexpr (SR == SS_REAL && FMT == SS_FORMAT_SLIMSELL) {
          unsigned mm[PULL_STEP];
#pragma unroll
          for (int u = 0; u < PULL_STEP; ++u)
            mm[u] = (q0 + 32 * u < nq) ? quad_hits(sm, sbits, gbm, c[u], first) & live : 0u;
          gather_step<PULL_STEP>(d, c, mm, sum, smf, sf);
        } else {
#pragma unroll
          for (int u = 0; u < PULL_STEP; ++u)  // (q0 + 32 u < nq is warp-uniform)
            if (q0 + 32 * u < nq) scan_quad<SR, FMT>(d, sm, sbits, gbm, c[u], v[u], first, sum, live, smf, sf);
        }
        if (MODE == MODE_FILTERED) {  // a row is done once visited or (not real) hit
          need = false;
#pragma unroll
          for (int r = 0; r < 4; ++r)
            need |= (L[r] == SS_INF) && (SR == SS_REAL || first[r] < 0);
        }
      }
      if (MODE != MODE_FILTERED && lane == 0) cnt.slots += (unsigned long long)(item.z - item.y) * C;
      // the largest original id among this lane's first hits of unvisited rows
      RowAcc acc;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc.best[r] = (first[r] >= 0 && L[r] == SS_INF) ? __ldg(d.perm + first[r]) : -1;
        acc.sum[r] = sum[r];
      }
      // (a non-zero real sum implies a hit on a live row of the same lane)
      const bool any_hit = (acc.best[0] >= 0) | (acc.best[1] >= 0) | (acc.best[2] >= 0) |
                           (acc.best[3] >= 0);
      if (__any_sync(SS_FULL_MASK, any_hit)) {  // lanes with equal lane mod Q share rows
#pragma unroll
        for (int off = Q; off < 32; off <<= 1)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            acc.best[r] = max(acc.best[r], __shfl_xor_sync(SS_FULL_MASK, acc.best[r], off));
            if (SR == SS_REAL) acc.sum[r] += __shfl_xor_sync(SS_FULL_MASK, acc.sum[r], off);
          }
      }
      if (item.w >= 0) {  // SlimChunk: combine partial rows, the last arriving item post-processes
        const size_t xo = (size_t)item.w * C + 4 * lane;
        if (lane < Q) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if (acc.best[r] >= 0) atomicMax(d.xpar + xo + r, acc.best[r]);
            if (SR == SS_REAL && acc.sum[r] != 0.0f) atomicAdd(d.xacc + xo + r, acc.sum[r]);
          }
          __threadfence();
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          const unsigned old = atomicAdd(d.arrive + item.w, 1u);
          last = (old == (unsigned)d.split_n[item.w] - 1u);
        }
        last = __shfl_sync(SS_FULL_MASK, last, 0);
        if (!last) continue;
        __threadfence();
        if (lane < Q) {
          // one 16-byte read and reset per array (xo is a multiple of 4 and the
          // scratch 16-byte aligned); the per-row scalar form of this rarely run
          // block made the whole real-semiring kernel 20-25 % slower on GB300
          const int4 b4 = __ldcg(reinterpret_cast<const int4*>(d.xpar + xo));
          *reinterpret_cast<int4*>(d.xpar + xo) = make_int4(-1, -1, -1, -1);
          acc.best[0] = b4.x; acc.best[1] = b4.y; acc.best[2] = b4.z; acc.best[3] = b4.w;
          if (SR == SS_REAL) {
            const float4 s4 = __ldcg(reinterpret_cast<const float4*>(d.xacc + xo));
            *reinterpret_cast<float4*>(d.xacc + xo) = make_float4(0.f, 0.f, 0.f, 0.f);
            acc.sum[0] = s4.x; acc.sum[1] = s4.y; acc.sum[2] = s4.z; acc.sum[3] = s4.w;
          }
        }
        if (lane == 0) d.arrive[item.w] = 0u;
      }
      if (lane == 0) cnt.act += 1;
      post_chunk<SR, C>(d, k, chunk, lane, lv, acc, cnt);
    }
  }
  if (MODE == MODE_FILTERED) cnt.slots = lane_slots;
  finish_iteration_block<PULL_THREADS>(d, cnt.nw, cnt.deg, cnt.slots, cnt.act, cnt.maxdeg,
                                       IterLaunch{variant, cond, use_cond});
}

__global__ void k_init(Dev d) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long r = t0; r < d.n_pad; r += stride) d.lvl[r] = r < d.n ? SS_INF : SS_PAD_LEVEL;
  for (long long w = t0; w < d.fb_words; w += stride) {
    d.fb[0][w] = 0u;
    d.fb[1][w] = 0u;
  }
  for (long long i = t0; i < d.n_c; i += stride) d.act[i] = 1;
  for (long long s = t0; s < (long long)d.n_split * d.C; s += stride) {
    d.xacc[s] = 0.0f;
    d.xpar[s] = -1;
  }
  for (long long r = t0; r < d.n_pad; r += stride) d.pbest[r] = -1;  // nothing visited
  if (d.ctl->error) {  // a previous run stopped early: restore the push scratch invariant
    for (long long r = t0; r < d.n_pad; r += stride) d.psum[r] = 0.0f;
  }
}

__global__ void k_init_root(Dev d, int root) { init_root_state(d, root); }

// DP transformation as a separate pass (Section II-C): the parent of a row at
// level L >= 1 is its largest-id neighbour at level L-1.  Neighbours are stored
// in descending original id, so each lane's first hit in its column sequence is
// that lane's maximum; lanes stop once their rows are resolved.
template <int C>
__global__ void __launch_bounds__(PULL_THREADS, 1) k_dp(Dev d) {
  constexpr int Q = C / 4;
  constexpr int PULL_STEP = SS_PULL_STEP;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (PULL_THREADS / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (PULL_THREADS / 32);
  unsigned long long my_slots = 0;
  for (long long b0 = wid; b0 < d.n_items; b0 += 32LL * nw) {
    const long long my_it = b0 + (long long)lane * nw;
    int4 my_item = make_int4(0, 0, 0, -1);
    long long my_start = 0;
    if (my_it < d.n_items) {
      my_item = d.items[my_it];
      my_start = d.cs[my_item.x] + (long long)my_item.y * C;
    }
    unsigned todo = __ballot_sync(SS_FULL_MASK, my_it < d.n_items);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int4 item = shfl_int4(my_item, src);
      const long long start = __shfl_sync(SS_FULL_MASK, my_start, src);
      const int chunk = item.x;
      const int R0 = chunk * C + 4 * (lane % Q);
      const int4 lv = *reinterpret_cast<const int4*>(d.lvl + R0);
      int tgt[4] = {lv.x, lv.y, lv.z, lv.w};
      int hit[4];
      bool need = false;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        tgt[r] = (tgt[r] >= 1 && tgt[r] != SS_INF) ? tgt[r] - 1 : -2;
        hit[r] = -1;
        need |= tgt[r] >= 0;
      }
      const int nq = (item.z - item.y) * Q;
      const int4* base = reinterpret_cast<const int4*>(d.col + start);
      for (int q0 = 0; q0 < nq && __any_sync(SS_FULL_MASK, need); q0 += 32 * PULL_STEP) {
        if (!need) continue;
        int4 c[PULL_STEP];
#pragma unroll
        for (int u = 0; u < PULL_STEP; ++u) {
          const int q = q0 + lane + 32 * u;
          c[u] = (q < nq) ? ld_stream(base + q) : make_int4(-1, -1, -1, -1);
          if (q < nq) my_slots += 4;
        }
        int Lv[PULL_STEP][4];
#pragma unroll
        for (int u = 0; u < PULL_STEP; ++u) {
          Lv[u][0] = d.lvl[max(c[u].x, 0)];
          Lv[u][1] = d.lvl[max(c[u].y, 0)];
          Lv[u][2] = d.lvl[max(c[u].z, 0)];
          Lv[u][3] = d.lvl[max(c[u].w, 0)];
        }
        need = false;
#pragma unroll
        for (int u = 0; u < PULL_STEP; ++u) {
          const int cc[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (hit[r] < 0 && tgt[r] >= 0 && cc[r] >= 0 && Lv[u][r] == tgt[r]) hit[r] = cc[r];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) need |= (tgt[r] >= 0 && hit[r] < 0);
      }
      int best[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) best[r] = hit[r] >= 0 ? d.perm[hit[r]] : -1;
#pragma unroll
      for (int off = Q; off < 32; off <<= 1)
#pragma unroll
        for (int r = 0; r < 4; ++r) best[r] = max(best[r], __shfl_xor_sync(SS_FULL_MASK, best[r], off));
      if (lane < Q) {
        if (item.w < 0) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (tgt[r] >= 0) d.par[R0 + r] = best[r] + 1;
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (best[r] >= 0) atomicMax(d.par + R0 + r, best[r] + 1);
        }
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

// Rows of split chunks start the DP pass at "no parent" (they combine by atomicMax).
__global__ void k_dp_clear(Dev d) {
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < d.n_items;
       it += (long long)gridDim.x * blockDim.x) {
    const int4 item = d.items[it];
    if (item.w >= 0 && item.y == 0)
      for (int l = 0; l < d.C; ++l)
        if (d.lvl[item.x * d.C + l] >= 1) d.par[item.x * d.C + l] = 0;
  }
}

__global__ void k_output(Dev d, int* dist, int* parent) { write_outputs(d, dist, parent); }

// Real-semiring values f of the last run in original vertex order; rows the run
// did not reach hold stale values and read as 0.
__global__ void k_values(Dev d, float* out) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < d.n;
       v += (long long)gridDim.x * blockDim.x) {
    const int r = d.invperm[v];
    out[v] = (d.lvl[r] == SS_INF) ? 0.0f : d.fr[r];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// One 1024-thread block per SM, fewer for small work lists (about 128 items
// per block), so that several small graphs can share the GPU.
int pull_grid(const slimsell_graph* h) {
  const long long want = ((long long)h->n_items + 127) / 128;
  return (int)std::max(1LL, std::min((long long)h->num_sms, want));
}

int vertex_grid(const slimsell_graph* h, int threads) {
  const long long want = ((long long)h->n_pad + threads - 1) / threads;
  return (int)std::max(1LL, std::min((long long)8 * h->num_sms, want));
}

template <int SR, int C, int MODE, int FMT>
static ss_status launch_pull(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                             cudaStream_t st) {
  static std::atomic<unsigned long long> configured{0};
  if (first_on_device(configured))
    SS_CUDA(cudaFuncSetAttribute(k_pull<SR, C, MODE, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SS_SMEM_LIMIT_BYTES));
  k_pull<SR, C, MODE, FMT><<<pull_grid(h), PULL_THREADS, (size_t)(d.smem_words + SMEM_GUARD) * 4, st>>>(
      d, il.variant, il.cond, il.use_cond);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

template <int SR, int MODE, int FMT>
static ss_status launch_pull_c(const slimsell_graph* h, const Dev& d, const IterLaunch& il,
                               cudaStream_t st) {
  switch (h->C) {
    case 8: return launch_pull<SR, 8, MODE, FMT>(h, d, il, st);
    case 16: return launch_pull<SR, 16, MODE, FMT>(h, d, il, st);
    case 32: return launch_pull<SR, 32, MODE, FMT>(h, d, il, st);
    default: return launch_pull<SR, 64, MODE, FMT>(h, d, il, st);
  }
}

// The Sell-C-sigma format is instantiated for the full and SlimWork passes only
// (slimsell_bfs accepts it with those policies).
template <int SR>
static ss_status launch_pull_m(const slimsell_graph* h, const Dev& d, int mode, const IterLaunch& il,
                               cudaStream_t st) {
  const bool sell = d.format == SS_FORMAT_SELL;
  switch (mode) {
    case MODE_FULL:
      return sell ? launch_pull_c<SR, MODE_FULL, SS_FORMAT_SELL>(h, d, il, st)
                  : launch_pull_c<SR, MODE_FULL, SS_FORMAT_SLIMSELL>(h, d, il, st);
    case MODE_SLIMWORK:
      return sell ? launch_pull_c<SR, MODE_SLIMWORK, SS_FORMAT_SELL>(h, d, il, st)
                  : launch_pull_c<SR, MODE_SLIMWORK, SS_FORMAT_SLIMSELL>(h, d, il, st);
    default:
      return launch_pull_c<SR, MODE_FILTERED, SS_FORMAT_SLIMSELL>(h, d, il, st);
  }
}

static ss_status launch_iteration(const slimsell_graph* h, const Dev& d, int sr, int mode,
                                  const IterLaunch& il, cudaStream_t st) {
  switch (sr) {
    case SS_TROPICAL: return launch_pull_m<SS_TROPICAL>(h, d, mode, il, st);
    case SS_REAL: return launch_pull_m<SS_REAL>(h, d, mode, il, st);
    case SS_BOOLEAN: return launch_pull_m<SS_BOOLEAN>(h, d, mode, il, st);
    default: return launch_pull_m<SS_SELMAX>(h, d, mode, il, st);
  }
}

// Queue the kernels of one iteration of the given variant.  The cluster push
// runs as many small levels as it can per launch (under profiling it times each
// level on the device).
static ss_status launch_variant(const slimsell_graph* h, const Dev& d, int sr, int variant,
                                const IterLaunch& il, cudaStream_t st) {
  switch (variant) {
    case VAR_FULL: return launch_iteration(h, d, sr, MODE_FULL, il, st);
    case VAR_SLIMWORK: return launch_iteration(h, d, sr, MODE_SLIMWORK, il, st);
    case VAR_PUSH: return launch_push(h, d, sr, il, st);
    case VAR_PUSH_LOCAL:
      return launch_push_local(h, d, sr, il, 1 << 30, st);
    default: return launch_iteration(h, d, sr, MODE_FILTERED, il, st);
  }
}

// Policies that choose the variant on the device before every iteration.
static bool adaptive(int policy) {
  return policy == SS_V_PUSH || policy == SS_V_HEURISTIC || policy == SS_V_LEARNED;
}

// Capture the kernels of one variant into graph g (a conditional body).
#ifndef SS_LOOP_UNROLL
#define SS_LOOP_UNROLL 3
#endif

static ss_status capture_into(slimsell_graph* h, const Dev& d, int sr, int variant,
                              const IterLaunch& il, cudaGraph_t g, int reps = 1) {
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    if (cs) cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
  }
  ss_status s = SS_OK;
  for (int i = 0; i < reps && s == SS_OK; ++i) s = launch_variant(h, d, sr, variant, il, cs);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (s != SS_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  return SS_OK;
}

// Add one device-side iteration loop to graph g after the given dependencies:
// a conditional WHILE node whose body is the fixed variant's kernels, or (adaptive
// policies) the decide kernel followed by a conditional SWITCH over the five
// executed variants.  The last block of each iteration's final kernel (or the
// single-block push, when it stops or hands back) sets the WHILE condition.
ss_status add_loop_node(slimsell_graph* h, const Dev& d, int sr, int policy, cudaGraph_t g,
                        const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* out) {
  cudaGraphConditionalHandle cw;
  cudaGraphNodeParams wp = {};
  cudaError_t e = cudaGraphConditionalHandleCreate(&cw, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = cw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    e = cudaGraphAddNode(out, g, deps, nullptr, ndeps, &wp);
  }
  if (e != cudaSuccess) return cuda_fail(e, "conditional WHILE node");
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  // a fixed variant's body holds SS_LOOP_UNROLL iterations: one more than the
  // run needs returns at once (every kernel checks the done flag first) and
  // leaves the WHILE condition as the finishing iteration set it; three per body
  // measured 2.3 % faster per Kronecker 22 BFS than one (fewer conditional trips)
  if (!adaptive(policy)) return capture_into(h, d, sr, policy, IterLaunch{policy, cw, 1}, body, SS_LOOP_UNROLL);
  cudaGraphConditionalHandle csw;
  cudaGraphNode_t dnode, snode;
  cudaGraphNodeParams sp = {};
  e = cudaGraphConditionalHandleCreate(&csw, body, 0, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphConditionalHandleCreate(switch)");
  ss_status s = add_decide_node(h, d, policy, csw, cw, body, &dnode);
  if (s != SS_OK) return s;
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = csw;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = N_VARIANTS;
  e = cudaGraphAddNode(&snode, body, &dnode, nullptr, 1, &sp);
  if (e != cudaSuccess) return cuda_fail(e, "conditional SWITCH node");
  for (int v = 0; v < N_VARIANTS && s == SS_OK; ++v)
    s = capture_into(h, d, sr, v, IterLaunch{v, cw, 1}, sp.conditional.phGraph_out[v]);
  return s;
}

void drop_loop_graphs(slimsell_graph* h) {
  for (auto& row : h->loop_exec)
    for (auto& e : row)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
}

// The single-call loop graph, built once per (semiring, policy, staged-prefix
// size) and cached in the handle.
static ss_status loop_graph(slimsell_graph* h, const Dev& d, int sr, int policy,
                            cudaGraphExec_t* out) {
  cudaGraphExec_t& slot = h->loop_exec[sr][policy];
  if (slot && h->loop_smem_words[sr][policy] == d.smem_words) {
    *out = slot;
    return SS_OK;
  }
  if (slot) {
    SS_CUDA(cudaGraphExecDestroy(slot));
    slot = nullptr;
  }
  cudaGraph_t g = nullptr;
  SS_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphNode_t wnode;
  ss_status s = add_loop_node(h, d, sr, policy, g, nullptr, 0, &wnode);
  if (s == SS_OK) {
    cudaError_t e = cudaGraphInstantiate(&slot, g, 0);
    if (e != cudaSuccess) {
      slot = nullptr;
      s = cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  cudaGraphDestroy(g);
  if (s != SS_OK) return s;
  h->loop_smem_words[sr][policy] = d.smem_words;
  *out = slot;
  return SS_OK;
}

template <int C>
static ss_status launch_dp_c(const slimsell_graph* h, const Dev& d, cudaStream_t st) {
  k_dp<C><<<h->num_sms, PULL_THREADS, 0, st>>>(d);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

static ss_status launch_dp(const slimsell_graph* h, const Dev& d, cudaStream_t st) {
  k_dp_clear<<<4 * h->num_sms, 256, 0, st>>>(d);
  SS_CUDA(cudaGetLastError());
  switch (h->C) {
    case 8: return launch_dp_c<8>(h, d, st);
    case 16: return launch_dp_c<16>(h, d, st);
    case 32: return launch_dp_c<32>(h, d, st);
    default: return launch_dp_c<64>(h, d, st);
  }
}

}  // namespace ss

namespace ss {
// Read back the counters of the last call once its work has finished.
static ss_status finish_run(slimsell_graph* h) {
  if (!h->pending) return SS_OK;
  SS_CUDA(cudaEventSynchronize(h->ev_done));
  h->pending = 0;
  const Ctl& c = *h->h_ctl;
  h->last.iterations = c.k - 1;
  h->last.reached = (long long)c.reached;
  h->last.reached_degree = (long long)c.reached_deg;
  h->last.slots = (long long)c.total_slots;
  h->last.dp_slots = (long long)c.dp_slots;
  if (h->profiling) {
    float ms = 0.f;
    SS_CUDA(cudaEventElapsedTime(&ms, h->ev_c, h->ev_d));
    h->last.total_ms = ms;
  }
  if (c.error) {
    set_error("slimsell_bfs: iteration limit reached (device error flags %d)", c.error);
    return SS_ERR_CUDA;
  }
  return SS_OK;
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
  if (h->format == SS_FORMAT_SELL && policy != SS_V_FULL && policy != SS_V_SLIMWORK) {
    set_error("slimsell_bfs: the Sell-C-sigma format runs the FULL and SLIMWORK policies only");
    return SS_ERR_UNSUPPORTED;
  }
  h->values_semiring = -1;  // set again once this run is queued
  cudaStream_t st = (cudaStream_t)stream;
  if (h->format == SS_FORMAT_SELL && !h->sell_col) {
    if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
    ss_status s = sell_arrays(h, st);
    if (s != SS_OK) return s;
  }
  Dev d = h->dev();
  if (h->format == SS_FORMAT_SELL) {
    d.format = SS_FORMAT_SELL;
    d.scol = h->sell_col;
    d.sval = semiring == SS_TROPICAL ? h->sell_vtrop : h->sell_vmul;
  }
  const int grid = vertex_grid(h, 256);
  const bool prof = h->profiling != 0;
  const bool device_loop = h->device_loop && !prof;
  // the previous call's statistics are dropped without waiting for it: its work is
  // ahead of this call's on the same stream (the handle's contract), and a host
  // wait here left the GPU idle between back-to-back runs
  h->pending = 0;
  h->iter_ns.clear();
  double iter_ms = 0.0;
  if (prof) SS_CUDA(cudaEventRecord(h->ev_c, st));

  k_init<<<grid, 256, 0, st>>>(d);
  k_init_root<<<1, 1, 0, st>>>(d, root);
  SS_CUDA(cudaGetLastError());

  if (device_loop) {
    cudaGraphExec_t exec = nullptr;
    ss_status s = loop_graph(h, d, semiring, policy, &exec);
    if (s != SS_OK) return s;
    SS_CUDA(cudaGraphLaunch(exec, st));
  } else if (!adaptive(policy) && h->profile_queue) {
    // fixed variant: iterations are queued QUEUE_BATCH at a time, each launch
    // bracketed by its own event pair when profiling, and the host reads the
    // counter once per batch; launches queued past the end of the run return
    // at once (every kernel checks the done flag) and their times are dropped
    constexpr int QUEUE_BATCH = 8;
    if (prof && h->evq.size() < 2 * (size_t)QUEUE_BATCH) {
      while (h->evq.size() < 2 * (size_t)QUEUE_BATCH) {
        cudaEvent_t e = nullptr;
        SS_CUDA(cudaEventCreate(&e));
        h->evq.push_back(e);
      }
    }
    const long long max_iter = (long long)h->n + 2;
    for (long long it = 0;;) {
      if (it > max_iter) {
        set_error("slimsell_bfs: no convergence after %lld iterations", it);
        return SS_ERR_CUDA;
      }
      for (int j = 0; j < QUEUE_BATCH; ++j) {
        ss_status s = launch_decide(h, d, policy, 0, 0, st);  // logs the iteration's features
        if (s != SS_OK) return s;
        if (prof) SS_CUDA(cudaEventRecord(h->evq[2 * j], st));
        s = launch_variant(h, d, semiring, policy, IterLaunch{policy, 0, 0}, st);
        if (s != SS_OK) return s;
        if (prof) SS_CUDA(cudaEventRecord(h->evq[2 * j + 1], st));
      }
      SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      SS_CUDA(cudaStreamSynchronize(st));
      const long long ran = (long long)h->h_ctl->k - 1;  // iterations the run has made so far
      if (prof)
        for (int j = 0; j < QUEUE_BATCH && it + j < ran; ++j) {
          float ms = 0.f;
          SS_CUDA(cudaEventElapsedTime(&ms, h->evq[2 * j], h->evq[2 * j + 1]));
          iter_ms += ms;
          h->iter_ns.push_back((int)(ms * 1.0e6f));
        }
      it += QUEUE_BATCH;
      if (h->h_ctl->done) break;
    }
  } else {
    const long long max_iter = (long long)h->n + 2;
    for (long long it = 0;; ++it) {
      if (it > max_iter) {
        set_error("slimsell_bfs: no convergence after %lld iterations", it);
        return SS_ERR_CUDA;
      }
      // the decide kernel logs the iteration's features; adaptive policies read its choice
      ss_status s = launch_decide(h, d, policy, 0, 0, st);
      if (s != SS_OK) return s;
      int variant = policy;
      if (adaptive(policy)) {
        SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        SS_CUDA(cudaStreamSynchronize(st));
        variant = h->h_ctl->variant;
      }
      const int k_before = h->h_ctl->k;  // valid when the cluster push is chosen (adaptive)
      if (prof) SS_CUDA(cudaEventRecord(h->ev_a, st));
      s = launch_variant(h, d, semiring, variant, IterLaunch{variant, 0, 0}, st);
      if (s != SS_OK) return s;
      if (prof) SS_CUDA(cudaEventRecord(h->ev_b, st));
      SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      SS_CUDA(cudaStreamSynchronize(st));
      if (prof) {
        float ms = 0.f;
        SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
        iter_ms += ms;
        h->iter_ns.push_back((int)(ms * 1.0e6f));
        // levels run inside one cluster-push launch were timed on the device;
        // slimsell_get_run_stats takes them from there (marker -1)
        if (variant == VAR_PUSH_LOCAL)  // (k_before is fresh: adaptive policies read ctl above)
          for (int extra = h->h_ctl->k - k_before - 1; extra > 0; --extra) h->iter_ns.push_back(-1);
      }
      if (h->h_ctl->done) break;
    }
  }

  if (d_parent && semiring != SS_SELMAX && h->dp_pass) {
    ss_status s = launch_dp(h, d, st);
    if (s != SS_OK) return s;
  }
  if (d_dist || d_parent) {
    k_output<<<grid, 256, 0, st>>>(d, d_dist, d_parent);
    SS_CUDA(cudaGetLastError());
  }
  if (prof) SS_CUDA(cudaEventRecord(h->ev_d, st));
  SS_CUDA(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaEventRecord(h->ev_done, st));
  h->last.semiring = semiring;
  h->values_semiring = semiring;
  h->last.iter_kernel_ms = iter_ms;
  h->last.total_ms = 0.0;
  h->pending = 1;
  if (!device_loop) return finish_run(h);
  return SS_OK;
}

ss_status slimsell_get_values(slimsell_handle h, float* d_out, void* stream) {
  using namespace ss;
  set_error("");
  if (!h || !d_out) {
    set_error("slimsell_get_values: NULL argument");
    return SS_ERR_INVALID;
  }
  if (h->values_semiring != SS_REAL) {
    set_error("slimsell_get_values: the handle's last run was not a real-semiring slimsell_bfs");
    return SS_ERR_INVALID;
  }
  const Dev d = h->dev();
  k_values<<<vertex_grid(h, 256), 256, 0, (cudaStream_t)stream>>>(d, d_out);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

ss_status slimsell_get_run_stats(slimsell_handle h, ss_run_stats* out, ss_iter_stats* h_iters,
                                 int32_t cap) {
  if (!h || !out) {
    ss::set_error("slimsell_get_run_stats: NULL argument");
    return SS_ERR_INVALID;
  }
  ss_status s = ss::finish_run(h);
  *out = h->last;
  if (h_iters && cap > 0) {
    int cnt = h->last.iterations + 1;
    if (cnt > cap) cnt = cap;
    if (cnt > h->iter_cap) cnt = h->iter_cap;
    SS_CUDA(cudaMemcpy(h_iters, h->iters, sizeof(ss_iter_stats) * (size_t)cnt, cudaMemcpyDeviceToHost));
    // host events time each launch; a launch that ran several levels (cluster
    // push) left -1 markers for its later levels, whose device-side times are
    // taken from the iteration records and moved out of the launch's first level
    int owner = -1;
    for (int i = 0; i < cnt; ++i) {
      const int host = (i >= 1 && i - 1 < (int)h->iter_ns.size()) ? h->iter_ns[i - 1] : 0;
      if (host >= 0) {
        h_iters[i].kernel_ns = host;
        owner = i;
      } else {
        if (owner >= 1) h_iters[owner].kernel_ns = std::max(0, h_iters[owner].kernel_ns - h_iters[i].kernel_ns);
      }
    }
  }
  return s;
}

ss_status slimsell_set_profiling(slimsell_handle h, int32_t on) {
  if (!h) {
    ss::set_error("slimsell_set_profiling: NULL handle");
    return SS_ERR_INVALID;
  }
  h->profiling = on ? 1 : 0;
  return SS_OK;
}

ss_status slimsell_set_option(slimsell_handle h, int32_t option, int64_t value) {
  if (!h) {
    ss::set_error("slimsell_set_option: NULL handle");
    return SS_ERR_INVALID;
  }
  // options change captured loops and buffers a queued run may still be using
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
  switch (option) {
    case SS_OPT_DP_PASS:
      h->dp_pass = value ? 1 : 0;
      return SS_OK;
    case SS_OPT_DEVICE_LOOP:
      h->device_loop = value ? 1 : 0;
      return SS_OK;
    case SS_OPT_PROFILE_QUEUE:
      h->profile_queue = value ? 1 : 0;
      return SS_OK;
    case SS_OPT_FORMAT:
      if (value != SS_FORMAT_SLIMSELL && value != SS_FORMAT_SELL) {
        ss::set_error("slimsell_set_option: format must be SS_FORMAT_SLIMSELL or SS_FORMAT_SELL");
        return SS_ERR_INVALID;
      }
      h->format = (int)value;
      ss::drop_loop_graphs(h);  // captured loops hold the previous kernels
      return SS_OK;
    case SS_OPT_PUSH_BLOCKS:
      if (value < 0 || value > 2) {
        ss::set_error("slimsell_set_option: push blocks must be 0, 1 or 2");
        return SS_ERR_INVALID;
      }
      h->push_blocks = (int)value;
      ss::drop_loop_graphs(h);  // captured loops hold the previous value
      return SS_OK;
    case SS_OPT_SELECTOR_MARGIN:
      if (value < 0 || value > 100000) {
        ss::set_error("slimsell_set_option: selector margin must be in [0, 100000] thousandths");
        return SS_ERR_INVALID;
      }
      h->sel_margin = (float)value / 1000.0f;
      ss::drop_loop_graphs(h);
      return SS_OK;
    case SS_OPT_SMEM_BYTES:
      if (value < 0 || value > SS_SMEM_MAX_BYTES) {
        ss::set_error("slimsell_set_option: shared-memory bytes must be in [0, %d]", SS_SMEM_MAX_BYTES);
        return SS_ERR_INVALID;
      }
      h->smem_bytes = (int)value;
      return SS_OK;
    default:
      ss::set_error("slimsell_set_option: unknown option %d", option);
      return SS_ERR_INVALID;
  }
}

}  // extern "C"
