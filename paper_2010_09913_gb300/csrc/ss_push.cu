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
