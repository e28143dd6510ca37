// Betweenness centrality on the SlimSell layout: Brandes' dependency
// accumulation, one of the algorithms the paper names in its conclusion as a
// target for SlimSell, run for up to 64 sources at once.
//
//   levels    the bit-packed multi-source BFS (the boolean semiring of Section
//             III-A on 64-source words, ss_multi.cu) gives, per level L, the
//             word LF[L][v] whose bit s says that v is at distance L from
//             source s; every level's word is kept;
//   forward,  level L = 1, 2, ...: each row v with LF[L][v] != 0 sums, for
//             every such source s, sigma[u][s] over its neighbours u with bit s
//             in LF[L-1][u] (the real-semiring step with the path counts kept);
//   backward, level L = D-1 .. 1: each row v at level L for source s sums
//             t[w][s] = (1 + delta[w][s]) / sigma[w][s] over its neighbours w
//             at level L+1 for s; then delta[v][s] = sigma[v][s] * sum and
//             bc(v) += delta[v][s].
//
// The rows of a level are cut into units of PUSH_UNIT neighbours (hub rows
// spread over many warps); one warp takes a unit, its lanes own sources
// (lane, lane + 32), and the 32 lanes first load 32 neighbours and their level
// words at once, then walk them together, each lane reading the per-source
// values of its two sources (one coalesced 512-byte row per neighbour).  Units
// of one row add into sigma / the dependency sums with fp64 atomicAdd, so sums
// may round in a different order than a serial run.  Path counts and
// dependencies are fp64 (path counts exact up to 2^53).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "ss_device.cuh"

namespace ss {

namespace {

constexpr int BCM_S = 64;  // sources per batch: one bit-packed word per row

struct BcScratch {
  double* sigma = nullptr;  // [n_pad][64] shortest-path counts
  double* dacc = nullptr;   // [n_pad][64] dependency sums of the rows' own level
  double* t = nullptr;      // [n_pad][64] (1 + delta) / sigma
  std::vector<unsigned long long*> lf;  // per level: [n_pad] level words
};

std::mutex g_bc_mu;
std::unordered_map<const slimsell_graph*, BcScratch> g_bc;

__global__ void k_bcm_init(Dev d, double* sigma, double* dacc) {
  const long long total = (long long)d.n_pad * BCM_S;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    sigma[i] = 0.0;
    dacc[i] = 0.0;
  }
}

// sigma = 1 for every source at its own row (level 0).
__global__ void k_bcm_roots(Dev d, const int* roots, int kb, double* sigma) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < kb) sigma[(long long)d.invperm[roots[s]] * BCM_S + s] = 1.0;
}

// Word 0 of every row of the multi-source frontier (W words per row) into lf.
__global__ void k_bcm_keep(Dev d, const unsigned long long* F, int W, unsigned long long* lf) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < d.n_pad;
       r += (long long)gridDim.x * blockDim.x)
    lf[r] = F[r * W];
}

// Work units of the rows with a non-zero level word.
__global__ void __launch_bounds__(256) k_bcm_expand(Dev d, const unsigned long long* lf) {
  const int lane = threadIdx.x & 31;
  const long long stride = ((long long)gridDim.x * blockDim.x) & ~31LL;
  for (long long r0 = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; r0 < d.n_pad; r0 += stride) {
    const long long r = r0 + lane;
    emit_units(d, (r < d.n_pad && lf[r] != 0ull) ? (int)r : -1, lane);
  }
}

// One unit: for every neighbour x of row v (in this unit) and every source s in
// lf_v[v] & lf_x[x], add val[x][s] into out[v][s].  Forward: lf_v = LF[L],
// lf_x = LF[L-1], val = sigma, out = sigma.  Backward: lf_v = LF[L], lf_x =
// LF[L+1], val = t, out = dacc.
__global__ void __launch_bounds__(256) k_bcm_gather(Dev d, const unsigned long long* __restrict__ lf_v,
                                                    const unsigned long long* __restrict__ lf_x,
                                                    const double* val, double* out) {
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nunits = min((long long)d.ctl->units, d.units_cap);
  for (long long ui = wid; ui < nunits; ui += nw) {
    const int2 un = d.units[ui];
    const long long v = un.x;
    const unsigned long long mv = lf_v[v];
    const int end = min(d.rdeg[v], un.y + PUSH_UNIT);
    const long long chunk = v / d.C;
    const long long base = d.cs[chunk] + (v - chunk * d.C);
    double a0 = 0.0, a1 = 0.0;
    for (int j0 = un.y; j0 < end; j0 += 32) {
      const int j = j0 + lane;
      int x = 0;
      unsigned long long mx = 0ull;
      if (j < end) {
        x = __ldg(d.col + base + (long long)j * d.C);
        mx = __ldg(lf_x + x) & mv;
      }
      unsigned any = __ballot_sync(SS_FULL_MASK, mx != 0ull);
      while (any) {  // the neighbours holding a source of this row, in turn
        const int q = __ffs(any) - 1;
        any &= any - 1;
        const unsigned long long m = __shfl_sync(SS_FULL_MASK, mx, q);
        const long long xq = __shfl_sync(SS_FULL_MASK, x, q);
        if (m >> lane & 1ull) a0 += val[xq * BCM_S + lane];
        if (m >> (lane + 32) & 1ull) a1 += val[xq * BCM_S + lane + 32];
      }
    }
    if (a0 != 0.0) atomicAdd(out + v * BCM_S + lane, a0);
    if (a1 != 0.0) atomicAdd(out + v * BCM_S + lane + 32, a1);
  }
}

// Backward post of level L, one warp per row: delta = sigma * dacc for the
// row's sources at level L, bc += their sum, t = (1 + delta) / sigma.
__global__ void __launch_bounds__(256) k_bcm_post(Dev d, const unsigned long long* __restrict__ lf,
                                                  const double* __restrict__ sigma,
                                                  const double* __restrict__ dacc, double* t,
                                                  double* bc) {
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = wid; v < d.n_pad; v += nw) {
    const unsigned long long mv = lf[v];
    if (!mv) continue;
    double sum = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sidx = lane + 32 * h;
      if (mv >> sidx & 1ull) {
        const long long i = v * BCM_S + sidx;
        const double sg = sigma[i];
        const double delta = sg * dacc[i];
        sum += delta;
        t[i] = (1.0 + delta) / sg;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(SS_FULL_MASK, sum, off);
    if (lane == 0 && sum != 0.0) bc[d.perm[v]] += sum;
  }
}

ss_status bc_scratch(slimsell_graph* h, BcScratch** out) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  BcScratch& b = g_bc[h];
  const size_t np = (size_t)h->n_pad * BCM_S;
  ss_status s;  // allocate whatever a failed earlier call left missing
  if (!b.sigma && (s = dmalloc(h, (void**)&b.sigma, sizeof(double) * np)) != SS_OK) return s;
  if (!b.dacc && (s = dmalloc(h, (void**)&b.dacc, sizeof(double) * np)) != SS_OK) return s;
  if (!b.t && (s = dmalloc(h, (void**)&b.t, sizeof(double) * np)) != SS_OK) return s;
  *out = &b;
  return SS_OK;
}

ss_status bc_level_word(slimsell_graph* h, BcScratch* b, size_t L, unsigned long long** out) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  while (b->lf.size() <= L) {
    unsigned long long* p = nullptr;
    ss_status s = dmalloc(h, (void**)&p, sizeof(unsigned long long) * (size_t)h->n_pad);
    if (s != SS_OK) return s;
    b->lf.push_back(p);
  }
  *out = b->lf[L];
  return SS_OK;
}

}  // namespace

void bc_release(slimsell_graph* h) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  auto it = g_bc.find(h);
  if (it == g_bc.end()) return;
  BcScratch& b = it->second;
  void* ptrs[] = {b.sigma, b.dacc, b.t};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (unsigned long long* p : b.lf) cudaFree(p);
  g_bc.erase(it);
}

}  // namespace ss

extern "C" ss_status slimsell_bc(slimsell_handle h, const int32_t* d_sources, int32_t k, double* d_bc,
                                 double* kernel_ms, void* stream) {
  using namespace ss;
  set_error("");
  if (!h || !d_sources || !d_bc) {
    set_error("slimsell_bc: NULL argument");
    return SS_ERR_INVALID;
  }
  h->values_semiring = -1;
  if (k < 1) {
    set_error("slimsell_bc: k must be at least 1 (got %d)", k);
    return SS_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> src((size_t)k);
  SS_CUDA(cudaMemcpyAsync(src.data(), d_sources, sizeof(int) * (size_t)k, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  for (int q = 0; q < k; ++q)
    if (src[(size_t)q] < 0 || src[(size_t)q] >= h->n) {
      set_error("slimsell_bc: source %d of entry %d out of range", src[(size_t)q], q);
      return SS_ERR_INVALID;
    }
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
  h->pending = 0;
  BcScratch* b = nullptr;
  ss_status s = bc_scratch(h, &b);
  if (s != SS_OK) return s;
  SS_CUDA(cudaMemsetAsync(d_bc, 0, sizeof(double) * (size_t)h->n, st));
  const int grid = 8 * h->num_sms;
  double ms_sum = 0.0;
  float ms = 0.f;
  auto tic = [&]() -> ss_status {
    if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_a, st));
    return SS_OK;
  };
  auto toc = [&]() -> ss_status {
    if (kernel_ms) {
      SS_CUDA(cudaEventRecord(h->ev_b, st));
      SS_CUDA(cudaEventSynchronize(h->ev_b));
      SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
      ms_sum += ms;
    }
    return SS_OK;
  };
  for (int b0 = 0; b0 < k; b0 += BCM_S) {
    const int kb = std::min(BCM_S, k - b0);
    if ((s = tic()) != SS_OK) return s;  // (the timed spans leave out the host's per-level reads)
    MultiDev m;
    int W = 1;
    if ((s = multi_start(h, d_sources + b0, kb, st, &m, &W)) != SS_OK) return s;
    const Dev d = m.d;
    k_bcm_init<<<grid, 256, 0, st>>>(d, b->sigma, b->dacc);
    k_bcm_roots<<<1, BCM_S, 0, st>>>(d, m.roots, kb, b->sigma);
    unsigned long long* lf0 = nullptr;
    if ((s = bc_level_word(h, b, 0, &lf0)) != SS_OK) return s;
    k_bcm_keep<<<grid, 256, 0, st>>>(d, m.F[0], W, lf0);
    SS_CUDA(cudaGetLastError());
    if ((s = toc()) != SS_OK) return s;
    // forward: the levels of the batch's sources and their path counts
    int D = 0;
    for (int L = 1;; ++L) {
      if (L > h->n + 1) {
        set_error("slimsell_bc: no convergence after %d levels", L);
        return SS_ERR_CUDA;
      }
      bool done = false;
      if ((s = multi_level(h, m, W, st, &done, kernel_ms ? h->ev_a : nullptr,
                           kernel_ms ? h->ev_b : nullptr)) != SS_OK)
        return s;
      if (kernel_ms) {
        SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
        ms_sum += ms;
      }
      if (done) break;
      if ((s = tic()) != SS_OK) return s;
      unsigned long long* lfL = nullptr;
      if ((s = bc_level_word(h, b, (size_t)L, &lfL)) != SS_OK) return s;
      k_bcm_keep<<<grid, 256, 0, st>>>(d, m.F[L & 1], W, lfL);
      SS_CUDA(cudaMemsetAsync(&h->ctl->units, 0, sizeof(unsigned long long), st));
      k_bcm_expand<<<grid, 256, 0, st>>>(d, lfL);
      k_bcm_gather<<<grid, 256, 0, st>>>(d, lfL, b->lf[(size_t)L - 1], b->sigma, b->sigma);
      SS_CUDA(cudaGetLastError());
      if ((s = toc()) != SS_OK) return s;
      D = L;
    }
    if ((s = tic()) != SS_OK) return s;
    // backward: the deepest level has no dependents (delta = 0, t = 1 / sigma)
    if (D >= 1) {
      k_bcm_post<<<grid, 256, 0, st>>>(d, b->lf[(size_t)D], b->sigma, b->dacc, b->t, d_bc);
      for (int L = D - 1; L >= 1; --L) {
        SS_CUDA(cudaMemsetAsync(&h->ctl->units, 0, sizeof(unsigned long long), st));
        k_bcm_expand<<<grid, 256, 0, st>>>(d, b->lf[(size_t)L]);
        k_bcm_gather<<<grid, 256, 0, st>>>(d, b->lf[(size_t)L], b->lf[(size_t)L + 1], b->t, b->dacc);
        k_bcm_post<<<grid, 256, 0, st>>>(d, b->lf[(size_t)L], b->sigma, b->dacc, b->t, d_bc);
      }
      SS_CUDA(cudaGetLastError());
    }
    if ((s = toc()) != SS_OK) return s;
  }
  SS_CUDA(cudaStreamSynchronize(st));
  if (kernel_ms) *kernel_ms = ms_sum;
  return SS_OK;
}
