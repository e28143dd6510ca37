// Betweenness centrality on the SlimSell layout: Brandes' dependency
// accumulation, one of the algorithms the paper names in its conclusion as a
// target for SlimSell.  For each source, two pulls over the handle's chunks and
// SlimChunk work items (thread l of a team of C owns row chunk * C + l, and the
// team reads C consecutive slots per column):
//
//   forward,  level L = 1, 2, ...: every row not yet reached sums sigma over its
//             neighbours at level L-1 (the real-semiring BFS step of Section
//             III-A with the path counts kept for every row); a row with a
//             non-zero sum enters level L with that many shortest paths;
//   backward, level L = D-1 .. 1 (D the last level): every row v at level L sums
//             t(w) = (1 + delta(w)) / sigma(w) over its neighbours, where t is
//             kept non-zero for the rows of level L+1 only; then
//             delta(v) = sigma(v) * sum and bc(v) += delta(v).
//
// Padding slots (col = -1) are skipped.  Split chunks combine partial sums with
// fp64 atomicAdd, so sums may round in a different order than a serial run.
// Path counts and dependencies are fp64 (path counts exact up to 2^53).
#include <climits>
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "ss_device.cuh"

namespace ss {

namespace {

constexpr int BC_THREADS = 256;  // a multiple of every supported C (8 .. 64)
constexpr int BC_PAD_LEVEL = INT_MAX;  // level of padding rows: never matches

struct BcScratch {
  int* lvl = nullptr;        // [n_pad] level (-1 unreached)
  double* sigma = nullptr;   // [n_pad] shortest-path counts
  double* acc = nullptr;     // [n_pad] pull sums of the current level
  double* t = nullptr;       // [n_pad] (1 + delta) / sigma of the rows one level deeper
  unsigned long long* cnt = nullptr;  // rows reached so far by the forward pass
};

std::mutex g_bc_mu;
std::unordered_map<const slimsell_graph*, BcScratch> g_bc;

__global__ void k_bc_init(Dev d, int root_row, int* lvl, double* sigma, double* acc, double* t,
                          unsigned long long* cnt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride) {
    const bool r = row == root_row;
    lvl[row] = r ? 0 : (row < d.n ? -1 : BC_PAD_LEVEL);
    sigma[row] = r ? 1.0 : 0.0;
    acc[row] = 0.0;
    t[row] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = 0ull;
}

// Forward pull of level L over the rows not yet reached.
__global__ void __launch_bounds__(BC_THREADS) k_bc_fwd(Dev d, int L, const int* __restrict__ lvl,
                                                       const double* __restrict__ sigma,
                                                       double* __restrict__ acc) {
  const int C = d.C;
  const int teams = BC_THREADS / C;
  const int team = threadIdx.x / C, lane = threadIdx.x - team * C;
  for (long long it = (long long)blockIdx.x * teams + team; it < d.n_items;
       it += (long long)gridDim.x * teams) {
    const int4 item = d.items[it];
    const long long row = (long long)item.x * C + lane;
    if (lvl[row] != -1) continue;  // reached already, or a padding row
    const long long base = d.cs[item.x] + lane;
    double a = 0.0;
#pragma unroll 4
    for (int j = item.y; j < item.z; ++j) {
      const int c = __ldcs(d.col + base + (long long)j * C);
      if (c >= 0 && lvl[c] == L - 1) a += sigma[c];
    }
    if (a != 0.0) {
      if (item.w < 0) acc[row] = a;
      else atomicAdd(acc + row, a);
    }
  }
}

__global__ void __launch_bounds__(BC_THREADS) k_bc_fwd_post(Dev d, int L, int* __restrict__ lvl,
                                                            double* __restrict__ sigma,
                                                            double* __restrict__ acc,
                                                            unsigned long long* cnt) {
  unsigned mine = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride) {
    const double a = acc[row];
    if (a != 0.0) {
      acc[row] = 0.0;
      if (lvl[row] == -1) {
        lvl[row] = L;
        sigma[row] = a;
        ++mine;
      }
    }
  }
  mine = __reduce_add_sync(SS_FULL_MASK, mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(cnt, (unsigned long long)mine);
}

// t for the deepest level D: delta = 0 there.
__global__ void k_bc_back_init(Dev d, int D, const int* __restrict__ lvl, const double* __restrict__ sigma,
                               double* __restrict__ t) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride)
    t[row] = lvl[row] == D ? 1.0 / sigma[row] : 0.0;
}

// Backward pull of level L: rows at level L sum t over their neighbours (t is
// non-zero exactly on the rows of level L+1).
__global__ void __launch_bounds__(BC_THREADS) k_bc_back(Dev d, int L, const int* __restrict__ lvl,
                                                        const double* __restrict__ t,
                                                        double* __restrict__ acc) {
  const int C = d.C;
  const int teams = BC_THREADS / C;
  const int team = threadIdx.x / C, lane = threadIdx.x - team * C;
  for (long long it = (long long)blockIdx.x * teams + team; it < d.n_items;
       it += (long long)gridDim.x * teams) {
    const int4 item = d.items[it];
    const long long row = (long long)item.x * C + lane;
    if (lvl[row] != L) continue;
    const long long base = d.cs[item.x] + lane;
    double a = 0.0;
#pragma unroll 4
    for (int j = item.y; j < item.z; ++j) {
      const int c = __ldcs(d.col + base + (long long)j * C);
      if (c >= 0) a += t[c];
    }
    if (a != 0.0) {
      if (item.w < 0) acc[row] = a;
      else atomicAdd(acc + row, a);
    }
  }
}

__global__ void __launch_bounds__(BC_THREADS) k_bc_back_post(Dev d, int L, const int* __restrict__ lvl,
                                                             const double* __restrict__ sigma,
                                                             double* __restrict__ acc,
                                                             double* __restrict__ t,
                                                             double* __restrict__ bc) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride) {
    const int l = lvl[row];
    if (l == L) {
      const double delta = sigma[row] * acc[row];
      acc[row] = 0.0;
      bc[d.perm[row]] += delta;
      t[row] = (1.0 + delta) / sigma[row];
    } else if (l == L + 1) {
      t[row] = 0.0;
    }
  }
}

ss_status bc_scratch(slimsell_graph* h, BcScratch** out) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  BcScratch& b = g_bc[h];
  const size_t np = (size_t)h->n_pad;
  ss_status s;  // allocate whatever a failed earlier call left missing
  if (!b.lvl && (s = dmalloc(h, (void**)&b.lvl, sizeof(int) * np)) != SS_OK) return s;
  if (!b.sigma && (s = dmalloc(h, (void**)&b.sigma, sizeof(double) * np)) != SS_OK) return s;
  if (!b.acc && (s = dmalloc(h, (void**)&b.acc, sizeof(double) * np)) != SS_OK) return s;
  if (!b.t && (s = dmalloc(h, (void**)&b.t, sizeof(double) * np)) != SS_OK) return s;
  if (!b.cnt && (s = dmalloc(h, (void**)&b.cnt, sizeof(unsigned long long))) != SS_OK) return s;
  *out = &b;
  return SS_OK;
}

}  // namespace

void bc_release(slimsell_graph* h) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  auto it = g_bc.find(h);
  if (it == g_bc.end()) return;
  BcScratch& b = it->second;
  void* ptrs[] = {b.lvl, b.sigma, b.acc, b.t, b.cnt};
  for (void* p : ptrs)
    if (p) cudaFree(p);
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
  std::vector<int> rows((size_t)k);
  for (int q = 0; q < k; ++q)
    SS_CUDA(cudaMemcpyAsync(&rows[(size_t)q], h->invperm + src[(size_t)q], sizeof(int),
                            cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaMemsetAsync(d_bc, 0, sizeof(double) * (size_t)h->n, st));
  SS_CUDA(cudaStreamSynchronize(st));
  const Dev d = h->dev();
  const int grid = 8 * h->num_sms;
  double ms_sum = 0.0;
  float ms = 0.f;
  for (int q = 0; q < k; ++q) {
    k_bc_init<<<grid, 256, 0, st>>>(d, rows[(size_t)q], b->lvl, b->sigma, b->acc, b->t, b->cnt);
    SS_CUDA(cudaGetLastError());
    unsigned long long prev = 0, now = 0;
    int D = 0;
    for (int L = 1;; ++L) {
      if (L > h->n + 1) {
        set_error("slimsell_bc: no convergence after %d levels", L);
        return SS_ERR_CUDA;
      }
      if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_a, st));
      k_bc_fwd<<<grid, BC_THREADS, 0, st>>>(d, L, b->lvl, b->sigma, b->acc);
      k_bc_fwd_post<<<grid, BC_THREADS, 0, st>>>(d, L, b->lvl, b->sigma, b->acc, b->cnt);
      SS_CUDA(cudaGetLastError());
      if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_b, st));
      SS_CUDA(cudaMemcpyAsync(&now, b->cnt, sizeof(now), cudaMemcpyDeviceToHost, st));
      SS_CUDA(cudaStreamSynchronize(st));
      if (kernel_ms) {
        SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
        ms_sum += ms;
      }
      if (now == prev) break;
      prev = now;
      D = L;
    }
    if (D < 2) continue;  // no vertex strictly between the source and another vertex
    if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_a, st));
    k_bc_back_init<<<grid, 256, 0, st>>>(d, D, b->lvl, b->sigma, b->t);
    for (int L = D - 1; L >= 1; --L) {
      k_bc_back<<<grid, BC_THREADS, 0, st>>>(d, L, b->lvl, b->t, b->acc);
      k_bc_back_post<<<grid, BC_THREADS, 0, st>>>(d, L, b->lvl, b->sigma, b->acc, b->t, d_bc);
    }
    SS_CUDA(cudaGetLastError());
    if (kernel_ms) {
      SS_CUDA(cudaEventRecord(h->ev_b, st));
      SS_CUDA(cudaEventSynchronize(h->ev_b));
      SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
      ms_sum += ms;
    }
  }
  SS_CUDA(cudaStreamSynchronize(st));
  if (kernel_ms) *kernel_ms = ms_sum;
  return SS_OK;
}
