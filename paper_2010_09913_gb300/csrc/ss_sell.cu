// Sell-C-sigma with an explicit value array against SlimSell: the storage-format
// comparison of Section IV (advantages of SlimSell).  Both formats run the same
// value-vector BFS-SpMV iteration of Section III-A over the handle's chunks and
// SlimChunk work items; they differ only in where a slot's matrix value comes
// from:
//
//   SlimSell (SS_FORMAT_SLIMSELL)  value = 1 where col >= 0 (Section III-B); a
//                                  padding slot (col = -1) is skipped and
//                                  gathers nothing;
//   Sell-C-sigma (SS_FORMAT_SELL)  value = val[slot]: 1 for an edge, the
//                                  semiring's zero for padding, whose col is 0
//                                  (Section II-D); every slot loads col and val
//                                  and gathers x[col].
//
// The iteration is the paper's x_k = A (x) f_{k-1} with the semiring's
// post-processing, on fp32 value vectors (one entry per row):
//   tropical  f = distances so far (inf unreached), x = min_j (a_j + f[col_j]);
//   real      f = path counts of the previous frontier, x = sum_j a_j * f[col_j];
//   boolean   f = 1 on the previous frontier, x = OR_j (a_j AND f[col_j]);
//   sel-max   f = vertex id + 1 on the previous frontier, x = max_j a_j * f[col_j];
// a row not yet reached whose x is not the semiring's zero enters level k.
// Real-semiring path counts saturate at the largest finite float, so that a
// Sell padding product 0 * f[0] stays 0.
// No SlimWork and no frontier bitmaps: every iteration streams every slot, so
// the two formats do identical work apart from the value array.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "ss_device.cuh"

namespace ss {

namespace {

constexpr int AB_THREADS = 256;  // a multiple of every supported C (8 .. 64)

// Per-handle scratch of the format comparison, allocated on first use and
// released with the handle.
struct AbScratch {
  int* scol = nullptr;      // [slots] Sell col: padding 0
  float* vtrop = nullptr;   // [slots] Sell val for the tropical semiring: 1 edge, inf padding
  float* vmul = nullptr;    // [slots] Sell val for the other semirings: 1 edge, 0 padding
  float* x[2] = {nullptr, nullptr};  // [n_pad] value vectors by level parity
  float* acc = nullptr;     // [n_pad] SpMV result of the current level
  int* lvl = nullptr;       // [n_pad] level of each row (-1 unreached)
  unsigned long long* cnt = nullptr;  // rows reached by the current level
};

std::mutex g_ab_mu;
std::unordered_map<const slimsell_graph*, AbScratch> g_ab;

template <int SR>
__device__ __forceinline__ float sr_zero() {
  return SR == SS_TROPICAL ? __int_as_float(0x7f800000) : 0.0f;
}

// a (x) x: the product of a matrix value and a vector entry
template <int SR>
__device__ __forceinline__ float sr_mul(float a, float x) {
  if (SR == SS_TROPICAL) return a + x;
  if (SR == SS_BOOLEAN) return fminf(a, x);  // AND on {0, 1}
  return a * x;                              // real, sel-max
}

// the semiring's addition
template <int SR>
__device__ __forceinline__ float sr_add(float a, float b) {
  if (SR == SS_TROPICAL) return fminf(a, b);
  if (SR == SS_REAL) return a + b;
  return fmaxf(a, b);  // boolean OR on {0, 1}, sel-max max
}

// Combine a split chunk's partial row results.  Every value is >= 0 (or +inf),
// so the float order equals the order of the bit patterns as signed ints.
template <int SR>
__device__ __forceinline__ void sr_atomic_add(float* p, float v) {
  if (SR == SS_TROPICAL) atomicMin(reinterpret_cast<int*>(p), __float_as_int(v));
  else if (SR == SS_REAL) atomicAdd(p, v);
  else atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));
}

// x = A (x) f over the work items: a team of C threads per item, thread l of a
// team owns row chunk * C + l and walks the item's columns (C consecutive slots
// per column: coalesced).
template <int SR, int FORMAT>
__global__ void __launch_bounds__(AB_THREADS) k_ab_spmv(Dev d, const int* __restrict__ scol,
                                                        const float* __restrict__ sval,
                                                        const float* __restrict__ f,
                                                        float* __restrict__ acc) {
  const int C = d.C;
  const int teams = AB_THREADS / C;
  const int team = threadIdx.x / C, lane = threadIdx.x - team * C;
  for (long long it = (long long)blockIdx.x * teams + team; it < d.n_items;
       it += (long long)gridDim.x * teams) {
    const int4 item = d.items[it];
    const long long row = (long long)item.x * C + lane;
    const long long base = d.cs[item.x] + lane;
    float a = sr_zero<SR>();
#pragma unroll 4
    for (int j = item.y; j < item.z; ++j) {
      const long long s = base + (long long)j * C;
      if (FORMAT == SS_FORMAT_SLIMSELL) {
        const int c = __ldcs(d.col + s);
        if (c >= 0) a = sr_add<SR>(a, sr_mul<SR>(1.0f, f[c]));
      } else {
        const int c = __ldcs(scol + s);
        const float v = __ldcs(sval + s);
        a = sr_add<SR>(a, sr_mul<SR>(v, f[c]));
      }
    }
    if (item.w < 0) acc[row] = a;
    else sr_atomic_add<SR>(acc + row, a);
  }
}

// Post-processing of level `level`: rows reached for the first time get their
// level and distance, the next value vector is written, acc is reset.
template <int SR>
__global__ void __launch_bounds__(AB_THREADS) k_ab_post(Dev d, int level, float* __restrict__ acc,
                                                        float* __restrict__ fn, int* __restrict__ lvl,
                                                        int* __restrict__ dist,
                                                        unsigned long long* cnt) {
  unsigned long long mine = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride) {
    const float a = acc[row];
    acc[row] = sr_zero<SR>();
    float out = sr_zero<SR>();
    if (row < d.n) {
      const int L = lvl[row];
      if (L < 0) {
        const bool hit = SR == SS_TROPICAL ? (a < __int_as_float(0x7f800000)) : (a > 0.0f);
        if (hit) {
          const int v = d.perm[row];
          lvl[row] = level;
          dist[v] = level;
          ++mine;
          out = SR == SS_TROPICAL ? (float)level
              : SR == SS_REAL     ? fminf(a, 3.402823466e38f)  // saturate: 0 * value stays 0
              : SR == SS_BOOLEAN  ? 1.0f
                                  : (float)(v + 1);
        }
      } else if (SR == SS_TROPICAL) {
        out = (float)L;  // distances stay in the tropical vector
      }
    }
    fn[row] = out;
  }
  mine = __reduce_add_sync(SS_FULL_MASK, (unsigned)mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(cnt, mine);
}

template <int SR>
__global__ void k_ab_init(Dev d, int root_row, int root, float* f, float* acc, int* lvl,
                          unsigned long long* cnt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < d.n_pad; row += stride) {
    const bool r = row == root_row;
    lvl[row] = r ? 0 : -1;
    acc[row] = sr_zero<SR>();
    f[row] = !r ? sr_zero<SR>()
           : SR == SS_TROPICAL ? 0.0f
           : SR == SS_SELMAX   ? (float)(root + 1)
                               : 1.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = 0ull;
}

__global__ void k_sell_arrays(const int* __restrict__ col, long long slots, int* __restrict__ scol,
                              float* __restrict__ vtrop, float* __restrict__ vmul) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += stride) {
    const int c = col[s];
    scol[s] = c < 0 ? 0 : c;
    vtrop[s] = c < 0 ? __int_as_float(0x7f800000) : 1.0f;
    vmul[s] = c < 0 ? 0.0f : 1.0f;
  }
}

ss_status ab_scratch(slimsell_graph* h, bool sell, cudaStream_t st, AbScratch** out) {
  std::lock_guard<std::mutex> lock(g_ab_mu);
  AbScratch& a = g_ab[h];
  ss_status s;
  const size_t np = (size_t)h->n_pad;
  // allocate whatever is missing (also after a failed earlier call)
  for (int b = 0; b < 2; ++b)
    if (!a.x[b] && (s = dmalloc(h, (void**)&a.x[b], sizeof(float) * np)) != SS_OK) return s;
  if (!a.acc && (s = dmalloc(h, (void**)&a.acc, sizeof(float) * np)) != SS_OK) return s;
  if (!a.lvl && (s = dmalloc(h, (void**)&a.lvl, sizeof(int) * np)) != SS_OK) return s;
  if (!a.cnt && (s = dmalloc(h, (void**)&a.cnt, sizeof(unsigned long long))) != SS_OK) return s;
  if (sell && !a.vmul) {  // vmul is written last: its presence means the arrays are built
    const size_t slots = (size_t)(h->slots > 0 ? h->slots : 1);
    if (!a.scol && (s = dmalloc(h, (void**)&a.scol, sizeof(int) * slots)) != SS_OK) return s;
    if (!a.vtrop && (s = dmalloc(h, (void**)&a.vtrop, sizeof(float) * slots)) != SS_OK) return s;
    if ((s = dmalloc(h, (void**)&a.vmul, sizeof(float) * slots)) != SS_OK) return s;
    if (h->slots > 0) {
      k_sell_arrays<<<8 * h->num_sms, 256, 0, st>>>(h->col, h->slots, a.scol, a.vtrop, a.vmul);
      SS_CUDA(cudaGetLastError());
    }
  }
  *out = &a;
  return SS_OK;
}

}  // namespace

// The Sell-C-sigma arrays of the handle (built on first use), for the
// production pull's format option.
ss_status sell_arrays(slimsell_graph* h, cudaStream_t st) {
  AbScratch* a = nullptr;
  ss_status s = ab_scratch(h, true, st, &a);
  if (s != SS_OK) return s;
  h->sell_col = a->scol;
  h->sell_vtrop = a->vtrop;
  h->sell_vmul = a->vmul;
  return SS_OK;
}

namespace {

template <int SR>
ss_status run_ab(slimsell_graph* h, int root, int format, int* d_dist, double* kernel_ms,
                 cudaStream_t st) {
  AbScratch* a = nullptr;
  ss_status s = ab_scratch(h, format == SS_FORMAT_SELL, st, &a);
  if (s != SS_OK) return s;
  const Dev d = h->dev();
  int root_row = 0;
  SS_CUDA(cudaMemcpyAsync(&root_row, h->invperm + root, sizeof(int), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  SS_CUDA(cudaMemsetAsync(d_dist, 0xff, sizeof(int) * (size_t)h->n, st));
  SS_CUDA(cudaMemsetAsync(d_dist + root, 0, sizeof(int), st));
  const int grid = 8 * h->num_sms;
  k_ab_init<SR><<<grid, 256, 0, st>>>(d, root_row, root, a->x[0], a->acc, a->lvl, a->cnt);
  SS_CUDA(cudaGetLastError());
  const float* sval = SR == SS_TROPICAL ? a->vtrop : a->vmul;
  double ms_sum = 0.0;
  unsigned long long prev = 0, now = 0;
  for (int level = 1;; ++level) {
    if (level > h->n + 1) {
      set_error("slimsell_bfs_spmv: no convergence after %d iterations", level);
      return SS_ERR_CUDA;
    }
    if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_a, st));
    const float* f = a->x[(level - 1) & 1];
    if (format == SS_FORMAT_SELL)
      k_ab_spmv<SR, SS_FORMAT_SELL><<<grid, AB_THREADS, 0, st>>>(d, a->scol, sval, f, a->acc);
    else
      k_ab_spmv<SR, SS_FORMAT_SLIMSELL><<<grid, AB_THREADS, 0, st>>>(d, nullptr, nullptr, f, a->acc);
    SS_CUDA(cudaGetLastError());
    k_ab_post<SR><<<grid, AB_THREADS, 0, st>>>(d, level, a->acc, a->x[level & 1], a->lvl, d_dist, a->cnt);
    SS_CUDA(cudaGetLastError());
    if (kernel_ms) SS_CUDA(cudaEventRecord(h->ev_b, st));
    SS_CUDA(cudaMemcpyAsync(&now, a->cnt, sizeof(now), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    if (kernel_ms) {
      float ms = 0.f;
      SS_CUDA(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
      ms_sum += ms;
    }
    if (now == prev) break;  // no row entered this level
    prev = now;
  }
  if (kernel_ms) *kernel_ms = ms_sum;
  return SS_OK;
}

}  // namespace

void ab_release(slimsell_graph* h) {
  std::lock_guard<std::mutex> lock(g_ab_mu);
  auto it = g_ab.find(h);
  if (it == g_ab.end()) return;
  AbScratch& a = it->second;
  void* ptrs[] = {a.scol, a.vtrop, a.vmul, a.x[0], a.x[1], a.acc, a.lvl, a.cnt};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  g_ab.erase(it);
}

}  // namespace ss

extern "C" ss_status slimsell_bfs_spmv(slimsell_handle h, int32_t root, int32_t semiring, int32_t format,
                                       int32_t* d_dist, double* kernel_ms, void* stream) {
  using namespace ss;
  set_error("");
  if (!h || !d_dist) {
    set_error("slimsell_bfs_spmv: NULL argument");
    return SS_ERR_INVALID;
  }
  h->values_semiring = -1;
  if (root < 0 || root >= h->n) {
    set_error("slimsell_bfs_spmv: root %d out of range [0, %d)", root, h->n);
    return SS_ERR_INVALID;
  }
  if (format != SS_FORMAT_SLIMSELL && format != SS_FORMAT_SELL) {
    set_error("slimsell_bfs_spmv: format must be SS_FORMAT_SLIMSELL or SS_FORMAT_SELL");
    return SS_ERR_INVALID;
  }
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));
  h->pending = 0;
  cudaStream_t st = (cudaStream_t)stream;
  switch (semiring) {
    case SS_TROPICAL: return run_ab<SS_TROPICAL>(h, root, format, d_dist, kernel_ms, st);
    case SS_REAL: return run_ab<SS_REAL>(h, root, format, d_dist, kernel_ms, st);
    case SS_BOOLEAN: return run_ab<SS_BOOLEAN>(h, root, format, d_dist, kernel_ms, st);
    case SS_SELMAX: return run_ab<SS_SELMAX>(h, root, format, d_dist, kernel_ms, st);
    default:
      set_error("slimsell_bfs_spmv: unknown semiring %d", semiring);
      return SS_ERR_INVALID;
  }
}
