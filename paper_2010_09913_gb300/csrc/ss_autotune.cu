// Layout autotuner: the chunk height C, the sorting scope sigma and the
// SlimChunk width of a graph are chosen by building the layout for every point
// of a grid and timing BFS on sample roots (the paper studies the same three
// parameters by hand, Sections III-D and IV).  Searches are cached by a graph
// signature, so graphs of one family and size share one search.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ss_common.cuh"

namespace ss {
namespace {

constexpr int TUNE_HIST = 24;       // log2-degree buckets of the signature
constexpr int TUNE_TOLERANCE = 3;   // L1 distance (histogram units) accepted by the cache
constexpr double TUNE_HIST_UNIT = 50.0;  // a bucket counts its share of vertices in 1/50 units

// Raw counts of vertices per floor(log2 degree) bucket (degree >= 1, buckets
// below TUNE_HIST), one shared-memory histogram per block.
__global__ void k_tune_hist(const long long* row_ptr, int n, unsigned long long* counts) {
  __shared__ unsigned h[TUNE_HIST];
  if (threadIdx.x < TUNE_HIST) h[threadIdx.x] = 0u;
  __syncthreads();
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    if (deg > 0) {
      const int b = 63 - __clzll((unsigned long long)deg);
      if (b < TUNE_HIST) atomicAdd(&h[b], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < TUNE_HIST && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

int bucket_of(long long deg) {
  int b = 0;
  while ((deg >> 1) > 0) {
    deg >>= 1;
    ++b;
  }
  return b;
}

// nnz rounded to two significant digits.
long long round2(long long x) {
  if (x < 100) return x;
  long long p = 1;
  while (x / p >= 100) p *= 10;
  return ((x + p / 2) / p) * p;
}

void finish_signature(int n, long long nnz, const unsigned long long* counts, ss_tune_signature* out) {
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->nnz_rounded = round2(nnz);
  const double scale = TUNE_HIST_UNIT / (double)(n > 0 ? n : 1);
  for (int b = 0; b < TUNE_HIST; ++b) out->hist[b] = (int32_t)std::lround((double)counts[b] * scale);
}

int hist_distance(const ss_tune_signature& a, const ss_tune_signature& b) {
  int d = 0;
  for (int i = 0; i < TUNE_HIST; ++i) d += std::abs(a.hist[i] - b.hist[i]);
  return d;
}

struct TuneEntry {
  ss_tune_signature sig;
  int semiring, policy;
  std::vector<int> gC, gS, gW;
  ss_tune_point best;
  std::vector<ss_tune_point> table;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune_cache;

// Exact signature match, else the closest matching one (same n, rounded nnz,
// semiring, policy and grid; histogram within TUNE_TOLERANCE); NULL if none.
const TuneEntry* tune_lookup(const ss_tune_signature& sig, int sr, int pol, const std::vector<int>& gC,
                             const std::vector<int>& gS, const std::vector<int>& gW) {
  const TuneEntry* best = nullptr;
  int best_d = TUNE_TOLERANCE + 1;
  for (const TuneEntry& e : g_tune_cache) {
    if (e.semiring != sr || e.policy != pol || e.gC != gC || e.gS != gS || e.gW != gW) continue;
    if (e.sig.n != sig.n || e.sig.nnz_rounded != sig.nnz_rounded) continue;
    const int d = hist_distance(e.sig, sig);
    if (d < best_d) {
      best = &e;
      best_d = d;
    }
  }
  return best;
}

}  // namespace
}  // namespace ss

extern "C" {

ss_status slimsell_tune_signature(const int64_t* h_row_ptr, int32_t n, ss_tune_signature* out) {
  using namespace ss;
  set_error("");
  if (!h_row_ptr || !out || n < 0) {
    set_error("slimsell_tune_signature: NULL pointer or n < 0");
    return SS_ERR_INVALID;
  }
  unsigned long long counts[TUNE_HIST] = {};
  for (int32_t v = 0; v < n; ++v) {
    const long long deg = h_row_ptr[v + 1] - h_row_ptr[v];
    if (deg > 0) {
      const int b = bucket_of(deg);
      if (b < TUNE_HIST) counts[b] += 1;
    }
  }
  finish_signature(n, n > 0 ? h_row_ptr[n] - h_row_ptr[0] : 0, counts, out);
  return SS_OK;
}

int32_t slimsell_tune_match(const ss_tune_signature* a, const ss_tune_signature* b) {
  if (!a || !b) return 0;
  if (a->n != b->n || a->nnz_rounded != b->nnz_rounded) return 0;
  return ss::hist_distance(*a, *b) <= ss::TUNE_TOLERANCE ? 1 : 0;
}

ss_status slimsell_autotune(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                            int32_t semiring, int32_t policy, const int32_t* h_roots, int32_t nroots,
                            const int32_t* h_C, int32_t nC, const int32_t* h_sigma, int32_t nsigma,
                            const int32_t* h_split_w, int32_t nw, int32_t repeats, int32_t use_cache,
                            ss_tune_result* h_result, ss_tune_point* h_table, int32_t table_cap,
                            void* stream) {
  using namespace ss;
  set_error("");
  if (!d_row_ptr || !d_col || !h_roots || !h_C || !h_sigma || !h_split_w || !h_result) {
    set_error("slimsell_autotune: NULL pointer");
    return SS_ERR_INVALID;
  }
  if (n < 1 || nnz < 0 || nroots < 1 || nC < 1 || nsigma < 1 || nw < 1 || repeats < 1 ||
      table_cap < 0 || (table_cap > 0 && !h_table)) {
    set_error("slimsell_autotune: n, nroots, grid sizes and repeats must be >= 1 (nnz, table_cap >= 0)");
    return SS_ERR_INVALID;
  }
  if (semiring < SS_TROPICAL || semiring > SS_SELMAX || policy < SS_V_FULL || policy > SS_V_LEARNED) {
    set_error("slimsell_autotune: unknown semiring %d or policy %d", semiring, policy);
    return SS_ERR_INVALID;
  }
  for (int i = 0; i < nroots; ++i)
    if (h_roots[i] < 0 || h_roots[i] >= n) {
      set_error("slimsell_autotune: root %d out of range [0, %d)", h_roots[i], n);
      return SS_ERR_INVALID;
    }
  for (int i = 0; i < nC; ++i)
    if (h_C[i] != 8 && h_C[i] != 16 && h_C[i] != 32 && h_C[i] != 64) {
      set_error("slimsell_autotune: C must be 8, 16, 32 or 64 (got %d)", h_C[i]);
      return SS_ERR_INVALID;
    }
  for (int i = 0; i < nsigma; ++i)
    if (h_sigma[i] < 0) {
      set_error("slimsell_autotune: sigma must be >= 0 (0 = n)");
      return SS_ERR_INVALID;
    }
  for (int i = 0; i < nw; ++i)
    if (h_split_w[i] < 0) {
      set_error("slimsell_autotune: split width must be >= 0");
      return SS_ERR_INVALID;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const std::vector<int> gC(h_C, h_C + nC), gS(h_sigma, h_sigma + nsigma), gW(h_split_w, h_split_w + nw);

  // signature from a device histogram of log2 degrees
  unsigned long long* d_counts = nullptr;
  SS_CUDA(cudaMallocAsync((void**)&d_counts, sizeof(unsigned long long) * TUNE_HIST, st));
  cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * TUNE_HIST, st);
  unsigned long long counts[TUNE_HIST] = {};
  if (e == cudaSuccess) {
    const int grid = (int)std::min<long long>(1024, ((long long)n + 255) / 256);
    k_tune_hist<<<grid, 256, 0, st>>>(reinterpret_cast<const long long*>(d_row_ptr), n, d_counts);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(d_counts, st);
  if (e != cudaSuccess) return cuda_fail(e, "slimsell_autotune: degree histogram");
  ss_tune_signature sig;
  finish_signature(n, nnz, counts, &sig);

  const int total = nC * nsigma * nw;
  if (use_cache) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const TuneEntry* hit = tune_lookup(sig, semiring, policy, gC, gS, gW);
    if (hit) {
      h_result->best = hit->best;
      h_result->points = 0;
      h_result->cached = 1;
      for (int i = 0; i < total && i < table_cap; ++i) h_table[i] = hit->table[i];
      return SS_OK;
    }
  }

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  std::vector<ss_tune_point> table;
  ss_status s = SS_OK;
  for (int ic = 0; ic < nC && s == SS_OK; ++ic)
    for (int is = 0; is < nsigma && s == SS_OK; ++is)
      for (int iw = 0; iw < nw && s == SS_OK; ++iw) {
        ss_tune_point p{h_C[ic], h_sigma[is], h_split_w[iw], 0.f};
        slimsell_handle h = nullptr;
        s = slimsell_build(d_row_ptr, d_col, n, nnz, p.C, p.sigma == 0 ? n : p.sigma, p.split_w, stream, &h);
        if (s != SS_OK) break;
        s = slimsell_bfs(h, h_roots[0], semiring, policy, nullptr, nullptr, stream);  // builds the loop
        ss_run_stats rs;
        if (s == SS_OK) s = slimsell_get_run_stats(h, &rs, nullptr, 0);
        if (s == SS_OK && cudaEventRecord(e0, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
        for (int rep = 0; rep < repeats && s == SS_OK; ++rep)
          for (int i = 0; i < nroots && s == SS_OK; ++i)
            s = slimsell_bfs(h, h_roots[i], semiring, policy, nullptr, nullptr, stream);
        if (s == SS_OK) {
          float ms = 0.f;
          if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            s = cuda_fail(cudaGetLastError(), "slimsell_autotune: timing");
          p.ms = ms / (float)(repeats * nroots);
        }
        if (s == SS_OK) s = slimsell_get_run_stats(h, &rs, nullptr, 0);  // device errors of the runs
        slimsell_destroy(h);
        if (s == SS_OK) table.push_back(p);
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SS_OK) return s;
  ss_tune_point best = table[0];
  for (const ss_tune_point& p : table)
    if (p.ms < best.ms) best = p;
  h_result->best = best;
  h_result->points = total;
  h_result->cached = 0;
  for (int i = 0; i < total && i < table_cap; ++i) h_table[i] = table[i];
  {  // every search is cached; use_cache only decides whether a search may be skipped
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back(TuneEntry{sig, semiring, policy, gC, gS, gW, best, table});
  }
  return SS_OK;
}

}  // extern "C"
