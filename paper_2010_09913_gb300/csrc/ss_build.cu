// Device-side SlimSell builder (Sections II-D and III-B; SlimChunk split table, Section III-D).
//
//   1. degrees and the sort key (window of sigma vertices, descending degree)
//   2. stable LSD radix sort of (key, vertex) -> perm; ties keep ascending id
//   3. invperm, per-row degree, chunk lengths cl, chunk starts cs (exclusive scan)
//   4. work-item tables: pack items (fixed width) and BFS items (SlimChunk width)
//   5. column-major pack: col[cs_i + j*C + l] = invperm[j-th neighbour of row i*C+l,
//      descending original id], or -1 for padding
#include <cstdarg>
#include <climits>
#include <algorithm>
#include <cstring>
#include <vector>

#include "ss_device.cuh"
#include "ss_sort.cuh"

namespace ss {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

ss_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA;
}

ss_status dmalloc(slimsell_graph* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  if (h) h->device_bytes += (long long)bytes;
  return SS_OK;
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum over int64 (three passes: tile sums, scan of sums, tile scans)
// ---------------------------------------------------------------------------

__device__ __forceinline__ long long warp_incl_scan(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(SS_FULL_MASK, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ long long block_excl_scan(long long v, long long* total) {
  __shared__ long long wsum[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = warp_incl_scan(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long s = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0;
    s = warp_incl_scan(s);
    if (lane < SCAN_THREADS / 32) wsum[lane] = s;
  }
  __syncthreads();
  long long before = (w > 0 ? wsum[w - 1] : 0) + inc - v;
  *total = wsum[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void k_tile_sum(const long long* in, long long n, long long* partial) {
  long long base = (long long)blockIdx.x * SCAN_TILE;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    long long idx = base + (long long)i * SCAN_THREADS + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  long long total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void k_scan_partials(long long* partial, int ntiles) {
  // one block of 1024 threads; each thread owns a contiguous run
  __shared__ long long sums[1024];
  const int t = threadIdx.x;
  const int per = (ntiles + 1023) / 1024;
  const int lo = min(t * per, ntiles), hi = min(lo + per, ntiles);
  long long s = 0;
  for (int i = lo; i < hi; ++i) s += partial[i];
  sums[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long v = (t >= o) ? sums[t - o] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  long long run = sums[t] - s;
  for (int i = lo; i < hi; ++i) {
    long long v = partial[i];
    partial[i] = run;
    run += v;
  }
}

__global__ void k_tile_scan(const long long* in, long long* out, long long n, const long long* partial) {
  __shared__ long long tile[SCAN_TILE];
  long long base = (long long)blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    long long idx = base + (long long)i * SCAN_THREADS + threadIdx.x;
    tile[i * SCAN_THREADS + threadIdx.x] = (idx < n) ? in[idx] : 0;
  }
  __syncthreads();
  long long s = 0;
  long long* mine = tile + threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) s += mine[i];
  long long total;
  long long run = block_excl_scan(s, &total) + partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    long long v = mine[i];
    mine[i] = run;
    run += v;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    long long idx = base + (long long)i * SCAN_THREADS + threadIdx.x;
    if (idx < n) out[idx] = tile[i * SCAN_THREADS + threadIdx.x];
  }
}

// exclusive scan of n int64 values in place; `tmp` must hold ceil(n / SCAN_TILE) entries
ss_status excl_scan(long long* data, long long n, long long* tmp, cudaStream_t st) {
  if (n <= 0) return SS_OK;
  long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_tile_sum<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(data, n, tmp);
  k_scan_partials<<<1, 1024, 0, st>>>(tmp, (int)ntiles);
  k_tile_scan<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(data, data, n, tmp);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, int32 value), 8-bit digits
// ---------------------------------------------------------------------------

__global__ void k_rs_hist(const unsigned long long* keys, int n, int shift, long long* hist, int nblk) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    long long idx = base + (long long)i * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long* kin, const int* vin, unsigned long long* kout,
                             int* vout, int n, int shift, const long long* offs, int nblk) {
  __shared__ long long base[256];
  __shared__ unsigned running[256];
  __shared__ unsigned wcnt[RS_THREADS / 32][256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base[t] = offs[(long long)t * nblk + blockIdx.x];
  running[t] = 0;
#pragma unroll
  for (int i = 0; i < RS_THREADS / 32; ++i) wcnt[i][t] = 0;
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  long long tile = (long long)blockIdx.x * RS_TILE;
  for (int i = 0; i < RS_ITEMS; ++i) {
    long long idx = tile + (long long)i * RS_THREADS + t;
    bool valid = idx < n;
    unsigned long long key = valid ? kin[idx] : 0ull;
    int val = valid ? vin[idx] : 0;
    unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 0xffffffffu;
    unsigned peers = __match_any_sync(SS_FULL_MASK, d);
    unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned before = running[d];
      for (int ww = 0; ww < w; ++ww) before += wcnt[ww][d];
      long long pos = base[d] + before + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    unsigned add = 0;
#pragma unroll
    for (int ww = 0; ww < RS_THREADS / 32; ++ww) {
      add += wcnt[ww][t];
      wcnt[ww][t] = 0;
    }
    running[t] += add;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Builder kernels
// ---------------------------------------------------------------------------
__global__ void k_degrees(const long long* row_ptr, int n, int* deg, int* maxdeg) {
  int m = 0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int d = (int)(row_ptr[v + 1] - row_ptr[v]);
    deg[v] = d;
    m = max(m, d);
  }
  m = __reduce_max_sync(SS_FULL_MASK, m);
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, m);
}

__global__ void k_make_keys(const int* deg, int n, int sigma, int maxdeg, int dbits,
                            unsigned long long* keys, int* vals) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    unsigned long long win = (unsigned long long)(v / sigma);
    // a degree above maxdeg (possible only for inputs that break the caller's
    // contract) is clamped so that it cannot spill into the window bits
    keys[v] = (win << dbits) | (unsigned long long)(maxdeg - min(deg[v], maxdeg));
    vals[v] = (int)v;
  }
}

__global__ void k_identity(int* vals, int n) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    vals[v] = (int)v;
}

// perm (padded), invperm, per-row degree
__global__ void k_perm_tables(const int* sorted_vals, const int* deg, int n, int n_pad, int* perm,
                              int* invperm, int* rdeg) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_pad;
       r += (long long)gridDim.x * blockDim.x) {
    if (r < n) {
      int v = sorted_vals[r];
      perm[r] = v;
      invperm[v] = (int)r;
      rdeg[r] = deg[v];
    } else {
      perm[r] = -1;
      rdeg[r] = 0;
    }
  }
}

// cl[i] = longest row of chunk i; cs[i] = C * cl[i] (scanned afterwards); cs[n_c] = 0
__global__ void k_chunk_len(const int* rdeg, int n_c, int C, int* cl, long long* cs) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n_c;
       i += (long long)gridDim.x * blockDim.x) {
    if (i == n_c) {
      cs[i] = 0;
      continue;
    }
    int m = 0;
    for (int l = 0; l < C; ++l) m = max(m, rdeg[i * C + l]);
    cl[i] = m;
    cs[i] = (long long)C * m;
  }
}

// items per chunk for a given width W (0 = one item per chunk); split flags
__global__ void k_item_count(const int* cl, int n_c, int W, long long* cnt, long long* split_flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n_c;
       i += (long long)gridDim.x * blockDim.x) {
    if (i == n_c) {
      cnt[i] = 0;
      if (split_flag) split_flag[i] = 0;
      continue;
    }
    int L = cl[i];
    bool split = (W > 0 && L > W);
    cnt[i] = (L == 0) ? 0 : (split ? (L + W - 1) / W : 1);  // chunks of isolated rows get no item
    if (split_flag) split_flag[i] = split ? 1 : 0;
  }
}

__global__ void k_item_fill(const int* cl, int n_c, int W, const long long* off,
                            const long long* split_idx, int4* items, int* split_n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_c;
       i += (long long)gridDim.x * blockDim.x) {
    int L = cl[i];
    long long o = off[i];
    if (W > 0 && L > W) {
      int cnt = (L + W - 1) / W;
      int s = split_idx ? (int)split_idx[i] : -1;
      for (int q = 0; q < cnt; ++q) items[o + q] = make_int4((int)i, q * W, min((q + 1) * W, L), s);
      if (split_n && s >= 0) split_n[s] = cnt;
    } else if (L > 0) {
      items[o] = make_int4((int)i, 0, L, -1);
    }
  }
}

// one warp per item: col[cs_i + j*C + l] for slots j0*C .. j1*C of the chunk
__global__ void k_pack(const int4* items, int n_items, const long long* cs, int C, const int* perm,
                       const int* invperm, const int* rdeg, const long long* row_ptr,
                       const int* csr_col, int* col) {
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = wid; it < n_items; it += nw) {
    int4 item = items[it];
    const long long c0 = cs[item.x];
    const long long s_end = (long long)item.z * C;
    for (long long s = (long long)item.y * C + lane; s < s_end; s += 32) {
      int j = (int)(s / C), l = (int)(s % C);
      long long r = (long long)item.x * C + l;
      int v = perm[r];
      int out = -1;
      if (v >= 0 && j < rdeg[r]) out = invperm[csr_col[row_ptr[v + 1] - 1 - j]];
      col[c0 + s] = out;
    }
  }
}

static int bit_width(unsigned long long x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// build an item table of width W; returns the item count through *n_items_out
static ss_status make_items(slimsell_graph* h, int W, long long* tmp_cnt, long long* tmp_flag,
                            long long* tmp_scan, int4** items_out, int* n_items_out, int** split_n_out,
                            int* n_split_out, bool owned, cudaStream_t st) {
  const int n_c = h->n_c;
  const int grid = 4 * h->num_sms;
  k_item_count<<<grid, 256, 0, st>>>(h->cl, n_c, W, tmp_cnt, split_n_out ? tmp_flag : nullptr);
  SS_CUDA(cudaGetLastError());
  ss_status s = excl_scan(tmp_cnt, n_c + 1, tmp_scan, st);
  if (s != SS_OK) return s;
  if (split_n_out) {
    s = excl_scan(tmp_flag, n_c + 1, tmp_scan, st);
    if (s != SS_OK) return s;
  }
  long long nitems = 0, nsplit = 0;
  SS_CUDA(cudaMemcpyAsync(&nitems, tmp_cnt + n_c, sizeof(long long), cudaMemcpyDeviceToHost, st));
  if (split_n_out)
    SS_CUDA(cudaMemcpyAsync(&nsplit, tmp_flag + n_c, sizeof(long long), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  if (nitems > 0x7fffffffLL) {
    set_error("too many work items (%lld)", nitems);
    return SS_ERR_UNSUPPORTED;
  }
  int4* items = nullptr;
  s = dmalloc(owned ? h : nullptr, (void**)&items, sizeof(int4) * (size_t)nitems);
  if (s != SS_OK) return s;
  int* split_n = nullptr;
  if (split_n_out) {
    s = dmalloc(h, (void**)&split_n, sizeof(int) * (size_t)(nsplit > 0 ? nsplit : 1));
    if (s != SS_OK) {
      cudaFree(items);
      return s;
    }
  }
  k_item_fill<<<grid, 256, 0, st>>>(h->cl, n_c, W, tmp_cnt, split_n_out ? tmp_flag : nullptr, items,
                                    split_n);
  SS_CUDA(cudaGetLastError());
  *items_out = items;
  *n_items_out = (int)nitems;
  if (split_n_out) {
    *split_n_out = split_n;
    *n_split_out = (int)nsplit;
  }
  return SS_OK;
}

// Order the BFS work items for the iteration kernels, whose warp w takes items
// w, w + W, w + 2W, ... (W = warps in the grid): items are sorted by estimated
// cost (slots plus a fixed per-item overhead), largest first, and every other
// group of W items is reversed ("snake" order) so each warp's total is balanced.
static ss_status order_items(slimsell_graph* h, cudaStream_t st) {
  const int n = h->n_items;
  if (n <= 1) return SS_OK;
  std::vector<int4> items((size_t)n), out((size_t)n);
  SS_CUDA(cudaMemcpyAsync(items.data(), h->items, sizeof(int4) * (size_t)n, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> idx((size_t)n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  const long long C = h->C, overhead = 24LL * h->C;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    return (items[a].z - items[a].y) * C + overhead > (items[b].z - items[b].y) * C + overhead;
  });
  const long long W = (long long)h->num_sms * (SS_PULL_THREADS / 32);
  for (long long p = 0; p < n; ++p) {
    const long long r = p / W, w = p % W;
    const long long round_len = std::min<long long>(W, n - r * W);
    const long long src = (r & 1) ? r * W + (round_len - 1 - w) : p;
    out[(size_t)p] = items[(size_t)idx[(size_t)src]];
  }
  SS_CUDA(cudaMemcpyAsync(h->items, out.data(), sizeof(int4) * (size_t)n, cudaMemcpyHostToDevice, st));
  SS_CUDA(cudaStreamSynchronize(st));
  return SS_OK;
}

static ss_status build_impl(slimsell_graph* h, const long long* row_ptr, const int* csr_col,
                            cudaStream_t st) {
  const int n = h->n, C = h->C;
  const int n_c = h->n_c, n_pad = h->n_pad;
  const int grid = 8 * h->num_sms;
  ss_status s;

  // temporaries
  int *deg = nullptr, *maxdeg = nullptr, *vals_a = nullptr, *vals_b = nullptr;
  unsigned long long *keys_a = nullptr, *keys_b = nullptr;
  long long *hist = nullptr, *tmp_scan = nullptr, *tmp_cnt = nullptr, *tmp_flag = nullptr;
  int4* pack_items = nullptr;
  int n_pack_items = 0;
  auto cleanup = [&]() {
    cudaFree(deg); cudaFree(maxdeg); cudaFree(vals_a); cudaFree(vals_b);
    cudaFree(keys_a); cudaFree(keys_b); cudaFree(hist); cudaFree(tmp_scan);
    cudaFree(tmp_cnt); cudaFree(tmp_flag); cudaFree(pack_items);
  };
#define SS_TRY(x)            \
  do {                       \
    s = (x);                 \
    if (s != SS_OK) {        \
      cleanup();             \
      return s;              \
    }                        \
  } while (0)
#define SS_TRYC(x) SS_TRY(((x) == cudaSuccess) ? SS_OK : cuda_fail(cudaGetLastError(), #x))

  const int nblk = (n + RS_TILE - 1) / RS_TILE;
  const long long scan_len = std::max<long long>((long long)256 * nblk, (long long)n_c + 1);
  SS_TRY(dmalloc(nullptr, (void**)&deg, sizeof(int) * (size_t)n));
  SS_TRY(dmalloc(nullptr, (void**)&maxdeg, sizeof(int)));
  SS_TRY(dmalloc(nullptr, (void**)&vals_a, sizeof(int) * (size_t)n));
  SS_TRY(dmalloc(nullptr, (void**)&vals_b, sizeof(int) * (size_t)n));
  SS_TRY(dmalloc(nullptr, (void**)&keys_a, sizeof(unsigned long long) * (size_t)n));
  SS_TRY(dmalloc(nullptr, (void**)&keys_b, sizeof(unsigned long long) * (size_t)n));
  SS_TRY(dmalloc(nullptr, (void**)&hist, sizeof(long long) * (size_t)256 * nblk));
  SS_TRY(dmalloc(nullptr, (void**)&tmp_scan, sizeof(long long) * (size_t)(scan_len / SCAN_TILE + 2)));
  SS_TRY(dmalloc(nullptr, (void**)&tmp_cnt, sizeof(long long) * (size_t)(n_c + 1)));
  SS_TRY(dmalloc(nullptr, (void**)&tmp_flag, sizeof(long long) * (size_t)(n_c + 1)));

  // permanent layout arrays
  SS_TRY(dmalloc(h, (void**)&h->perm, sizeof(int) * (size_t)n_pad));
  SS_TRY(dmalloc(h, (void**)&h->invperm, sizeof(int) * (size_t)n));
  SS_TRY(dmalloc(h, (void**)&h->rdeg, sizeof(int) * (size_t)n_pad));
  SS_TRY(dmalloc(h, (void**)&h->cl, sizeof(int) * (size_t)n_c));
  SS_TRY(dmalloc(h, (void**)&h->cs, sizeof(long long) * (size_t)(n_c + 1)));

  // 1. degrees and sort keys
  SS_TRYC(cudaMemsetAsync(maxdeg, 0, sizeof(int), st));
  k_degrees<<<grid, 256, 0, st>>>(row_ptr, n, deg, maxdeg);
  int h_maxdeg = 0;
  SS_TRYC(cudaMemcpyAsync(&h_maxdeg, maxdeg, sizeof(int), cudaMemcpyDeviceToHost, st));
  SS_TRYC(cudaStreamSynchronize(st));
  h->max_degree = h_maxdeg;

  // 2. sigma-window sort by descending degree (stable: ties keep ascending id)
  int* sorted = vals_a;
  if (h->sigma <= 1) {
    k_identity<<<grid, 256, 0, st>>>(vals_a, n);
  } else {
    const int sigma = h->sigma >= n ? n : h->sigma;  // already a multiple of C (or >= n)
    const int dbits = bit_width((unsigned long long)h_maxdeg);
    const long long nwin = ((long long)n + sigma - 1) / sigma;
    const int wbits = bit_width((unsigned long long)(nwin - 1));
    const int bits = dbits + wbits;
    k_make_keys<<<grid, 256, 0, st>>>(deg, n, sigma, h_maxdeg, dbits, keys_a, vals_a);
    unsigned long long *kin = keys_a, *kout = keys_b;
    int *vin = vals_a, *vout = vals_b;
    for (int shift = 0; shift < bits; shift += 8) {
      k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(kin, n, shift, hist, nblk);
      SS_TRY(excl_scan(hist, (long long)256 * nblk, tmp_scan, st));
      k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblk);
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    sorted = vin;
  }
  SS_TRYC(cudaGetLastError());

  // 3. perm / invperm / row degrees, chunk lengths and starts
  k_perm_tables<<<grid, 256, 0, st>>>(sorted, deg, n, n_pad, h->perm, h->invperm, h->rdeg);
  k_chunk_len<<<grid, 256, 0, st>>>(h->rdeg, n_c, C, h->cl, h->cs);
  SS_TRYC(cudaGetLastError());
  SS_TRY(excl_scan(h->cs, n_c + 1, tmp_scan, st));
  long long slots = 0;
  SS_TRYC(cudaMemcpyAsync(&slots, h->cs + n_c, sizeof(long long), cudaMemcpyDeviceToHost, st));
  SS_TRYC(cudaStreamSynchronize(st));
  h->slots = slots;

  // 4. item tables
  SS_TRY(make_items(h, 256, tmp_cnt, tmp_flag, tmp_scan, &pack_items, &n_pack_items, nullptr,
                    nullptr, false, st));
  SS_TRY(make_items(h, h->split_w, tmp_cnt, tmp_flag, tmp_scan, &h->items, &h->n_items, &h->split_n,
                    &h->n_split, true, st));
  SS_TRY(order_items(h, st));

  // 5. pack
  SS_TRY(dmalloc(h, (void**)&h->col, sizeof(int) * (size_t)(slots > 0 ? slots : 1)));
  k_pack<<<grid, 256, 0, st>>>(pack_items, n_pack_items, h->cs, C, h->perm, h->invperm, h->rdeg,
                               row_ptr, csr_col, h->col);
  SS_TRYC(cudaGetLastError());
  SS_TRYC(cudaStreamSynchronize(st));
  cleanup();
#undef SS_TRY
#undef SS_TRYC
  return SS_OK;
}

static ss_status alloc_state(slimsell_graph* h) {
  ss_status s;
  const size_t np = (size_t)h->n_pad;
  // bitmap words rounded up to whole int4 groups, plus one spare group
  h->fb_words = (long long)((((np + 31) / 32) + 3) / 4 * 4 + 4);
  if ((s = dmalloc(h, (void**)&h->lvl, sizeof(int) * np)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->act, (size_t)h->n_c)) != SS_OK) return s;
  for (int b = 0; b < 2; ++b)
    if ((s = dmalloc(h, (void**)&h->fb[b], sizeof(unsigned) * (size_t)h->fb_words)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->fr, sizeof(float) * np)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->par, sizeof(int) * np)) != SS_OK) return s;
  const size_t ns = (size_t)(h->n_split > 0 ? h->n_split : 1);
  if ((s = dmalloc(h, (void**)&h->xacc, sizeof(float) * ns * h->C)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->xpar, sizeof(int) * ns * h->C)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->arrive, sizeof(unsigned) * ns)) != SS_OK) return s;
  h->units_cap = (long long)np + h->nnz / 256 + 1024;  // any frontier fits
  if ((s = dmalloc(h, (void**)&h->units, sizeof(int2) * (size_t)h->units_cap)) != SS_OK) return s;
  // block units cover PUSH_BLOCK_SLOTS / C columns each: at most one partial unit per chunk
  h->bunits_cap = (long long)h->n_c + h->slots / PUSH_BLOCK_SLOTS + 1024;
  if ((s = dmalloc(h, (void**)&h->bunits, sizeof(int2) * (size_t)h->bunits_cap)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->pbest, sizeof(int) * np)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->psum, sizeof(float) * np)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->touched, sizeof(unsigned) * (size_t)h->fb_words)) != SS_OK) return s;
  for (int b = 0; b < 2; ++b) {
    if ((s = dmalloc(h, (void**)&h->qlist[b], sizeof(int) * np)) != SS_OK) return s;
    if ((s = dmalloc(h, (void**)&h->qdeg[b], sizeof(int) * SS_LOCAL_LIST_CAP)) != SS_OK) return s;
    if ((s = dmalloc(h, (void**)&h->qbase[b], sizeof(long long) * SS_LOCAL_LIST_CAP)) != SS_OK) return s;
    if ((s = dmalloc(h, (void**)&h->qorig[b], sizeof(int) * SS_LOCAL_LIST_CAP)) != SS_OK) return s;
  }
  if ((s = dmalloc(h, (void**)&h->qovf, sizeof(int) * SS_LOCAL_LIST_CAP)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->qovf_n, 2 * sizeof(unsigned long long))) != SS_OK) return s;
  SS_CUDA(cudaMemset(h->qovf_n, 0, 2 * sizeof(unsigned long long)));
  h->local_cluster = push_local_cluster_size();
  if (h->local_cluster <= 0) {
    set_error("slimsell_build: no thread-block cluster of the push kernel fits on this device");
    return SS_ERR_CUDA;
  }
  SS_CUDA(cudaMemset(h->pbest, 0xff, sizeof(int) * np));
  SS_CUDA(cudaMemset(h->psum, 0, sizeof(float) * np));
  SS_CUDA(cudaMemset(h->touched, 0, sizeof(unsigned) * (size_t)h->fb_words));
  if ((s = dmalloc(h, (void**)&h->ctl, sizeof(Ctl))) != SS_OK) return s;
  h->iter_cap = 1 << 16;
  if ((s = dmalloc(h, (void**)&h->feats, sizeof(float) * SS_SELECTOR_FEATURES * (size_t)h->iter_cap)) != SS_OK)
    return s;
  if ((s = dmalloc(h, (void**)&h->iters, sizeof(ss_iter_stats) * (size_t)h->iter_cap)) != SS_OK) return s;
  if ((s = dmalloc(h, (void**)&h->lstat, sizeof(unsigned long long) * SS_LSTAT * (size_t)h->iter_cap)) != SS_OK)
    return s;
  SS_CUDA(cudaMemset(h->arrive, 0, sizeof(unsigned) * ns));
  SS_CUDA(cudaMemset(h->fb[0], 0, sizeof(unsigned) * (size_t)h->fb_words));
  SS_CUDA(cudaMemset(h->fb[1], 0, sizeof(unsigned) * (size_t)h->fb_words));
  SS_CUDA(cudaHostAlloc((void**)&h->h_ctl, sizeof(Ctl), cudaHostAllocDefault));
  SS_CUDA(cudaEventCreate(&h->ev_a));
  SS_CUDA(cudaEventCreate(&h->ev_b));
  SS_CUDA(cudaEventCreate(&h->ev_c));
  SS_CUDA(cudaEventCreate(&h->ev_d));
  SS_CUDA(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  SS_CUDA(cudaMemset(h->ctl, 0, sizeof(Ctl)));
  return SS_OK;
}

void ab_release(slimsell_graph* h);  // format-comparison scratch (ss_sell.cu)
void bc_release(slimsell_graph* h);  // betweenness-centrality scratch (ss_bc.cu)

void free_handle(slimsell_graph* h) {
  if (!h) return;
  ab_release(h);
  bc_release(h);
  void* ptrs[] = {h->perm, h->invperm, h->rdeg, h->cl, h->cs, h->col, h->items, h->split_n,
                  h->lvl, h->act, h->fb[0], h->fb[1], h->fr, h->par, h->xacc, h->xpar,
                  h->arrive, h->ctl, h->iters, h->units, h->bunits, h->pbest,
                  h->psum, h->touched, h->qlist[0], h->qlist[1], h->qdeg[0], h->qdeg[1], h->qbase[0],
                  h->qbase[1], h->qorig[0], h->qorig[1], h->qovf, h->qovf_n, h->lstat, h->mlp, h->feats, h->mF[0],
                  h->mF[1], h->mV, h->mxacc, h->mroots};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->ev_c) cudaEventDestroy(h->ev_c);
  if (h->ev_d) cudaEventDestroy(h->ev_d);
  for (cudaEvent_t e : h->evq) cudaEventDestroy(e);
  if (h->ev_done) {
    cudaEventSynchronize(h->ev_done);
    cudaEventDestroy(h->ev_done);
  }
  for (auto& row : h->loop_exec)
    for (auto& e : row)
      if (e) cudaGraphExecDestroy(e);
  delete h;
}

}  // namespace ss

ss::Dev slimsell_graph::dev() const {
  ss::Dev d;
  d.n = n; d.C = C; d.n_c = n_c; d.n_pad = n_pad; d.n_items = n_items; d.n_split = n_split;
  d.perm = perm; d.invperm = invperm; d.rdeg = rdeg; d.cl = cl; d.cs = cs; d.col = col;
  d.items = items; d.split_n = split_n; d.lvl = lvl; d.act = act;
  d.fb[0] = fb[0]; d.fb[1] = fb[1]; d.fb_words = fb_words;
  // staged prefix: whole int4 groups, never past the allocated bitmap
  long long need = ((((long long)n_pad + 31) / 32) + 3) / 4 * 4;
  long long cap = (long long)(smem_bytes / 16) * 4;
  d.smem_words = (int)(need < cap ? need : cap);
  d.fr = fr; d.par = par; d.xacc = xacc; d.xpar = xpar; d.arrive = arrive;
  d.units = units; d.units_cap = units_cap;
  d.bunits = bunits; d.bunits_cap = bunits_cap; d.push_blocks = push_blocks;
  d.format = SS_FORMAT_SLIMSELL; d.scol = nullptr; d.sval = nullptr;  // set per call by slimsell_bfs
  d.pbest = pbest; d.psum = psum; d.touched = touched; d.mlp = mlp; d.feats = feats;
  d.sel_margin = sel_margin;
  for (int b = 0; b < 2; ++b) {
    d.qlist[b] = qlist[b]; d.qdeg[b] = qdeg[b]; d.qbase[b] = qbase[b]; d.qorig[b] = qorig[b];
  }
  d.qovf = qovf; d.qovf_n = qovf_n;
  d.local_cluster = local_cluster;
  d.local_max_nf = (long long)local_cluster * SS_LOCAL_SLICE;
  d.local_max_e = (long long)local_cluster * SS_LOCAL_EDGES_PER_CTA;
  d.nnz = nnz; d.total_slots = slots; d.reach_cap = (unsigned long long)n;
  d.ctl = ctl; d.iters = iters; d.iter_cap = iter_cap; d.lstat = lstat;
  return d;
}

extern "C" {

ss_status slimsell_build(const int64_t* d_row_ptr, const int32_t* d_col, int32_t n, int64_t nnz,
                         int32_t C, int32_t sigma, int32_t split_w, void* stream,
                         slimsell_handle* out) {
  ss::set_error("");
  if (!out) {
    ss::set_error("slimsell_build: out is NULL");
    return SS_ERR_INVALID;
  }
  *out = nullptr;
  if (n < 1 || nnz < 0 || !d_row_ptr || (nnz > 0 && !d_col)) {
    ss::set_error("slimsell_build: bad graph arguments (n=%d nnz=%lld)", n, (long long)nnz);
    return SS_ERR_INVALID;
  }
  if (!(C == 8 || C == 16 || C == 32 || C == 64)) {
    ss::set_error("slimsell_build: C must be 8, 16, 32 or 64 (got %d)", C);
    return SS_ERR_INVALID;
  }
  if (sigma < 1 || split_w < 0) {
    ss::set_error("slimsell_build: sigma must be >= 1 and split_w >= 0");
    return SS_ERR_INVALID;
  }
  long long n_c = ((long long)n + C - 1) / C;
  if (n_c * C > 0x7fffffffLL) {
    ss::set_error("slimsell_build: n too large for int32 row ids");
    return SS_ERR_UNSUPPORTED;
  }
  slimsell_graph* h = new slimsell_graph();
  cudaStream_t st = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->n = n;
  h->nnz = nnz;
  h->C = C;
  // sigma > 1 is rounded up to a multiple of C (the paper takes it as one, Section IV)
  h->sigma = sigma <= 1 ? 1 : (int)std::min<long long>(((long long)sigma + C - 1) / C * C, INT_MAX);
  h->split_w = split_w;
  h->n_c = (int)n_c;
  h->n_pad = (int)(n_c * C);
  ss_status s = ss::build_impl(h, (const long long*)d_row_ptr, d_col, st);
  if (s == SS_OK) s = ss::alloc_state(h);
  if (s != SS_OK) {
    ss::free_handle(h);
    return s;
  }
  *out = h;
  return SS_OK;
}

const char* slimsell_last_error(void) { return ss::last_error(); }

const char* slimsell_version(void) { return "slimsell-gb300 0.1 (sm_103a)"; }

void slimsell_destroy(slimsell_handle h) { ss::free_handle(h); }

ss_status slimsell_get_info(slimsell_handle h, ss_info* out) {
  if (!h || !out) {
    ss::set_error("slimsell_get_info: NULL argument");
    return SS_ERR_INVALID;
  }
  out->n = h->n; out->C = h->C; out->sigma = h->sigma; out->split_w = h->split_w;
  out->n_chunks = h->n_c; out->n_items = h->n_items; out->n_split_chunks = h->n_split;
  out->max_degree = h->max_degree; out->nnz = h->nnz; out->slots = h->slots;
  out->padding = h->slots - h->nnz; out->device_bytes = h->device_bytes;
  return SS_OK;
}

ss_status slimsell_export_layout(slimsell_handle h, int32_t* d_perm, int32_t* d_cl, int64_t* d_cs,
                                 int32_t* d_col, int32_t* d_items, void* stream) {
  if (!h) {
    ss::set_error("slimsell_export_layout: NULL handle");
    return SS_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (d_perm) SS_CUDA(cudaMemcpyAsync(d_perm, h->perm, sizeof(int) * (size_t)h->n_pad, cudaMemcpyDeviceToDevice, st));
  if (d_cl) SS_CUDA(cudaMemcpyAsync(d_cl, h->cl, sizeof(int) * (size_t)h->n_c, cudaMemcpyDeviceToDevice, st));
  if (d_cs) SS_CUDA(cudaMemcpyAsync(d_cs, h->cs, sizeof(long long) * (size_t)(h->n_c + 1), cudaMemcpyDeviceToDevice, st));
  if (d_col && h->slots > 0) SS_CUDA(cudaMemcpyAsync(d_col, h->col, sizeof(int) * (size_t)h->slots, cudaMemcpyDeviceToDevice, st));
  if (d_items && h->n_items > 0) SS_CUDA(cudaMemcpyAsync(d_items, h->items, sizeof(int4) * (size_t)h->n_items, cudaMemcpyDeviceToDevice, st));
  SS_CUDA(cudaStreamSynchronize(st));
  return SS_OK;
}

}  // extern "C"
