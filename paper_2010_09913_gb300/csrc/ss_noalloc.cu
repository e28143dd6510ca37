// Allocation-free variant of the builder's sigma-window degree sort.
//
// Some callers cannot allocate device memory at the moment they need a layout
// order: a process whose device memory is entirely reserved by another
// allocator (a framework's caching pool) would see cudaMalloc fail, and
// latency-bound loops cannot accept the implicit device synchronisation and
// unbounded latency of cudaMalloc/cudaFree.  For them this file keeps the sort's
// scratch in one fixed device array, reserved when the library's device code is
// loaded and held on every GPU that loads it until the process exits.
#include <mutex>

#include "ss_sort.cuh"

namespace ss {
namespace {

constexpr int NOALLOC_MAX_N = 1 << 19;            // largest vertex count accepted
constexpr int NOALLOC_DBITS = 19;                 // degree < NOALLOC_MAX_N fits in 19 bits
constexpr int NOALLOC_MAX_NBLK = NOALLOC_MAX_N / RS_TILE;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_DEG = 0;
constexpr size_t OFF_KEYS_A = align256(OFF_DEG + sizeof(int) * NOALLOC_MAX_N);
constexpr size_t OFF_KEYS_B = align256(OFF_KEYS_A + sizeof(unsigned long long) * NOALLOC_MAX_N);
constexpr size_t OFF_VALS_B = align256(OFF_KEYS_B + sizeof(unsigned long long) * NOALLOC_MAX_N);
constexpr size_t OFF_HIST = align256(OFF_VALS_B + sizeof(int) * NOALLOC_MAX_N);
constexpr size_t OFF_SCAN = align256(OFF_HIST + sizeof(long long) * 256 * NOALLOC_MAX_NBLK);
constexpr size_t OFF_MAXDEG =
    align256(OFF_SCAN + sizeof(long long) * ((256 * NOALLOC_MAX_NBLK) / SCAN_TILE + 2));
constexpr size_t NOALLOC_BYTES = align256(OFF_MAXDEG + sizeof(int));  // about 12.3 MiB

// The scratch itself.  In host code this name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void* g_scratch_addr[256] = {};

// Device address of the scratch on the current device.  Outside stream capture
// it is looked up on every call: a context reset (cudaDeviceReset, or a reset of
// the primary context by the host framework) unloads the module, and the array
// may come back at another address.  While `st` is being captured the address
// of the last lookup on this device is used (capture cannot span a reset), so
// the first call on a device must come before any capture.
ss_status scratch_address(cudaStream_t st, unsigned char** out) {
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("slimsell_sigma_sort_noalloc: device index %d out of range", dev);
    return SS_ERR_UNSUPPORTED;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SS_CUDA(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  } else if (!g_scratch_addr[dev]) {
    set_error("slimsell_sigma_sort_noalloc: first call on device %d made during stream capture; "
              "call it once outside capture first", dev);
    return SS_ERR_INVALID;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return SS_OK;
}

int bit_width_u64(unsigned long long x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace
}  // namespace ss

extern "C" ss_status slimsell_sigma_sort_noalloc(const int64_t* d_row_ptr, int32_t n, int32_t sigma,
                                                 int32_t* d_perm, void* stream) {
  using namespace ss;
  set_error("");
  if (!d_row_ptr || !d_perm) {
    set_error("slimsell_sigma_sort_noalloc: NULL pointer");
    return SS_ERR_INVALID;
  }
  if (n < 1 || n > NOALLOC_MAX_N) {
    set_error("slimsell_sigma_sort_noalloc: n = %d is outside [1, %d], the size of the fixed "
              "scratch array", n, NOALLOC_MAX_N);
    return SS_ERR_INVALID;
  }
  if (sigma < 1) {
    set_error("slimsell_sigma_sort_noalloc: sigma must be >= 1");
    return SS_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ss_status s = scratch_address(st, &base);
  if (s != SS_OK) return s;
  int* deg = reinterpret_cast<int*>(base + OFF_DEG);
  unsigned long long* keys_a = reinterpret_cast<unsigned long long*>(base + OFF_KEYS_A);
  unsigned long long* keys_b = reinterpret_cast<unsigned long long*>(base + OFF_KEYS_B);
  int* vals_b = reinterpret_cast<int*>(base + OFF_VALS_B);
  long long* hist = reinterpret_cast<long long*>(base + OFF_HIST);
  long long* scan_tmp = reinterpret_cast<long long*>(base + OFF_SCAN);
  int* maxdeg = reinterpret_cast<int*>(base + OFF_MAXDEG);

  const int grid = 1024;
  if (sigma <= 1) {  // no sorting scope: identity order
    k_identity<<<grid, 256, 0, st>>>(d_perm, n);
    SS_CUDA(cudaGetLastError());
    return SS_OK;
  }
  // the shared degree kernel also folds the largest degree into `maxdeg`; this
  // call does not read it (the keys use a fixed 19-bit degree field, and
  // k_make_keys clamps degrees to it), so the slot is never cleared
  k_degrees<<<grid, 256, 0, st>>>(reinterpret_cast<const long long*>(d_row_ptr), n, deg, maxdeg);
  const int window = sigma >= n ? n : sigma;
  const long long nwin = ((long long)n + window - 1) / window;
  const int bits = NOALLOC_DBITS + bit_width_u64((unsigned long long)(nwin - 1));
  // fixed-width degree field: (2^19 - 1 - degree) orders like (max degree - degree)
  k_make_keys<<<grid, 256, 0, st>>>(deg, n, window, NOALLOC_MAX_N - 1, NOALLOC_DBITS, keys_a, d_perm);
  const int nblk = (n + RS_TILE - 1) / RS_TILE;
  unsigned long long *kin = keys_a, *kout = keys_b;
  int *vin = d_perm, *vout = vals_b;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(kin, n, shift, hist, nblk);
    s = excl_scan(hist, (long long)256 * nblk, scan_tmp, st);
    if (s != SS_OK) return s;
    k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblk);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  SS_CUDA(cudaGetLastError());
  if (vin != d_perm)
    SS_CUDA(cudaMemcpyAsync(d_perm, vin, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  return SS_OK;
}
