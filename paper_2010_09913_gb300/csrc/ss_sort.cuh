// Degree-sort building blocks of the device builder (radix sort and prefix sum),
// declared for the translation units that launch them.
#pragma once

#include "ss_common.cuh"

namespace ss {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

// exclusive prefix sum of n int64 values in place; tmp holds ceil(n / SCAN_TILE) entries
ss_status excl_scan(long long* data, long long n, long long* tmp, cudaStream_t st);

__global__ void k_rs_hist(const unsigned long long* keys, int n, int shift, long long* hist, int nblk);
__global__ void k_rs_scatter(const unsigned long long* kin, const int* vin, unsigned long long* kout,
                             int* vout, int n, int shift, const long long* offs, int nblk);
__global__ void k_degrees(const long long* row_ptr, int n, int* deg, int* maxdeg);
__global__ void k_make_keys(const int* deg, int n, int sigma, int maxdeg, int dbits,
                            unsigned long long* keys, int* vals);
__global__ void k_identity(int* vals, int n);

}  // namespace ss
