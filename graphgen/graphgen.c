/*
 * Seeded synthetic graph inputs for SlimSell BFS (input preparation only).
 *
 * This module produces the cleaned, symmetric CSR graphs that both the CPU
 * oracle and the GPU library consume.  It contains none of the BFS method's
 * arithmetic: only random edge generation, label permutation, and the
 * symmetrise / drop-self-loop / deduplicate / CSR conversion that the
 * evaluation applies to every input (Section IV, "Selection of Benchmarks":
 * Kronecker and Erdos-Renyi graphs; lattices stand in for the high-diameter
 * road network of Table "graphs").
 *
 * Random numbers come from a counter-based generator built on the SplitMix64
 * output function (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): value(key, i) = mix64(key + (i + 1) * gamma).
 * Every draw is addressed by (seed, stream, counter), so the graphs are
 * identical for any thread count and on any host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9e3779b97f4a7c15ULL

enum {
  GG_STREAM_KRON = 1,
  GG_STREAM_PERM = 2,
  GG_STREAM_LATTICE = 3,
  GG_STREAM_ER = 4,
  GG_STREAM_ROOT = 5
};

static inline uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Key of one (seed, stream) pair: a SplitMix64 output of the seed, offset by stream. */
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix64(seed * GG_GAMMA + stream * 0xd1b54a32d192ed03ULL);
}

uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return gg_mix64(gg_key(seed, stream) + (ctr + 1) * GG_GAMMA);
}

static inline double gg_unit(uint64_t h) { /* uniform in [0, 1) with 53 bits */
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Kronecker (R-MAT style) edges: 2^scale vertices, edgefactor * 2^scale edges.
 * For every edge and every bit level the quadrant is drawn with probabilities
 * (a, b, c, 1 - a - b - c); bit level l of (src, dst) is set from that quadrant.
 */
int gg_kronecker_edges(int32_t scale, int64_t m, double a, double b, double c,
                       uint64_t seed, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || m < 0) return -1;
  const uint64_t key = gg_key(seed, GG_STREAM_KRON);
  const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    uint32_t u = 0, v = 0;
    for (int32_t l = 0; l < scale; ++l) {
      double r = gg_unit(gg_mix64(key + ((uint64_t)e * 64u + (uint64_t)l + 1u) * GG_GAMMA));
      uint32_t bu, bv;
      if (r < a) { bu = 0; bv = 0; }
      else if (r < ab) { bu = 0; bv = 1; }
      else if (r < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u |= bu << l;
      v |= bv << l;
    }
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
  }
  return 0;
}

/* Seeded uniform random permutation of [0, n) (Fisher-Yates, counter-addressed draws). */
int gg_permutation(int32_t n, uint64_t seed, int32_t* perm) {
  if (n < 0) return -1;
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  const uint64_t key = gg_key(seed, GG_STREAM_PERM);
  for (int64_t i = (int64_t)n - 1; i > 0; --i) {
    uint64_t h = gg_mix64(key + ((uint64_t)i + 1u) * GG_GAMMA);
    int64_t j = (int64_t)(h % (uint64_t)(i + 1));
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  return 0;
}

/*
 * L x L four-neighbour lattice, vertex (i, j) -> i * L + j.  Each of the
 * 2 L (L - 1) edges is deleted independently with probability p_del.
 * Returns the number of kept edges (written to src/dst, capacity 2L(L-1)).
 */
int64_t gg_lattice_edges(int32_t L, double p_del, uint64_t seed, int32_t* src, int32_t* dst) {
  if (L < 1) return -1;
  const uint64_t key = gg_key(seed, GG_STREAM_LATTICE);
  const int64_t nh = (int64_t)L * (L - 1);
  int64_t kept = 0;
  for (int64_t e = 0; e < 2 * nh; ++e) {
    double r = gg_unit(gg_mix64(key + ((uint64_t)e + 1u) * GG_GAMMA));
    if (r < p_del) continue;
    int64_t u, v;
    if (e < nh) { /* horizontal (i, j) - (i, j + 1) */
      int64_t i = e / (L - 1), j = e % (L - 1);
      u = i * L + j; v = u + 1;
    } else {      /* vertical (i, j) - (i + 1, j) */
      int64_t f = e - nh;
      int64_t i = f / L, j = f % L;
      u = i * L + j; v = u + L;
    }
    src[kept] = (int32_t)u;
    dst[kept] = (int32_t)v;
    ++kept;
  }
  return kept;
}

/* Erdos-Renyi G(n, M): M endpoint pairs drawn uniformly (cleaned later). */
int gg_er_edges(int32_t n, int64_t M, uint64_t seed, int32_t* src, int32_t* dst) {
  if (n < 1 || M < 0) return -1;
  const uint64_t key = gg_key(seed, GG_STREAM_ER);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    uint64_t h0 = gg_mix64(key + ((uint64_t)(2 * e) + 1u) * GG_GAMMA);
    uint64_t h1 = gg_mix64(key + ((uint64_t)(2 * e + 1) + 1u) * GG_GAMMA);
    src[e] = (int32_t)(h0 % (uint64_t)n);
    dst[e] = (int32_t)(h1 % (uint64_t)n);
  }
  return 0;
}

static int gg_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void gg_sort_row(int32_t* p, int64_t len) {
  if (len <= 24) { /* insertion sort for the many short rows */
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > x) { p[j + 1] = p[j]; --j; }
      p[j + 1] = x;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), gg_cmp_i32);
  }
}

/*
 * Edge list -> cleaned symmetric CSR.  Optional relabel[old] = new is applied
 * to both endpoints; self-loops are dropped; both directions are inserted;
 * duplicates are removed; each row is sorted by ascending neighbour id.
 * row_ptr has n + 1 entries; col_out has capacity col_cap.
 * Returns nnz (directed entries), or -1 on bad arguments, -2 on OOM,
 * -3 if col_cap is too small.
 */
int64_t gg_edges_to_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const int32_t* relabel, int64_t* row_ptr, int32_t* col_out,
                        int64_t col_cap) {
  if (n < 0 || m < 0) return -1;
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= n || v >= n) continue;
    if (relabel) { u = relabel[u]; v = relabel[v]; }
    if (u == v) continue;
    __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
  }
  int64_t* start = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!start) { free(deg); return -2; }
  start[0] = 0;
  for (int32_t v = 0; v < n; ++v) start[v + 1] = start[v] + deg[v];
  const int64_t total = start[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!tmp) { free(deg); free(start); return -2; }
  for (int32_t v = 0; v < n; ++v) deg[v] = start[v]; /* reuse as cursor */
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= n || v >= n) continue;
    if (relabel) { u = relabel[u]; v = relabel[v]; }
    if (u == v) continue;
    int64_t pu = __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
    int64_t pv = __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
    tmp[pu] = v;
    tmp[pv] = u;
  }
  /* sort + dedup every row; deg[v] becomes the unique count */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t v = 0; v < n; ++v) {
    int32_t* p = tmp + start[v];
    int64_t len = start[v + 1] - start[v];
    gg_sort_row(p, len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i)
      if (w == 0 || p[i] != p[w - 1]) p[w++] = p[i];
    deg[v] = w;
  }
  row_ptr[0] = 0;
  for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + deg[v];
  const int64_t nnz = row_ptr[n];
  if (nnz > col_cap) { free(deg); free(start); free(tmp); return -3; }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t v = 0; v < n; ++v)
    memcpy(col_out + row_ptr[v], tmp + start[v], (size_t)deg[v] * sizeof(int32_t));
  free(deg);
  free(start);
  free(tmp);
  return nnz;
}

int gg_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
