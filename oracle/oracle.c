/*
 * CPU ORACLE for SlimSell BFS -- test infrastructure only.
 *
 * Plain, serial, deliberately unoptimised restatements of what the method
 * computes.  Only the tests, the smoke check and the benchmark's CPU baseline
 * use this file; the GPU library shares no code with it.
 *
 *   oracle_bfs_queue     traditional queue BFS (Section II-C, "Traditional BFS")
 *   oracle_dp            DP transformation p = DP(d) (Section II-C): parent of v
 *                        is a neighbour w with d[w] = d[v] - 1; ties go to the
 *                        largest vertex id (the paper leaves the choice open).
 *   oracle_bfs_semiring  algebraic BFS x_k = A (x) f_{k-1} over one of the four
 *                        semirings of Section III-A, with dense vectors over the
 *                        plain CSR (no chunking, no sorting), in the paper's order:
 *                        tropical  (Section III-A1): f_k = x_k = A' (x)_T f_{k-1}
 *                        real      (Section III-A2): f_k = x_k (.) g_k,
 *                                  g_k = not(sum_{l<k} f_l)
 *                        boolean   (Section III-A3): f_k = x_k and g_k
 *                        sel-max   (Section III-A4): x_k = A (x) x_{k-1},
 *                                  f_k = nn(x_k) - g_k, p_k = p_{k-1} + not(p_{k-1}) (.) x_k,
 *                                  then x_k = nn(x_k) (.) (1..n)
 *   oracle_bfs_multi     k independent queue BFS runs (multi-source extension).
 *   oracle_bc            betweenness centrality summed over a set of sources, by
 *                        Brandes' dependency accumulation (the "other algorithms"
 *                        the paper names as future work in its conclusion): for each
 *                        source s, a queue BFS counts shortest paths sigma_s, then
 *                        in reverse BFS order
 *                        delta_s(v) = sum over neighbours w with d(w) = d(v) + 1 of
 *                                     sigma_s(v) / sigma_s(w) * (1 + delta_s(w)),
 *                        and bc(v) += delta_s(v) for v != s.
 *
 * Floating point values (tropical distances, real-semiring path counts) are
 * fp64.  Parity status: every function here is pinned by the CPU tests
 * (brute force over all small graphs, closed forms, library routines and the
 * BFS invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_TROPICAL = 0, OR_REAL = 1, OR_BOOLEAN = 2, OR_SELMAX = 3 };

/* Traditional BFS with a FIFO queue.  dist[v] = hop count from root, -1 if unreached.
 * Returns the number of reached vertices, or -1 on a bad root. */
int64_t oracle_bfs_queue(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t root,
                         int32_t* dist) {
  if (root < 0 || root >= n) return -1;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!queue) return -2;
  for (int32_t v = 0; v < n; ++v) dist[v] = -1;
  int64_t head = 0, tail = 0;
  dist[root] = 0;
  queue[tail++] = root;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t w = col[e];
      if (dist[w] < 0) {
        dist[w] = dist[u] + 1;
        queue[tail++] = w;
      }
    }
  }
  free(queue);
  return tail;
}

/* DP transformation: parent[v] = max id w in N(v) with dist[w] == dist[v] - 1.
 * parent[root] = root; unreached vertices (dist < 0) get -1. */
void oracle_dp(int32_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* dist,
               int32_t root, int32_t* parent) {
  for (int32_t v = 0; v < n; ++v) {
    parent[v] = -1;
    if (dist[v] < 0) continue;
    if (v == root) { parent[v] = root; continue; }
    int32_t best = -1;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t w = col[e];
      if (dist[w] == dist[v] - 1 && w > best) best = w;
    }
    parent[v] = best;
  }
}

/*
 * Algebraic BFS over one semiring.  Outputs (each may be NULL):
 *   dist[n]   level at which v entered the frontier, -1 if never
 *   parent[n] sel-max: p_D - 1 (ids are stored 1-based so that 0 means "none");
 *             other semirings: DP(d); -1 if unreached
 *   fval[n]   real semiring: f_{d(v)}^v, the value carried when v entered the frontier
 *   level_counts[cap]  number of vertices entering the frontier at each level 0..
 * Returns the number of SpMV iterations performed (the last one adds no vertex),
 * or a negative value on error.
 */
int64_t oracle_bfs_semiring(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t root,
                            int32_t semiring, int32_t* dist, int32_t* parent, double* fval,
                            int64_t* level_counts, int32_t cap) {
  if (root < 0 || root >= n) return -1;
  if (semiring < 0 || semiring > 3) return -1;
  size_t N = (size_t)(n > 0 ? n : 1);
  int32_t* d = (int32_t*)malloc(sizeof(int32_t) * N);
  double* x = (double*)malloc(sizeof(double) * N);    /* x_k (tropical: also f_k) */
  double* xn = (double*)malloc(sizeof(double) * N);   /* x_{k+1} under construction */
  double* f = (double*)malloc(sizeof(double) * N);    /* f_{k} for real / boolean / sel-max */
  double* g = (double*)malloc(sizeof(double) * N);    /* filtering term */
  double* p = (double*)malloc(sizeof(double) * N);    /* sel-max parents p_k (1-based ids) */
  if (!d || !x || !xn || !f || !g || !p) {
    free(d); free(x); free(xn); free(f); free(g); free(p);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) d[v] = -1;
  if (level_counts)
    for (int32_t i = 0; i < cap; ++i) level_counts[i] = 0;

  /* initial vectors x_0, f_0 (and p_0 for sel-max) */
  for (int32_t v = 0; v < n; ++v) {
    switch (semiring) {
      case OR_TROPICAL: x[v] = (v == root) ? 0.0 : INFINITY; break;
      case OR_REAL:
      case OR_BOOLEAN: x[v] = f[v] = (v == root) ? 1.0 : 0.0; break;
      case OR_SELMAX:
        x[v] = (v == root) ? (double)(root + 1) : 0.0;
        f[v] = (v == root) ? 1.0 : 0.0;
        p[v] = x[v];
        break;
    }
    if (fval) fval[v] = 0.0;
  }
  d[root] = 0;
  if (fval && (semiring == OR_REAL || semiring == OR_BOOLEAN)) fval[root] = 1.0;
  if (level_counts && cap > 0) level_counts[0] = 1;
  /* g_1 = not(f_0): everything but the root still unvisited */
  for (int32_t v = 0; v < n; ++v) g[v] = (v == root) ? 0.0 : 1.0;

  int64_t k = 0;
  for (;;) {
    ++k;
    int64_t added = 0;
    for (int32_t v = 0; v < n; ++v) {
      double acc;
      switch (semiring) {
        case OR_TROPICAL: /* min over A'(v,u) + f_{k-1}^u; A'(v,v) = 0, A'(v,u) = 1 on edges */
          acc = x[v];
          for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            double t = x[col[e]] + 1.0;
            if (t < acc) acc = t;
          }
          break;
        case OR_REAL: /* sum over u of A(v,u) * f_{k-1}^u */
          acc = 0.0;
          for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) acc += f[col[e]];
          break;
        case OR_BOOLEAN: /* or over u of A(v,u) and f_{k-1}^u */
          acc = 0.0;
          for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (f[col[e]] != 0.0) { acc = 1.0; }
          break;
        default: /* sel-max: max over u of A(v,u) * x_{k-1}^u */
          acc = 0.0;
          for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            double t = x[col[e]];
            if (t > acc) acc = t;
          }
          break;
      }
      xn[v] = acc;
    }
    /* post-processing: derive f_k (and d, g, p) from x_k */
    for (int32_t v = 0; v < n; ++v) {
      switch (semiring) {
        case OR_TROPICAL:
          if (isinf(x[v]) && !isinf(xn[v])) { d[v] = (int32_t)xn[v]; ++added; }
          break;
        case OR_REAL:
          /* f_k = x_k (.) g_k, with the Hadamard product by a 0/1 vector taken as a select */
          f[v] = (g[v] != 0.0) ? xn[v] : 0.0;
          break;
        case OR_BOOLEAN:
          f[v] = (xn[v] != 0.0 && g[v] != 0.0) ? 1.0 : 0.0;
          break;
        default: /* sel-max */
          f[v] = (xn[v] != 0.0 && g[v] != 0.0) ? 1.0 : 0.0;
          if (p[v] == 0.0) p[v] = xn[v];                 /* p_k = p_{k-1} + not(p_{k-1}) (.) x_k */
          xn[v] = (xn[v] != 0.0) ? (double)(v + 1) : 0.0; /* x_k = nn(x_k) (.) (1..n) */
          break;
      }
      if (semiring != OR_TROPICAL && f[v] != 0.0) {
        d[v] = (int32_t)k; /* d = union / sum over l of l f_l, read as the level of entry */
        if (fval) fval[v] = (semiring == OR_REAL) ? f[v] : 1.0;
        ++added;
      }
    }
    for (int32_t v = 0; v < n; ++v) {
      x[v] = xn[v];
      if (semiring != OR_TROPICAL && f[v] != 0.0) g[v] = 0.0; /* g_{k+1} = not(sum_{l<=k} f_l) */
    }
    if (level_counts && k < cap) level_counts[k] = added;
    if (added == 0) break; /* convergence: the iteration reached no new vertex */
  }

  if (parent) {
    if (semiring == OR_SELMAX) {
      for (int32_t v = 0; v < n; ++v) parent[v] = (p[v] != 0.0) ? (int32_t)(p[v] - 1.0) : -1;
    } else {
      oracle_dp(n, row_ptr, col, d, root, parent);
    }
  }
  if (dist) memcpy(dist, d, sizeof(int32_t) * (size_t)n);
  free(d); free(x); free(xn); free(f); free(g); free(p);
  return k;
}

/* Multi-source BFS: k independent queue BFS runs; dist is k x n row-major. */
int64_t oracle_bfs_multi(int32_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* roots, int32_t k, int32_t* dist) {
  int64_t total = 0;
  for (int32_t s = 0; s < k; ++s) {
    int64_t r = oracle_bfs_queue(n, row_ptr, col, roots[s], dist + (size_t)s * (size_t)n);
    if (r < 0) return r;
    total += r;
  }
  return total;
}

/* Betweenness centrality over the given sources (Brandes): bc[v] = sum over
 * sources s and targets t != s, v of sigma_st(v) / sigma_st.  On an undirected
 * graph with every vertex as a source each unordered pair counts twice.
 * Returns 0, or -1 on a bad source. */
int32_t oracle_bc(int32_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* sources,
                  int32_t k, double* bc) {
  int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double* sigma = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* delta = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
  int32_t status = 0;
  for (int32_t q = 0; q < k; ++q) {
    const int32_t s = sources[q];
    if (s < 0 || s >= n) { status = -1; break; }
    for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0.0; delta[v] = 0.0; }
    /* forward: BFS order and shortest-path counts */
    int32_t head = 0, tail = 0;
    dist[s] = 0; sigma[s] = 1.0; order[tail++] = s;
    while (head < tail) {
      const int32_t v = order[head++];
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const int32_t w = col[e];
        if (dist[w] < 0) { dist[w] = dist[v] + 1; order[tail++] = w; }
        if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];
      }
    }
    /* backward: dependencies in reverse BFS order */
    for (int32_t i = tail - 1; i >= 0; --i) {
      const int32_t v = order[i];
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const int32_t w = col[e];
        if (dist[w] == dist[v] + 1) delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
      }
      if (v != s) bc[v] += delta[v];
    }
  }
  free(dist); free(order); free(sigma); free(delta);
  return status;
}
