"""Pins for the CPU oracle's BFS functions (no GPU).

The oracle is checked against things other than itself:
* brute force over every labelled graph with n <= 5 (and random n = 6, 7
  graphs): distances from boolean matrix powers of (I + A), shortest-path
  counts from integer powers of A;
* closed forms: path, cycle, star, complete, complete bipartite, full lattice
  (Manhattan distances, binomial path counts, max-id parent rule);
* library routines: scipy.sparse.csgraph shortest_path / connected_components;
* the BFS invariants on Kronecker, lattice and Erdos-Renyi graphs.
"""
import itertools
from math import comb

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import graphgen as gg
import oracle

SEMIRINGS = ["tropical", "real", "boolean", "selmax"]


def adjacency(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1
    return A


def brute_force(A, r):
    """Distances from reachability powers, path counts from A^d, max-id parents."""
    n = A.shape[0]
    dist = np.full(n, -1, dtype=np.int64)
    reach = np.zeros(n, dtype=bool)
    reach[r] = True
    dist[r] = 0
    step = (A + np.eye(n, dtype=np.int64)) > 0
    for k in range(1, n + 1):
        nxt = (reach.astype(np.int64) @ step.astype(np.int64)) > 0
        dist[nxt & ~reach] = k
        if np.array_equal(nxt, reach):
            break
        reach = nxt
    counts = np.zeros(n, dtype=np.int64)
    P = np.eye(n, dtype=np.int64)
    for k in range(0, n + 1):
        sel = dist == k
        counts[sel] = P[r, sel]
        P = P @ A
    parent = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        if dist[v] == 0:
            parent[v] = v
        elif dist[v] > 0:
            cands = [w for w in range(n) if A[v, w] and dist[w] == dist[v] - 1]
            parent[v] = max(cands)
    return dist, parent, counts


def check_all(g, r, exp_dist, exp_parent, exp_counts=None):
    d = oracle.bfs_queue(g.row_ptr, g.col, r)
    np.testing.assert_array_equal(d, exp_dist)
    np.testing.assert_array_equal(oracle.dp(g.row_ptr, g.col, d, r), exp_parent)
    ecc = int(np.max(exp_dist))
    for s in SEMIRINGS:
        dist, parent, fval, it, levels = oracle.bfs_semiring(g.row_ptr, g.col, r, s)
        np.testing.assert_array_equal(dist, exp_dist, err_msg=s)
        np.testing.assert_array_equal(parent, exp_parent, err_msg=s)
        assert it == ecc + 1, s  # the last SpMV pass reaches nothing new
        np.testing.assert_array_equal(levels[: ecc + 1],
                                      np.bincount(exp_dist[exp_dist >= 0], minlength=ecc + 1))
        if s == "real" and exp_counts is not None:
            reached = exp_dist >= 0
            np.testing.assert_array_equal(fval[reached], exp_counts[reached].astype(np.float64))


def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [p for b, p in enumerate(pairs) if mask >> b & 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_brute_force_all_small_graphs(n):
    for edges in all_graphs(n):
        g = gg.from_edges(n, edges)
        A = adjacency(g)
        for r in range(n):
            dist, parent, counts = brute_force(A, r)
            check_all(g, r, dist, parent, counts)


@pytest.mark.parametrize("n,trials", [(6, 300), (7, 150)])
def test_brute_force_random_graphs(n, trials):
    rng = np.random.default_rng(1234 + n)
    pairs = list(itertools.combinations(range(n), 2))
    for _ in range(trials):
        keep = rng.random(len(pairs)) < rng.uniform(0.15, 0.8)
        g = gg.from_edges(n, [p for p, k in zip(pairs, keep) if k])
        A = adjacency(g)
        r = int(rng.integers(n))
        dist, parent, counts = brute_force(A, r)
        check_all(g, r, dist, parent, counts)


def test_path_closed_form():
    n = 37
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    for r in [0, 5, 36]:
        v = np.arange(n)
        dist = np.abs(v - r)
        parent = np.where(v > r, v - 1, np.where(v < r, v + 1, r))
        check_all(g, r, dist, parent, np.ones(n, dtype=np.int64))


@pytest.mark.parametrize("n", [9, 10])
def test_cycle_closed_form(n):
    g = gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    for r in [0, 3]:
        v = np.arange(n)
        off = (v - r) % n
        dist = np.minimum(off, n - off)
        parent = np.empty(n, dtype=np.int64)
        counts = np.ones(n, dtype=np.int64)
        for u in range(n):
            if u == r:
                parent[u] = r
                continue
            nb = [(u - 1) % n, (u + 1) % n]
            parent[u] = max(w for w in nb if dist[w] == dist[u] - 1)
            if n % 2 == 0 and off[u] == n // 2:
                counts[u] = 2
        check_all(g, r, dist, parent, counts)


def test_star_and_complete():
    n = 12
    star = gg.from_edges(n, [(0, i) for i in range(1, n)])
    dist = np.ones(n, dtype=np.int64); dist[0] = 0
    check_all(star, 0, dist, np.zeros(n, dtype=np.int64), np.ones(n, dtype=np.int64))
    dist = np.full(n, 2); dist[0] = 1; dist[4] = 0
    parent = np.zeros(n, dtype=np.int64); parent[0] = 4; parent[4] = 4
    check_all(star, 4, dist, parent, np.ones(n, dtype=np.int64))
    K = gg.from_edges(n, itertools.combinations(range(n), 2))
    dist = np.ones(n, dtype=np.int64); dist[7] = 0
    check_all(K, 7, dist, np.full(n, 7), np.ones(n, dtype=np.int64))


def test_complete_bipartite():
    a, b = 5, 7
    g = gg.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    r = 2
    dist = np.array([2] * a + [1] * b); dist[r] = 0
    parent = np.array([a + b - 1] * a + [r] * b); parent[r] = r
    counts = np.array([b] * a + [1] * b); counts[r] = 1
    check_all(g, r, dist, parent, counts)


def test_full_lattice_closed_form():
    L = 9
    g = gg.lattice(L, 0.0, seed=3)
    assert g.nnz == 4 * L * (L - 1)
    for ri, rj in [(0, 0), (4, 6), (8, 3)]:
        r = ri * L + rj
        i, j = np.divmod(np.arange(L * L), L)
        dist = np.abs(i - ri) + np.abs(j - rj)
        ids = i * L + j
        parent = np.where(i < ri, ids + L, np.where(j < rj, ids + 1,
                          np.where(j > rj, ids - 1, np.where(i > ri, ids - L, r))))
        counts = np.array([comb(int(abs(a - ri) + abs(c - rj)), int(abs(a - ri)))
                           for a, c in zip(i, j)], dtype=np.int64)
        check_all(g, r, dist, parent, counts)


def test_disconnected_and_isolated_root():
    g = gg.from_edges(8, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 4)])
    dist = np.array([0, 1, 2, -1, -1, -1, -1, -1])
    parent = np.array([0, 0, 1, -1, -1, -1, -1, -1])
    check_all(g, 0, dist, parent, np.array([1, 1, 1, 0, 0, 0, 0, 0]))
    dist = np.full(8, -1); dist[3] = 0
    parent = np.full(8, -1); parent[3] = 3
    check_all(g, 3, dist, parent, None)
    dist = np.full(8, -1); dist[7] = 0
    parent = np.full(8, -1); parent[7] = 7
    check_all(g, 7, dist, parent, None)


def library_check(g, r):
    """scipy distances + components, path counts by level DP, max-id parents."""
    A = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    sd = csgraph.shortest_path(A, method="D", unweighted=True, indices=r)
    exp = np.where(np.isinf(sd), -1, sd).astype(np.int64)
    _, labels = csgraph.connected_components(A, directed=False)
    assert np.array_equal(exp >= 0, labels == labels[r])
    return exp


def check_invariants(g, r, dist, parent):
    n = g.n
    src = np.repeat(np.arange(n), g.degrees())
    dst = g.col
    assert dist[r] == 0 and parent[r] == r
    both = (dist[src] >= 0) & (dist[dst] >= 0)
    assert np.all(np.abs(dist[src][both] - dist[dst][both]) <= 1)
    assert np.all((dist[src] >= 0) == (dist[dst] >= 0))  # no edge leaves the reached set
    reached = np.flatnonzero((dist >= 0) & (np.arange(n) != r))
    # parent edge exists and is one level closer; it is the max-id such neighbour
    cand = np.where(dist[dst] == dist[src] - 1, dst, -1)
    best = np.full(n, -1, dtype=np.int64)
    np.maximum.at(best, src, cand)
    assert np.array_equal(parent[reached], best[reached])
    assert np.all(dist[parent[reached]] == dist[reached] - 1)
    assert np.all(parent[dist < 0] == -1)


@pytest.mark.parametrize("maker", [
    lambda: gg.kronecker(10, seed=7),
    lambda: gg.kronecker(11, seed=2),
    lambda: gg.lattice(40, 0.05, seed=5),
    lambda: gg.erdos_renyi(3000, 3.0, seed=4),
])
def test_library_and_invariants(maker):
    g = maker()
    for r in gg.roots(g, 3, seed=11):
        exp = library_check(g, int(r))
        d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
        np.testing.assert_array_equal(d, exp)
        p = oracle.dp(g.row_ptr, g.col, d, int(r))
        check_invariants(g, int(r), d, p)
        # shortest-path counts by a level-ordered DP over the library distances
        order = np.argsort(np.where(exp < 0, np.iinfo(np.int64).max, exp), kind="stable")
        cnt = np.zeros(g.n)
        cnt[int(r)] = 1.0
        for v in order:
            if exp[v] <= 0:
                continue
            nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
            cnt[v] = cnt[nb[exp[nb] == exp[v] - 1]].sum()
        for s in SEMIRINGS:
            dist, parent, fval, it, _ = oracle.bfs_semiring(g.row_ptr, g.col, int(r), s)
            np.testing.assert_array_equal(dist, exp, err_msg=s)
            np.testing.assert_array_equal(parent, p, err_msg=s)
            if s == "real":
                m = exp >= 0
                np.testing.assert_allclose(fval[m], cnt[m], rtol=1e-12)


def test_multi_equals_single():
    g = gg.kronecker(9, seed=3)
    rs = gg.roots(g, 5, seed=4)
    D = oracle.bfs_multi(g.row_ptr, g.col, rs)
    for i, r in enumerate(rs):
        np.testing.assert_array_equal(D[i], oracle.bfs_queue(g.row_ptr, g.col, int(r)))


def test_reached_edges_counts_component_edges():
    g = gg.from_edges(7, [(0, 1), (1, 2), (2, 0), (4, 5)])
    d = oracle.bfs_queue(g.row_ptr, g.col, 0)
    assert oracle.reached_edges(g.row_ptr, d) == 3
    d = oracle.bfs_queue(g.row_ptr, g.col, 5)
    assert oracle.reached_edges(g.row_ptr, d) == 1


def test_bad_root_rejected():
    g = gg.from_edges(3, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.bfs_queue(g.row_ptr, g.col, 3)
    with pytest.raises(ValueError):
        oracle.bfs_semiring(g.row_ptr, g.col, -1, "tropical")
