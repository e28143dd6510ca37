"""Pins of the oracle's betweenness centrality (Brandes' dependency accumulation)
against closed forms, brute-force path enumeration and networkx."""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle


def csr(n, edges):
    g = gg.from_edges(n, edges)
    return g.row_ptr, g.col


def test_path_graph_closed_form():
    # on a path 0 - 1 - ... - (n-1), vertex i lies on every shortest path between
    # its i left and n-1-i right vertices: i(n-1-i) unordered pairs, counted twice
    n = 9
    rp, col = csr(n, [(i, i + 1) for i in range(n - 1)])
    want = np.array([2.0 * i * (n - 1 - i) for i in range(n)])
    np.testing.assert_allclose(oracle.bc(rp, col, np.arange(n)), want, rtol=0, atol=1e-12)


def test_star_and_complete_graph():
    n = 7  # star: the centre is on every path between two leaves
    rp, col = csr(n, [(0, i) for i in range(1, n)])
    bc = oracle.bc(rp, col, np.arange(n))
    assert bc[0] == pytest.approx((n - 1) * (n - 2))
    assert np.all(bc[1:] == 0)
    rp, col = csr(5, list(itertools.combinations(range(5), 2)))  # complete: no intermediates
    assert np.all(oracle.bc(rp, col, np.arange(5)) == 0)


def test_cycle_graph_even_splits_paths():
    # C_6: opposite vertices are joined by two shortest paths, each carrying 1/2
    n = 6
    rp, col = csr(n, [(i, (i + 1) % n) for i in range(n)])
    # per vertex: pairs at distance 2 through it (2 ordered pairs, weight 1)
    # plus opposite pairs whose two paths it lies on (4 ordered pairs, weight 1/2)
    np.testing.assert_allclose(oracle.bc(rp, col, np.arange(n)), np.full(n, 2 + 4 * 0.5), atol=1e-12)


def brute_force_bc(n, adj, sources):
    """Enumerate every shortest path by BFS layers and count vertex visits."""
    bc = np.zeros(n)
    for s in sources:
        dist = {s: 0}
        frontier = [s]
        while frontier:
            nxt = []
            for u in frontier:
                for w in adj[u]:
                    if w not in dist:
                        dist[w] = dist[u] + 1
                        nxt.append(w)
            frontier = nxt

        def paths(t):  # all shortest s-t paths as vertex lists
            if t == s:
                return [[s]]
            return [p + [t] for u in adj[t] if dist.get(u, -9) == dist[t] - 1 for p in paths(u)]

        for t in dist:
            if t == s:
                continue
            ps = paths(t)
            for p in ps:
                for v in p[1:-1]:
                    bc[v] += 1.0 / len(ps)
    return bc


def test_brute_force_small_random_graphs():
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = int(rng.integers(2, 9))
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.4]
        rp, col = csr(n, pairs)
        adj = [[] for _ in range(n)]
        for i, j in pairs:
            adj[i].append(j)
            adj[j].append(i)
        sources = rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False)
        np.testing.assert_allclose(oracle.bc(rp, col, sources), brute_force_bc(n, adj, sources),
                                   rtol=1e-12, atol=1e-12, err_msg=f"trial {trial}")


def test_matches_networkx():
    nx = pytest.importorskip("networkx")
    for g in [gg.kronecker(8, seed=3), gg.lattice(12, 0.1, seed=4), gg.erdos_renyi(300, 3.0, seed=5)]:
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        G.add_edges_from(zip(src.tolist(), g.col.tolist()))
        want = nx.betweenness_centrality(G, normalized=False)  # unordered pairs
        got = oracle.bc(g.row_ptr, g.col, np.arange(g.n)) / 2.0
        np.testing.assert_allclose(got, [want[v] for v in range(g.n)], rtol=1e-9, atol=1e-9)


def test_bad_source_raises():
    rp, col = csr(3, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.bc(rp, col, [3])
