"""GPU parity of the real semiring's values (Section III-A, (R, +, *, 0, 1)).

The pull, the push variants and SlimChunk's partial rows all add up the values
of a row's frontier neighbours; slimsell_get_values exports them and they are
compared with the oracle's fp64 semiring BFS, whose values are pinned to
brute-force shortest-path counts in the oracle tests.

Tolerance: the device sums fp32 values in no fixed order.  A sum of positive
integers is exact in fp32 while every partial sum stays below 2^24, so vertices
whose count is below 2^24 must match exactly.  Above that each fp32 addition
rounds with relative error at most u = 2^-24; in any order of summation a term
of a sum of m terms passes through at most m - 1 additions, and a sum of
positive terms keeps the largest relative error of its inputs.  So the value of
a vertex at level L is within (1 + u)^(L (Dmax - 1)) - 1 of the exact count,
relatively (Dmax the largest degree bounds the terms of one sum).
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
POLICIES = ["full", "slimwork", "pull_filtered", "push", "heuristic"]


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()
    assert torch.cuda.is_available()


_oracle_cache = {}


def oracle_values(g, r):
    key = (g.name, g.n, int(r))
    if key not in _oracle_cache:
        d_o, _, fval, _, _ = oracle.bfs_semiring(g.row_ptr, g.col, int(r), "real")
        _oracle_cache.clear()
        _oracle_cache[key] = (d_o, fval)
    return _oracle_cache[key]


def check_values(g, G, r, pol, label):
    dist, _ = G.bfs(int(r), "real", pol)
    vals = G.values()
    torch.cuda.synchronize()
    d_o, fval = oracle_values(g, r)
    np.testing.assert_array_equal(dist.cpu().numpy(), d_o, err_msg=label)
    v = vals.cpu().numpy().astype(np.float64)
    reached = d_o >= 0
    assert np.all(v[~reached] == 0.0), label
    assert v[int(r)] == 1.0, label
    exact = reached & (fval < 2.0 ** 24)
    np.testing.assert_array_equal(v[exact], fval[exact], err_msg=label)
    big = reached & ~exact
    if big.any():
        dmax = int(np.diff(g.row_ptr).max())
        bound = np.expm1(d_o[big].astype(np.float64) * max(dmax - 1, 1) * np.log1p(U))
        rel = np.abs(v[big] - fval[big]) / fval[big]
        assert np.all(rel <= bound), (label, float(rel.max()))
    return int(big.sum())


@pytest.mark.parametrize("pol", POLICIES)
def test_values_kron14(pol):
    g = gg.kronecker(14, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    for r in gg.roots(g, 3, seed=2):
        check_values(g, G, r, pol, f"kron14 {pol} r={r}")
    G.close()


@pytest.mark.parametrize("C,sigma_kind,split_w", [(8, "one", 0), (16, "window", 16), (32, "full", 4),
                                                  (64, "full", 0), (64, "window", 16)])
def test_values_layouts(C, sigma_kind, split_w):
    """Every chunk height, sorting scope and SlimChunk split (split rows add their
    partial sums with atomics before the last arriving item posts the row)."""
    g = gg.kronecker(11, seed=3)
    sigma = {"one": 1, "window": 256, "full": g.n}[sigma_kind]
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma, split_w=split_w)
    for r in gg.roots(g, 2, seed=5):
        for pol in ("full", "slimwork", "push"):
            check_values(g, G, r, pol, f"C={C} sigma={sigma} w={split_w} {pol}")
    G.close()


def test_values_lattice_er_and_edge_cases():
    """A lattice (path counts are binomial coefficients: most exceed 2^24, so the
    rounding bound is exercised), an ER graph and the degenerate graphs."""
    graphs = [gg.lattice(64, 0.05, seed=1), gg.erdos_renyi(1 << 14, 16.0, seed=1),
              gg.from_edges(1, []), gg.from_edges(70, [(i, i + 1) for i in range(69)]),
              gg.from_edges(40, [(0, i) for i in range(1, 40)]),
              gg.from_edges(33, [(i, j) for i in range(33) for j in range(i + 1, 33)]),
              gg.from_edges(9, [(0, 1), (1, 2), (5, 6), (6, 7), (7, 5)])]
    rounded = 0
    for g in graphs:
        for C, split_w in [(8, 2), (32, 256)]:
            G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=g.n, split_w=split_w)
            for r in sorted({0, g.n - 1, g.n // 2}):
                for pol in POLICIES:
                    rounded += check_values(g, G, r, pol, f"{g.name} C={C} {pol} r={r}")
            G.close()
    assert rounded > 0  # the lattice has counts above 2^24


def test_values_sell_format():
    """The pull over the Sell-C-sigma arrays multiplies each gathered value by the
    stored matrix value (1) and gives the same path counts."""
    g = gg.kronecker(12, seed=3)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=64)
    G.set_option(ss.OPT_FORMAT, ss.FORMAT_SELL)
    for r in gg.roots(g, 2, seed=6):
        for pol in ("full", "slimwork"):
            check_values(g, G, r, pol, f"sell {pol}")
    G.close()


def test_values_kron22_hub_levels():
    """Full-size Kronecker scale 22: the hub level stages the values of the
    highest-degree rows in shared memory (the path the smaller graphs barely use)."""
    g = gg.kronecker(22, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    for r in gg.roots(g, 2, seed=2):
        for pol in ("slimwork", "heuristic"):
            check_values(g, G, r, pol, f"kron22 {pol} r={r}")
    G.close()


def test_values_refused_after_other_runs():
    g = gg.kronecker(9, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    with pytest.raises(ss.SlimSellError):  # no run yet
        G.values()
    G.bfs(0, "real", "slimwork")
    G.values()
    G.bfs(0, "tropical", "slimwork")
    with pytest.raises(ss.SlimSellError):
        G.values()
    G.bfs(0, "real", "slimwork")
    G.bfs_multi([0, 1], "slimwork")
    with pytest.raises(ss.SlimSellError):
        G.values()
    torch.cuda.synchronize()
    G.close()
