"""GPU: batched BFS over many graphs in one CUDA-graph launch, and the autotuner."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss
from paper_2010_09913_gb300 import autotune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()


def make_graphs():
    rng = np.random.default_rng(5)
    graphs = [gg.kronecker(int(s), seed=100 + i) for i, s in enumerate(rng.integers(6, 13, 8))]
    graphs += [gg.lattice(30, 0.05, seed=3), gg.erdos_renyi(3000, 5.0, seed=4),
               gg.from_edges(40, [(i, i + 1) for i in range(39)]), gg.from_edges(3, [(0, 1)])]
    params = [(32, 0, 64), (8, 1, 0), (16, 256, 16), (64, 0, 8)] * 3  # sigma 0 = n
    return graphs, params


@pytest.mark.parametrize("policy", ["slimwork", "heuristic"])
@pytest.mark.parametrize("sr", ["tropical", "selmax", "real"])
def test_batch_matches_oracle_and_replays(policy, sr):
    graphs, params = make_graphs()
    Gs = [ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=s if s != 0 else g.n, split_w=w)
          for g, (C, s, w) in zip(graphs, params)]
    b = ss.slimsell_batch_create([G.h for G in Gs], ss.SEMIRINGS[sr], ss.POLICIES[policy])
    for rep in range(2):  # the same executable graph, new roots
        roots = [int(gg.roots(g, 2, seed=rep)[rep]) if g.n > 3 else 1 for g in graphs]
        dists = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
        pars = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
        ss.slimsell_batch_run(b, torch.tensor(roots, dtype=torch.int32, device="cuda"), dists, pars)
        stats = ss.slimsell_batch_get_stats(b, len(graphs))
        for g, r, dd, pp, st in zip(graphs, roots, dists, pars, stats):
            d = oracle.bfs_queue(g.row_ptr, g.col, r)
            np.testing.assert_array_equal(dd.cpu().numpy(), d, err_msg=g.name)
            np.testing.assert_array_equal(pp.cpu().numpy(), oracle.dp(g.row_ptr, g.col, d, r))
            assert st.reached == int((d >= 0).sum())
            assert st.iterations == int(d.max()) + 1
    ss.slimsell_batch_destroy(b)
    for G in Gs:
        G.close()


def test_batch_invalid():
    g = gg.kronecker(8, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_batch_create([G.h, G.h], 0, 1)
    b = ss.slimsell_batch_create([G.h], 0, 1)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_batch_run(b, torch.tensor([g.n], dtype=torch.int32, device="cuda"))
    ss.slimsell_batch_destroy(b)
    G.close()


def test_autotune_returns_grid_point_and_caches():
    """slimsell_autotune through the C ABI: every grid point timed once, the best
    point's layout gives the oracle's BFS, and graphs with a matching signature
    (same family and size, same grid) are answered from the cache."""
    g = gg.kronecker(11, seed=4)
    roots = gg.roots(g, 2, seed=1)
    grid = {"C": (16, 32), "sigma": (1, 256, "n"), "split_w": (256, 4096)}
    best, table, res = autotune.tune(g.row_ptr, g.col, roots, grid=grid, repeats=1, use_cache=False,
                                     with_result=True)
    assert res.cached == 0 and res.points == 12 and len(table) == 12
    assert [p for p, _ in table][:3] == [{"C": 16, "sigma": 1, "split_w": 256},
                                         {"C": 16, "sigma": 1, "split_w": 4096},
                                         {"C": 16, "sigma": 256, "split_w": 256}]
    assert all(ms > 0 for _, ms in table)
    assert best == min(table, key=lambda t: t[1])[0]
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=best["C"],
                                   sigma=g.n if best["sigma"] == "n" else best["sigma"],
                                   split_w=best["split_w"])
    r = int(roots[0])
    d = oracle.bfs_queue(g.row_ptr, g.col, r)
    dist, parent = G.bfs(r, "tropical", "slimwork")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dist.cpu().numpy(), d)
    np.testing.assert_array_equal(parent.cpu().numpy(), oracle.dp(g.row_ptr, g.col, d, r))
    G.close()
    again, table2, res2 = autotune.tune(g.row_ptr, g.col, roots, grid=grid, with_result=True)
    assert res2.cached == 1 and res2.points == 0 and again == best and table2 == table
    other, _, res3 = autotune.tune(gg.kronecker(11, seed=5).row_ptr, gg.kronecker(11, seed=5).col,
                                   roots, grid=grid, with_result=True)
    assert res3.cached == 1 and other == best  # same family and size
    _, _, res4 = autotune.tune(g.row_ptr, g.col, roots, grid=grid, semiring="real", repeats=1,
                               with_result=True)
    assert res4.cached == 0 and res4.points == 12  # another semiring searches again


def test_autotune_rejects_bad_grids():
    g = gg.kronecker(8, seed=1)
    with pytest.raises(ss.SlimSellError):
        autotune.tune(g.row_ptr, g.col, [0], grid={"C": (12,), "sigma": (1,), "split_w": (0,)})
    with pytest.raises(ss.SlimSellError):
        autotune.tune(g.row_ptr, g.col, [g.n], grid={"C": (8,), "sigma": (1,), "split_w": (0,)})
