"""GPU parity at the benchmark's other full sizes, on sampled roots: Kronecker
scale 24 (the roofline configuration; single-source SlimWork and the adaptive
schedule, and 64 sources at once with two of them checked), and the 4096 x 4096
lattice with 5 % of its edges deleted (thousands of levels in the cluster push)."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()


def expected(g, r):
    d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
    return d, oracle.dp(g.row_ptr, g.col, d, int(r))


def test_kron24_sampled():
    g = gg.kronecker(24, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    r = int(gg.roots(g, 1, seed=2)[0])
    d, p = expected(g, r)
    for sr, pol in [("tropical", "slimwork"), ("real", "heuristic"), ("selmax", "push")]:
        dist, parent = G.bfs(r, sr, pol)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dist.cpu().numpy(), d, err_msg=f"{sr} {pol}")
        np.testing.assert_array_equal(parent.cpu().numpy(), p, err_msg=f"{sr} {pol}")
    roots = gg.roots(g, 64, seed=84)
    dist = G.bfs_multi(roots, "slimwork")
    torch.cuda.synchronize()
    for s in (5, 50):
        np.testing.assert_array_equal(dist[:, s].cpu().numpy(), oracle.bfs_queue(g.row_ptr, g.col, int(roots[s])))
    G.close()


def test_lattice4096_sampled():
    g = gg.lattice(4096, 0.05, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    r = int(gg.roots(g, 1, seed=2)[0])
    d, p = expected(g, r)
    for sr in ("selmax", "tropical"):
        dist, parent = G.bfs(r, sr, "heuristic")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dist.cpu().numpy(), d, err_msg=sr)
        np.testing.assert_array_equal(parent.cpu().numpy(), p, err_msg=sr)
        st, its = G.run_stats(cap=g.n + 2)
        assert st.iterations == int(d.max()) + 1  # eccentricity + the pass that adds nothing
    G.close()


def test_batch_of_200_graphs_as_benchmarked():
    """The many-graph configuration exactly as the benchmark times it: 200
    Kronecker graphs of scales 10..18, autotuned layouts, every BFS in one
    CUDA-graph launch (200 device-side loops side by side), replayed once;
    every graph's distances and parents equal the oracle's."""
    import bench
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    graphs, scales, handles, roots, tuned, _ = bench.batch_workload(ss, torch, 200, stream, dev)
    assert sorted(set(int(s) for s in scales)) == list(range(10, 19))
    for policy in ("slimwork", "heuristic"):
        b = ss.slimsell_batch_create(handles, ss.SEMIRINGS["tropical"], ss.POLICIES[policy])
        dists = [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
        pars = [torch.empty(g.n, dtype=torch.int32, device=dev) for g in graphs]
        r_d = torch.tensor(roots, dtype=torch.int32, device=dev)
        for _ in range(2):  # the second launch replays the executable graph
            for t in dists + pars:
                t.fill_(-7)
            ss.slimsell_batch_run(b, r_d, dists, pars, stream)
            stats = ss.slimsell_batch_get_stats(b, len(graphs))
            for i, (g, r) in enumerate(zip(graphs, roots)):
                d, p = expected(g, r)
                np.testing.assert_array_equal(dists[i].cpu().numpy(), d, err_msg=f"{policy} graph {i}")
                np.testing.assert_array_equal(pars[i].cpu().numpy(), p, err_msg=f"{policy} graph {i}")
                assert stats[i].iterations == int(d.max()) + 1
                assert stats[i].reached == int((d >= 0).sum())
        ss.slimsell_batch_destroy(b)
    for h in handles:
        ss.slimsell_destroy(h)


@pytest.mark.parametrize("sigma", [1024, 1])
def test_kron22_sorting_scopes_sampled(sigma):
    """Kronecker 22 with the sigma ablations the benchmark times (sigma = 1024,
    and sigma = 1: no sorting, the most padding): one sampled root, all four
    semirings on the paper's method, plus an adaptive schedule."""
    g = gg.kronecker(22, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=sigma, split_w=256)
    assert G.info().sigma == sigma
    r = int(gg.roots(g, 1, seed=2)[0])
    d, p = expected(g, r)
    for sr, pol in [("tropical", "slimwork"), ("real", "slimwork"), ("boolean", "slimwork"),
                    ("selmax", "slimwork"), ("tropical", "heuristic")]:
        dist, parent = G.bfs(r, sr, pol)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dist.cpu().numpy(), d, err_msg=f"{sr} {pol}")
        np.testing.assert_array_equal(parent.cpu().numpy(), p, err_msg=f"{sr} {pol}")
    G.close()
