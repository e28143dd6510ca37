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
