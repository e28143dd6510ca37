"""GPU: betweenness centrality on the SlimSell layout vs the oracle's Brandes
(fp64 both; the GPU sums in another order, split chunks with atomics, so the
tolerance is relative 1e-9 of the largest value)."""
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


def check(G, g, sources):
    got = G.bc(sources)
    torch.cuda.synchronize()
    want = oracle.bc(g.row_ptr, g.col, sources)
    scale = max(1.0, float(np.abs(want).max()))
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=1e-9, atol=1e-9 * scale)


@pytest.mark.parametrize("C,sigma,w", [(32, None, 0), (8, 16, 4), (64, 128, 64), (16, 1, 16)])
def test_bc_matches_oracle(C, sigma, w):
    for g, k in [(gg.kronecker(12, seed=4), 16), (gg.lattice(30, 0.1, seed=5), 4),
                 (gg.erdos_renyi(3000, 4.0, seed=6), 8)]:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma or g.n, split_w=w)
        check(G, g, gg.roots(g, k, seed=7))
        G.close()


def test_bc_small_and_degenerate():
    # a path (closed form 2 i (n-1-i) with every vertex a source), two components,
    # an isolated source, a repeated source, and a star whose hub row is split
    n = 9
    g = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)], name="path")
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=1, split_w=2)
    got = G.bc(np.arange(n)).cpu().numpy()
    np.testing.assert_allclose(got, [2.0 * i * (n - 1 - i) for i in range(n)], atol=1e-9)
    G.close()
    g = gg.from_edges(7, [(0, 1), (1, 2), (3, 4), (4, 5)], name="two-components+isolated")
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=g.n, split_w=0)
    check(G, g, np.array([0, 6, 4, 4, 2], dtype=np.int32))
    G.close()
    g = gg.from_edges(301, [(0, i) for i in range(1, 301)] + [(i, i + 1) for i in range(1, 300, 2)],
                      name="star+matching")
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=8)
    check(G, g, np.arange(0, 301, 7, dtype=np.int32))
    G.close()


def test_bc_kron18_sampled_sources():
    g = gg.kronecker(18, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    check(G, g, gg.roots(g, 3, seed=9))
    G.close()


def test_bc_invalid_arguments():
    g = gg.kronecker(8, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    src = torch.tensor([0, g.n], dtype=torch.int32, device="cuda")
    with pytest.raises(ss.SlimSellError) as e:
        ss.slimsell_bc(G.h, src, out)
    assert e.value.status == 1
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bc(G.h, src[:0], out)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bc(G.h, src[:1], None)
    G.close()
