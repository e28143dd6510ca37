"""GPU: the storage-format comparison path (plain value-vector BFS-SpMV in the
SlimSell and the Sell-C-sigma formats) against the oracle's queue BFS, bit-exact."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu
SEMIRINGS = ["tropical", "real", "boolean", "selmax"]


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()


@pytest.mark.parametrize("fmt", ["slimsell", "sell"])
def test_formats_match_oracle(fmt):
    graphs = [gg.kronecker(12, seed=4), gg.lattice(40, 0.1, seed=5), gg.erdos_renyi(3000, 4.0, seed=6),
              gg.from_edges(5, [(0, 1), (1, 2), (3, 4)], name="two-components")]
    for g in graphs:
        for C, sigma, w in [(32, g.n, 0), (8, 16, 4), (64, 128, 64), (16, 1, 16)]:
            G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma, split_w=w)
            for r in list(gg.roots(g, 2, seed=7)) + [g.n - 1]:
                want = oracle.bfs_queue(g.row_ptr, g.col, int(r))
                for sr in SEMIRINGS:
                    dist = G.bfs_spmv(int(r), sr, fmt)
                    torch.cuda.synchronize()
                    np.testing.assert_array_equal(dist.cpu().numpy(), want,
                                                  err_msg=f"{g.name} C={C} sigma={sigma} w={w} {sr} {fmt}")
            G.close()


def test_formats_time_and_agree_on_kron18():
    """Both formats give the same distances on a larger graph with split chunks;
    kernel times are reported and positive."""
    g = gg.kronecker(18, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    r = int(gg.roots(g, 1, seed=3)[0])
    want = oracle.bfs_queue(g.row_ptr, g.col, r)
    for sr in (ss.TROPICAL, ss.REAL, ss.BOOLEAN, ss.SELMAX):
        for f in (ss.FORMAT_SLIMSELL, ss.FORMAT_SELL):
            dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
            ms = ss.slimsell_bfs_spmv(G.h, r, sr, f, dist, timed=True)
            torch.cuda.synchronize()
            assert ms > 0
            np.testing.assert_array_equal(dist.cpu().numpy(), want)
    G.close()


def test_format_invalid_arguments():
    g = gg.kronecker(8, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for args in [(g.n, 0, 0), (-1, 0, 0), (0, 4, 0), (0, 0, 2)]:
        with pytest.raises(ss.SlimSellError) as e:
            ss.slimsell_bfs_spmv(G.h, *args, dist)
        assert e.value.status == 1
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs_spmv(G.h, 0, 0, 0, None)
    G.close()
