"""GPU: bit-packed multi-source BFS vs k independent oracle queue BFS runs, bit-exact."""
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


def check(G, g, roots, policy):
    dist = G.bfs_multi(roots, policy)
    torch.cuda.synchronize()
    want = oracle.bfs_multi(g.row_ptr, g.col, roots)  # (k, n)
    np.testing.assert_array_equal(dist.cpu().numpy(), want.T)
    st, _ = G.run_stats()
    assert st.reached == int((want >= 0).sum())
    assert st.reached_degree == sum(2 * oracle.reached_edges(g.row_ptr, want[s]) for s in range(len(roots)))
    return st


@pytest.mark.parametrize("k", [64, 100, 256, 1024])
@pytest.mark.parametrize("policy", ["full", "slimwork"])
def test_kron_multi(k, policy):
    g = gg.kronecker(12, seed=9)
    rng = np.random.default_rng(k)
    roots = gg.roots(g, min(k, 600), seed=3)
    roots = np.concatenate([roots, rng.choice(roots, k - len(roots))]) if k > len(roots) else roots
    for C, w in [(32, 0), (32, 16), (64, 64)]:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=g.n, split_w=w)
        check(G, g, roots.astype(np.int32), policy)
        G.close()


def test_lattice_and_ragged_multi():
    g = gg.lattice(45, 0.08, seed=2)  # several components, long diameter
    roots = np.array(list(gg.roots(g, 40, seed=4)) + [0, g.n - 1, 7], dtype=np.int32)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=16, sigma=g.n, split_w=2)
    st = check(G, g, roots, "slimwork")
    assert st.iterations > 40
    G.close()


def test_multi_invalid_arguments():
    g = gg.kronecker(8, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32)
    r = torch.zeros(5, dtype=torch.int32, device="cuda")
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs_multi(G.h, r[:0], ss.V_SLIMWORK, None)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs_multi(G.h, torch.zeros(1025, dtype=torch.int32, device="cuda"), 1, None)
    bad = torch.tensor([0, g.n], dtype=torch.int32, device="cuda")
    with pytest.raises(ss.SlimSellError) as e:
        ss.slimsell_bfs_multi(G.h, bad, ss.V_SLIMWORK, None)
    assert e.value.status == 1
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs_multi(G.h, r, ss.V_PUSH, None)
    G.close()


def test_small_chunks_and_few_sources():
    """C = 8 with 5 sources: the words per vertex are padded up to a full warp."""
    g = gg.kronecker(10, seed=6)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=g.n, split_w=4)
    check(G, g, gg.roots(g, 5, seed=1), "slimwork")
    G.close()


def test_kron22_multi_sampled():
    """Full-size Kronecker scale 22, 64 sources; 4 sampled sources checked exactly."""
    g = gg.kronecker(22, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    roots = gg.roots(g, 64, seed=2)
    dist = G.bfs_multi(roots, "slimwork")
    torch.cuda.synchronize()
    for s in (0, 17, 40, 63):
        want = oracle.bfs_queue(g.row_ptr, g.col, int(roots[s]))
        np.testing.assert_array_equal(dist[:, s].cpu().numpy(), want)
    G.close()


@pytest.mark.parametrize("offset", [0, 1])
def test_distance_writes_aligned_and_not(offset):
    """k = 100 (a multiple of 4): an aligned output takes 16-byte group writes, one
    shifted by a single int32 takes per-entry writes; both equal the oracle."""
    g = gg.kronecker(11, seed=4)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=64)
    roots = gg.roots(g, 100, seed=6)
    buf = torch.full((g.n * 100 + 4,), 7, dtype=torch.int32, device="cuda")
    dist = buf[offset:offset + g.n * 100].view(g.n, 100)
    ss.slimsell_bfs_multi(G.h, torch.from_numpy(roots).cuda(), ss.V_SLIMWORK, dist)
    torch.cuda.synchronize()
    want = oracle.bfs_multi(g.row_ptr, g.col, roots)
    np.testing.assert_array_equal(dist.cpu().numpy(), want.T)
    rest = torch.cat([buf[:offset], buf[offset + g.n * 100:]]).cpu().numpy()
    assert (rest == 7).all()  # nothing written outside the output
    G.close()


def check_parents(G, g, roots, policy):
    dist, parent = G.bfs_multi_parents(roots, policy)
    torch.cuda.synchronize()
    want = oracle.bfs_multi(g.row_ptr, g.col, roots)  # (k, n)
    np.testing.assert_array_equal(dist.cpu().numpy(), want.T)
    got = parent.cpu().numpy()
    for s, r in enumerate(roots):
        np.testing.assert_array_equal(got[:, s], oracle.dp(g.row_ptr, g.col, want[s], int(r)),
                                      err_msg=f"source {s} root {r}")


@pytest.mark.parametrize("k", [64, 100, 1024])
def test_multi_parents_kron(k):
    """Parents per source equal the oracle's largest-id DP parents, with and without
    SlimChunk splits (split items combine their candidates with atomicMax)."""
    g = gg.kronecker(12, seed=9)
    rng = np.random.default_rng(k)
    roots = gg.roots(g, min(k, 600), seed=3)
    roots = np.concatenate([roots, rng.choice(roots, k - len(roots))]) if k > len(roots) else roots
    for C, w, policy in [(32, 0, "slimwork"), (32, 16, "slimwork"), (64, 64, "full")]:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=g.n, split_w=w)
        check_parents(G, g, roots.astype(np.int32), policy)
        G.close()


def test_multi_parents_lattice_and_ragged():
    g = gg.lattice(45, 0.08, seed=2)  # several components: unreached parents stay -1
    roots = np.array(list(gg.roots(g, 40, seed=4)) + [0, g.n - 1, 7, 7], dtype=np.int32)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=16, sigma=g.n, split_w=2)
    check_parents(G, g, roots, "slimwork")
    G.close()


def test_multi_parents_without_distances_and_plain_call_unchanged():
    """dist = NULL with parents; then the parent-less call on the same handle."""
    g = gg.erdos_renyi(3000, 5.0, seed=7)
    roots = gg.roots(g, 70, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=64, split_w=4)
    _, parent = G.bfs_multi_parents(roots, "slimwork", want_dist=False)
    torch.cuda.synchronize()
    want = oracle.bfs_multi(g.row_ptr, g.col, roots)
    got = parent.cpu().numpy()
    for s, r in enumerate(roots):
        np.testing.assert_array_equal(got[:, s], oracle.dp(g.row_ptr, g.col, want[s], int(r)))
    check(G, g, roots, "slimwork")
    G.close()


def test_kron22_multi_parents_sampled():
    """Full-size Kronecker scale 22, 64 sources with parents; 3 sampled sources exact."""
    g = gg.kronecker(22, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    roots = gg.roots(g, 64, seed=2)
    dist, parent = G.bfs_multi_parents(roots, "slimwork")
    torch.cuda.synchronize()
    for s in (0, 31, 63):
        d = oracle.bfs_queue(g.row_ptr, g.col, int(roots[s]))
        np.testing.assert_array_equal(dist[:, s].cpu().numpy(), d)
        np.testing.assert_array_equal(parent[:, s].cpu().numpy(), oracle.dp(g.row_ptr, g.col, d, int(roots[s])))
    G.close()


def test_multi_parents_far_in_a_long_row():
    """A row of 1,200 neighbours whose only frontier neighbour at its level is
    stored last (the smallest id): the walk has to reach the end of the row."""
    hub = 1300
    edges = [(u, hub) for u in range(1200)] + [(1200 + t, t) for t in range(100)]
    g = gg.from_edges(hub + 1, edges, name="far-parent")
    roots = np.arange(1200, 1270, dtype=np.int32)  # each reaches the hub through one leaf
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=0)
    check_parents(G, g, roots, "slimwork")
    G.close()
