"""GPU parity of the cluster push: small frontiers (at most 4096 vertices and
8192 edges per CTA of a 16- or 8-CTA thread-block cluster) run level after
level inside one launch, with the frontier kept as a vertex list, and hand back
to the grid-wide variants when a level outgrows the cluster.  Results must equal
the oracle's bit for bit, for every semiring, in the device-side and the
host-driven loop, across hand-overs in both directions.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu

SEMIRINGS = ["tropical", "real", "boolean", "selmax"]
LOCAL = ss.VARIANT_PUSH_LOCAL


@pytest.fixture(scope="module", autouse=True)
def _build():
    ss.build()
    assert torch.cuda.is_available()


def relabelled(n, edges, seed, name):
    """Graph from an edge list with vertex ids shuffled by a seeded permutation."""
    p = gg.permutation(n, seed)
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return gg.edges_to_csr(n, p[e[:, 0]], p[e[:, 1]], None, name=name), p


def path_graph(n, seed=1):
    return relabelled(n, [(i, i + 1) for i in range(n - 1)], seed, f"path{n}")


def grow_shrink(tail=300, fan=70000, seed=2):
    """path -- hub -- fan leaves -- hub -- path: a level of `fan` vertices between
    two long runs of one-vertex levels."""
    e, v = [], 0
    for i in range(tail):
        e.append((v, v + 1))
        v += 1
    hub1 = v
    leaves = list(range(hub1 + 1, hub1 + 1 + fan))
    hub2 = hub1 + 1 + fan
    for x in leaves:
        e += [(hub1, x), (x, hub2)]
    v = hub2
    for i in range(tail):
        e.append((v, v + 1))
        v += 1
    return relabelled(v + 1, e, seed, f"growshrink{tail}-{fan}")


def wide_star(tail=200, leaves=140000, seed=3):
    """A path ending in a hub whose degree alone exceeds the block's edge capacity."""
    e = [(i, i + 1) for i in range(tail)]
    hub = tail
    e += [(hub, hub + 1 + j) for j in range(leaves)]
    return relabelled(hub + 1 + leaves, e, seed, f"widestar{leaves}")


def hub_graph(tail=50, leaves=100000, seed=5):
    """A path into a hub with 100000 leaves, every leaf also tied to a second hub:
    the hubs' rows are longer than one cluster-push slice entry, so their edges
    are spread over the cluster in units."""
    e = [(i, i + 1) for i in range(tail)]
    hub1, hub2 = tail, tail + 1 + leaves
    for j in range(leaves):
        e += [(hub1, tail + 1 + j), (tail + 1 + j, hub2)]
    return relabelled(hub2 + 1, e, seed, f"hubs{leaves}")


def expected(g, r):
    d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
    return d, oracle.dp(g.row_ptr, g.col, d, int(r))


def check(G, g, r, sr, policy):
    dist, parent = G.bfs(int(r), sr, policy)
    torch.cuda.synchronize()
    d, p = expected(g, r)
    np.testing.assert_array_equal(dist.cpu().numpy(), d, err_msg=f"{g.name} {sr} {policy}")
    np.testing.assert_array_equal(parent.cpu().numpy(), p, err_msg=f"{g.name} {sr} {policy}")
    _, _, _, it, levels = oracle.bfs_semiring(g.row_ptr, g.col, int(r), sr)
    st, its = G.run_stats(cap=it + 2)
    assert st.iterations == it, (g.name, sr, policy)
    got = np.array([its[i].frontier for i in range(it + 1)])
    np.testing.assert_array_equal(got[: len(levels)], levels)
    assert not got[len(levels):].any()  # the final pass discovers nothing
    return [its[i].variant for i in range(1, it + 1)]


@pytest.mark.parametrize("loop", [1, 0])
@pytest.mark.parametrize("policy", ["push", "heuristic"])
def test_path_runs_in_one_block(policy, loop):
    g, p = path_graph(3000)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    G.set_option(ss.OPT_DEVICE_LOOP, loop)
    for r in [int(p[0]), int(p[1500]), int(p[2999])]:
        for sr in SEMIRINGS:
            seq = check(G, g, r, sr, policy)
            assert all(v == LOCAL for v in seq), seq
    G.close()


@pytest.mark.parametrize("loop", [1, 0])
@pytest.mark.parametrize("policy", ["push", "heuristic", "learned"])
def test_hand_over_both_ways(policy, loop):
    g, p = grow_shrink()
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=16, sigma=256, split_w=64)
    G.set_option(ss.OPT_DEVICE_LOOP, loop)
    if policy == "learned":
        ss.slimsell_selector_load(G.h, gg.mlp_weights(7, scale=3.0))
    for r in [int(p[0]), int(p[305])]:
        for sr in SEMIRINGS:
            seq = check(G, g, r, sr, policy)
            if policy != "learned":
                i = seq.index(next(v for v in seq if v != LOCAL))  # the wide level left the cluster
                assert LOCAL in seq[:i] and LOCAL in seq[i + 1:], seq
    G.close()


@pytest.mark.parametrize("loop", [1, 0])
def test_edge_capacity_hand_back(loop):
    g, p = wide_star()
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    G.set_option(ss.OPT_DEVICE_LOOP, loop)
    r = int(p[0])
    for sr in SEMIRINGS:
        for policy in ["push", "heuristic"]:
            seq = check(G, g, r, sr, policy)
            assert seq[0] == LOCAL and seq[-1] != LOCAL, seq  # the hub's 140001 edges
    G.close()


@pytest.mark.parametrize("loop", [1, 0])
def test_long_rows_split_into_units(loop):
    g, p = hub_graph()
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    G.set_option(ss.OPT_DEVICE_LOOP, loop)
    for r in [int(p[0]), int(p[50]), int(p[40000]), int(p[100051])]:  # path end, hubs, a leaf
        for sr in SEMIRINGS:
            seq = check(G, g, r, sr, "push")
            assert seq.count(LOCAL) >= 1, seq
    G.close()


@pytest.mark.parametrize("maker", [lambda: gg.lattice(96, 0.1, seed=4, permute=True),
                                   lambda: gg.erdos_renyi(20000, 1.6, seed=5),
                                   lambda: gg.kronecker(12, seed=6)])
def test_sparse_families_device_vs_host_loop(maker):
    g = maker()
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=4096, split_w=1024)
    for r in gg.roots(g, 3, seed=9):
        for loop in [1, 0]:
            G.set_option(ss.OPT_DEVICE_LOOP, loop)
            for sr in SEMIRINGS:
                check(G, g, int(r), sr, "heuristic")
    G.close()


def test_alternating_policies_keep_scratch_clean():
    """Pull, cluster push and grid push share the frontier bitmaps and push
    scratch; alternating runs on one handle must not leak state between runs."""
    g, p = grow_shrink(tail=120, fan=66000, seed=7)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    roots = [int(p[0]), int(p[130]), int(p[66200]), int(p[60])]
    for i, r in enumerate(roots * 2):
        for pol in ["slimwork", "push", "pull_filtered", "heuristic"][i % 4:] + ["full"]:
            check(G, g, r, SEMIRINGS[i % 4], pol)
    G.close()


def test_host_loop_times_every_level():
    g, p = path_graph(500, seed=11)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    G.set_option(ss.OPT_DEVICE_LOOP, 0)
    ss.slimsell_set_profiling(G.h, True)
    G.bfs(int(p[0]), "tropical", "push")
    torch.cuda.synchronize()
    st, its = G.run_stats(cap=g.n + 2)
    assert st.iterations == 500
    # all 500 levels run in one cluster launch: each level has its device-side time,
    # the launch's entry counted in the first, and together they make the launch time
    assert all(its[k].variant == LOCAL and its[k].kernel_ns > 0 for k in range(1, 501))
    total_ms = sum(its[k].kernel_ns for k in range(1, 501)) / 1e6
    assert abs(total_ms - st.iter_kernel_ms) <= 0.05 * st.iter_kernel_ms + 0.05
    ss.slimsell_set_profiling(G.h, False)
    G.close()

