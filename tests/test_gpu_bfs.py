"""GPU parity: SlimSell BFS through the C ABI vs the CPU oracle, bit-exact.

Distances and parents are integers and must match exactly (parents are the
canonical max-id parent for every semiring).  Iteration counts and the number
of vertices discovered per iteration must match the oracle's semiring BFS.
"""
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
    assert torch.cuda.is_available()


def expected(g, r):
    d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
    return d, oracle.dp(g.row_ptr, g.col, d, int(r))


def run(G, r, sr, pol):
    dist, parent = G.bfs(int(r), sr, pol)
    torch.cuda.synchronize()
    return dist.cpu().numpy(), parent.cpu().numpy()


def check_stats(G, g, r, sr):
    _, _, _, it, levels = oracle.bfs_semiring(g.row_ptr, g.col, int(r), sr)
    st, iters = G.run_stats(cap=it + 1)
    assert st.iterations == it
    got = np.array([iters[i].frontier for i in range(it + 1)])
    np.testing.assert_array_equal(got[: len(levels)], levels)
    d = oracle.bfs_queue(g.row_ptr, g.col, int(r))
    assert st.reached == int((d >= 0).sum())
    assert st.reached_degree == 2 * oracle.reached_edges(g.row_ptr, d)


@pytest.mark.parametrize("sr", SEMIRINGS)
@pytest.mark.parametrize("pol", ["full", "slimwork", "pull_filtered", "push", "heuristic"])
def test_kron14_parity(sr, pol):
    """Kronecker scale 14, C = 32, sigma = n (the small configuration), several roots."""
    g = gg.kronecker(14, seed=1)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=256)
    for r in gg.roots(g, 4, seed=2):
        d, p = expected(g, r)
        dist, parent = run(G, r, sr, pol)
        np.testing.assert_array_equal(dist, d)
        np.testing.assert_array_equal(parent, p)
        check_stats(G, g, r, sr)
    G.close()


@pytest.mark.parametrize("C", [8, 16, 32, 64])
@pytest.mark.parametrize("sigma_kind", ["one", "window", "full"])
@pytest.mark.parametrize("split_w", [0, 16])
def test_layout_independence(C, sigma_kind, split_w):
    g = gg.kronecker(11, seed=3)
    sigma = {"one": 1, "window": 256, "full": g.n}[sigma_kind]
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma, split_w=split_w)
    r = int(gg.roots(g, 1, seed=5)[0])
    d, p = expected(g, r)
    for sr in SEMIRINGS:
        dist, parent = run(G, r, sr, "slimwork")
        np.testing.assert_array_equal(dist, d, err_msg=sr)
        np.testing.assert_array_equal(parent, p, err_msg=sr)
    G.close()


@pytest.mark.parametrize("C", [8, 32, 64])
def test_layout_matches_oracle(C):
    for g in [gg.kronecker(10, seed=4), gg.lattice(23, 0.1, seed=2)]:  # n = 529 is ragged
        for sigma in (1, 64, g.n):
            for split_w in (0, 7):
                G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma, split_w=split_w)
                L = oracle.slimsell_layout(g.row_ptr, g.col, C, sigma, split_w)
                got = {k: v.cpu().numpy() for k, v in G.export_layout().items()}
                perm = L["perm"]
                np.testing.assert_array_equal(got["perm"][: g.n], perm)
                assert np.all(got["perm"][g.n:] == -1)
                np.testing.assert_array_equal(got["cl"], L["cl"])
                np.testing.assert_array_equal(got["cs"], L["cs"])
                np.testing.assert_array_equal(got["col"], L["col"])
                # the work list omits chunks of isolated rows and is reordered for load balance
                want_items = L["items"][L["items"][:, 2] > L["items"][:, 1]]
                got_items = got["items"][:, :3]
                key = lambda a: a[np.lexsort((a[:, 1], a[:, 0]))]
                np.testing.assert_array_equal(key(got_items), key(want_items))
                inf = G.info()
                assert inf.slots == L["cs"][-1] and inf.padding == L["padding"]
                assert inf.max_degree == int(g.degrees().max())
                G.close()


@pytest.mark.parametrize("smem", [0, 16, 4096])
@pytest.mark.parametrize("dp_pass", [0, 1])
def test_options_do_not_change_results(smem, dp_pass):
    """Bitmap prefix in shared memory (0 = all global reads) and the separate DP pass."""
    g = gg.kronecker(13, seed=8)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=64)
    G.set_option(ss.OPT_SMEM_BYTES, smem)
    G.set_option(ss.OPT_DP_PASS, dp_pass)
    for r in gg.roots(g, 2, seed=9):
        d, p = expected(g, r)
        for sr in SEMIRINGS:
            for pol in ("full", "slimwork", "pull_filtered"):
                dist, parent = run(G, r, sr, pol)
                np.testing.assert_array_equal(dist, d, err_msg=f"{sr} {pol}")
                np.testing.assert_array_equal(parent, p, err_msg=f"{sr} {pol}")
                if dp_pass and sr != "selmax":
                    assert G.run_stats()[0].dp_slots > 0
    with pytest.raises(ss.SlimSellError):
        G.set_option(ss.OPT_SMEM_BYTES, 1 << 30)
    with pytest.raises(ss.SlimSellError):
        G.set_option(99, 1)
    G.close()


def test_device_loop_matches_host_loop():
    """The conditional-graph iteration loop and the host-driven loop (queued in
    batches, and one iteration at a time) agree exactly."""
    g = gg.kronecker(12, seed=4)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=32)
    for r in gg.roots(g, 3, seed=7):
        d, p = expected(g, r)
        for sr in SEMIRINGS:
            for pol in ("full", "slimwork", "pull_filtered", "push", "heuristic"):
                res = []
                for loop, queue in ((1, 1), (0, 1), (0, 0)):
                    G.set_option(ss.OPT_DEVICE_LOOP, loop)
                    G.set_option(ss.OPT_PROFILE_QUEUE, queue)
                    dist, parent = run(G, r, sr, pol)
                    np.testing.assert_array_equal(dist, d)
                    np.testing.assert_array_equal(parent, p)
                    st, iters = G.run_stats(cap=64)
                    res.append((st.iterations, st.reached, st.slots,
                                [(iters[i].frontier, iters[i].slots) for i in range(st.iterations + 1)]))
                assert res[0] == res[1] == res[2]
    G.close()


@pytest.mark.parametrize("queue", [1, 0])
def test_profiled_loop_times_every_iteration(queue):
    """Profiling with a fixed variant: every iteration of a long run (a 70-vertex
    path: 70 passes, so the queued loop ends inside its ninth batch of eight)
    gets a kernel time, and the results equal the oracle's."""
    g = gg.from_edges(70, [(i, i + 1) for i in range(69)])
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=g.n, split_w=2)
    G.set_option(ss.OPT_PROFILE_QUEUE, queue)
    ss.slimsell_set_profiling(G.h, True)
    for sr in SEMIRINGS:
        for pol in ("full", "slimwork", "pull_filtered"):
            d, p = expected(g, 0)
            dist, parent = run(G, 0, sr, pol)
            np.testing.assert_array_equal(dist, d)
            np.testing.assert_array_equal(parent, p)
            st, iters = G.run_stats(cap=80)
            assert st.iterations == 70
            ns = [iters[i].kernel_ns for i in range(1, st.iterations + 1)]
            assert all(x > 0 for x in ns), (sr, pol, ns)
            assert st.iter_kernel_ms > 0
    ss.slimsell_set_profiling(G.h, False)
    G.close()


def test_edge_cases():
    cases = [
        gg.from_edges(1, []),                                      # single vertex, no edges
        gg.from_edges(5, [(0, 1)]),                                # isolated vertices
        gg.from_edges(70, [(i, i + 1) for i in range(69)]),        # long path, ragged n
        gg.from_edges(40, [(0, i) for i in range(1, 40)]),         # star: hub chunk split
        gg.from_edges(33, [(i, j) for i in range(33) for j in range(i + 1, 33)]),  # complete
        gg.from_edges(9, [(0, 1), (1, 2), (5, 6), (6, 7), (7, 5)]),  # disconnected
        gg.lattice(17, 0.0, seed=1),
    ]
    for g in cases:
        for C, split_w, smem in [(8, 0, 0), (32, 4, 16), (64, 2, 212992)]:
            G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=g.n, split_w=split_w)
            G.set_option(ss.OPT_SMEM_BYTES, smem)
            for r in sorted({0, g.n - 1, g.n // 2}):
                d, p = expected(g, r)
                for sr in SEMIRINGS:
                    for pol in ("full", "slimwork", "pull_filtered", "push", "heuristic"):
                        dist, parent = run(G, r, sr, pol)
                        np.testing.assert_array_equal(dist, d, err_msg=f"{g.name} {sr} {pol} r={r}")
                        np.testing.assert_array_equal(parent, p, err_msg=f"{g.name} {sr} {pol}")
            G.close()


def test_lattice_and_er_parity():
    for g in [gg.lattice(64, 0.05, seed=1), gg.erdos_renyi(1 << 14, 16.0, seed=1)]:
        G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=1024)
        G.set_option(ss.OPT_SMEM_BYTES, 1024)  # most frontier bits read from global memory
        for r in gg.roots(g, 2, seed=2):
            d, p = expected(g, r)
            for sr in ("selmax", "tropical"):
                dist, parent = run(G, r, sr, "slimwork")
                np.testing.assert_array_equal(dist, d)
                np.testing.assert_array_equal(parent, p)
                check_stats(G, g, r, sr)
        G.close()


def test_outputs_optional():
    g = gg.kronecker(9, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    r = int(gg.roots(g, 1, seed=1)[0])
    d, _ = expected(g, r)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    ss.slimsell_bfs(G.h, r, ss.TROPICAL, ss.V_SLIMWORK, dist, None)
    np.testing.assert_array_equal(dist.cpu().numpy(), d)
    ss.slimsell_bfs(G.h, r, ss.BOOLEAN, ss.V_SLIMWORK, None, None)  # nothing written, still runs
    G.close()


def test_invalid_arguments_on_gpu():
    g = gg.kronecker(8, seed=2)
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(ss.SlimSellError) as e:
        ss.slimsell_bfs(G.h, g.n, 0, 1, dist, None)
    assert e.value.status == 1
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs(G.h, 0, 7, 1, dist, None)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_bfs(G.h, 0, 0, 99, dist, None)
    with pytest.raises(ss.SlimSellError):
        ss.slimsell_selector_load(G.h, np.zeros(10, dtype=np.float32))
    G.close()


@pytest.mark.parametrize("sr", SEMIRINGS)
@pytest.mark.parametrize("pol", ["slimwork", "pull_filtered", "heuristic"])
def test_kron22_sampled_parity(sr, pol):
    """Full-size Kronecker scale 22 (the main benchmark graph), 2 roots, SlimWork + SlimChunk."""
    g = _kron22()
    G = _kron22_handle()
    for r in gg.roots(g, 2, seed=2):
        d, p = expected(g, r)
        dist, parent = run(G, r, sr, pol)
        np.testing.assert_array_equal(dist, d)
        np.testing.assert_array_equal(parent, p)
        st, _ = G.run_stats()
        assert st.reached_degree == 2 * oracle.reached_edges(g.row_ptr, d)


_cache = {}


def _kron22():
    if "g" not in _cache:
        _cache["g"] = gg.kronecker(22, seed=1)
    return _cache["g"]


def _kron22_handle():
    if "G" not in _cache:
        g = _kron22()
        _cache["G"] = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=32, sigma=g.n, split_w=1024)
    return _cache["G"]


@pytest.mark.parametrize("blocks", [0, 1, 2])
def test_push_block_sparse_frontier(blocks):
    """The push variant with the frontier seen block-sparse (chunks of C rows
    pushed as blocks with coalesced column reads), per row, or mixed: every
    semiring, C, sigma (sigma = 1 pads hub chunks heavily) and split width give
    the oracle's distances and parents, for the push policy and the adaptive
    schedules that use it."""
    graphs = [gg.kronecker(13, seed=9), gg.lattice(40, 0.05, seed=4), gg.erdos_renyi(3000, 6.0, seed=5)]
    for g in graphs:
        for C, sigma, split_w in [(32, 0, 256), (8, 1, 16), (64, 128, 0), (16, 1, 64)]:
            G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma or g.n, split_w=split_w)
            G.set_option(ss.OPT_PUSH_BLOCKS, blocks)
            for r in gg.roots(g, 2, seed=13):
                d, p = expected(g, r)
                for sr in SEMIRINGS:
                    for pol in ("push", "heuristic"):
                        dist, parent = run(G, r, sr, pol)
                        np.testing.assert_array_equal(dist, d, err_msg=f"{g.name} C={C} {sr} {pol}")
                        np.testing.assert_array_equal(parent, p, err_msg=f"{g.name} C={C} {sr} {pol}")
            G.close()
    with pytest.raises(ss.SlimSellError):
        G = ss.SlimSellGraph.from_host(graphs[0].row_ptr, graphs[0].col)
        try:
            G.set_option(ss.OPT_PUSH_BLOCKS, 3)
        finally:
            G.close()


def test_sell_format_in_the_production_pull():
    """The pull over the Sell-C-sigma arrays (explicit values, padding column 0
    with the semiring's zero) gives the oracle's distances and parents for every
    semiring, C and sigma with the full and SlimWork passes; other policies are
    refused with that format, and switching back restores SlimSell."""
    for g in [gg.kronecker(12, seed=3), gg.lattice(33, 0.05, seed=2), gg.from_edges(5, [(0, 1), (3, 4)])]:
        for C, sigma, split_w in [(32, 0, 64), (8, 1, 4), (64, 128, 0), (16, 1, 16)]:
            G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=C, sigma=sigma or g.n, split_w=split_w)
            G.set_option(ss.OPT_FORMAT, ss.FORMAT_SELL)
            for r in gg.roots(g, 2, seed=6):
                d, p = expected(g, r)
                for sr in SEMIRINGS:
                    for pol in ("slimwork", "full"):
                        dist, parent = run(G, r, sr, pol)
                        np.testing.assert_array_equal(dist, d, err_msg=f"{g.name} C={C} {sr} {pol}")
                        np.testing.assert_array_equal(parent, p, err_msg=f"{g.name} C={C} {sr} {pol}")
            with pytest.raises(ss.SlimSellError):
                run(G, int(gg.roots(g, 1, seed=6)[0]), "tropical", "heuristic")
            G.set_option(ss.OPT_FORMAT, ss.FORMAT_SLIMSELL)
            r = int(gg.roots(g, 1, seed=6)[0])
            d, p = expected(g, r)
            dist, parent = run(G, r, "selmax", "heuristic")
            np.testing.assert_array_equal(dist, d)
            G.close()
