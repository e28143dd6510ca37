"""Pins for the oracle's SlimSell layout (no GPU).

* a hand-derived layout of a 5-vertex star (C = 4);
* the storage identity |col| = sum_i C * cl_i = nnz + P and the word counts of
  Table "sizes" (SlimSell 2m + 2n/C + P vs Sell-C-sigma 4m + 2n/C + P, where
  P counts padded cells, so Sell-C-sigma's P is twice SlimSell's);
* the padding bound P <= C * max degree for sigma = n (Section III-A);
* sigma = 1 keeps the identity order; sigma < C never lowers padding below
  the no-sort layout restricted to chunk-local reordering;
* every row's slots hold exactly its neighbours, descending original id.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle


def test_star_layout_by_hand():
    g = gg.from_edges(5, [(0, i) for i in range(1, 5)])
    L = oracle.slimsell_layout(g.row_ptr, g.col, C=4, sigma=5)
    assert L["perm"].tolist() == [0, 1, 2, 3, 4]
    assert L["cl"].tolist() == [4, 1]
    assert L["cs"].tolist() == [0, 16, 20]
    assert L["col"].tolist() == [4, 0, 0, 0,
                                 3, -1, -1, -1,
                                 2, -1, -1, -1,
                                 1, -1, -1, -1,
                                 0, -1, -1, -1]
    assert L["padding"] == 12
    L2 = oracle.slimsell_layout(g.row_ptr, g.col, C=4, sigma=5, split_w=3)
    assert L2["items"].tolist() == [[0, 0, 3], [0, 3, 4], [1, 0, 1]]


def test_sort_moves_hub_first():
    # vertex 3 has the largest degree; with sigma = n it becomes row 0
    g = gg.from_edges(6, [(3, 0), (3, 1), (3, 2), (3, 4), (0, 1), (5, 4)])
    L = oracle.slimsell_layout(g.row_ptr, g.col, C=2, sigma=6)
    # degrees: 0:2 1:2 2:1 3:4 4:2 5:1 -> order 3, 0, 1, 4, 2, 5
    assert L["perm"].tolist() == [3, 0, 1, 4, 2, 5]
    assert L["cl"].tolist() == [4, 2, 1]
    inv = L["invperm"]
    # chunk 0 = rows (3, 0); column 0 holds the max-id neighbours 4 and 3
    assert L["col"][:2].tolist() == [inv[4], inv[3]]


def test_sigma_rounds_up_to_a_multiple_of_C():
    """Section IV takes sigma as a multiple of C: any other sigma > 1 acts as the
    next multiple (here 5 -> 8 and 9 -> 12 with C = 4); sigma = 1 keeps the order."""
    g = gg.kronecker(9, seed=12)
    for s, s_eff in [(5, 8), (9, 12), (8, 8)]:
        a = oracle.slimsell_layout(g.row_ptr, g.col, C=4, sigma=s)
        b = oracle.slimsell_layout(g.row_ptr, g.col, C=4, sigma=s_eff)
        np.testing.assert_array_equal(a["perm"], b["perm"])
        np.testing.assert_array_equal(a["col"], b["col"])
    # by hand: degrees 2, 0, 1, 1; C = 2 and sigma = 3 give one window of 4
    # vertices (not 3 + 1), so the order is 0, 2, 3, 1 (unrounded: 0, 2, 1, 3)
    h = gg.from_edges(4, [(0, 2), (0, 3)])
    L = oracle.slimsell_layout(h.row_ptr, h.col, C=2, sigma=3)
    assert L["perm"].tolist() == [0, 2, 3, 1]


def check_layout(g, C, sigma, split_w=0):
    L = oracle.slimsell_layout(g.row_ptr, g.col, C, sigma, split_w)
    if sigma > 1:
        sigma = -(-sigma // C) * C  # the window the layout uses
    n, deg = g.n, g.degrees()
    perm, inv, cl, cs, col = L["perm"], L["invperm"], L["cl"], L["cs"], L["col"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(inv[perm], np.arange(n))
    n_c = (n + C - 1) // C
    assert cl.shape[0] == n_c and cs.shape[0] == n_c + 1
    assert np.all(np.diff(cs) == C * cl)
    # size identity and word counts (m = undirected edges, nnz = 2m)
    P = L["padding"]
    assert col.shape[0] == g.nnz + P and P >= 0
    slim_words = col.shape[0] + 2 * n_c
    sell_words = 2 * col.shape[0] + 2 * n_c
    assert slim_words == 2 * g.m + 2 * n_c + P
    # Sell-C-sigma pads val and col alike, so its padded cells are 2P slots
    assert sell_words == 4 * g.m + 2 * n_c + 2 * P
    # row content: neighbours in descending original id, then -1 padding
    for r in range(n):
        v = perm[r]
        i, l = divmod(r, C)
        slots = col[cs[i] + np.arange(cl[i]) * C + l]
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]][::-1]
        assert np.array_equal(slots[: nb.shape[0]], inv[nb])
        assert np.all(slots[nb.shape[0]:] == -1)
    for r in range(n, n_c * C):  # padding rows are empty
        i, l = divmod(r, C)
        assert np.all(col[cs[i] + np.arange(cl[i]) * C + l] == -1)
    # sort order inside windows: degree descending, ties by ascending id
    if sigma > 1:
        for w0 in range(0, n, sigma):
            blk = perm[w0:w0 + sigma]
            assert set(blk.tolist()) == set(range(w0, min(w0 + sigma, n)))
            key = np.stack([-deg[blk], blk])
            assert all(tuple(key[:, t]) < tuple(key[:, t + 1]) for t in range(blk.shape[0] - 1))
    else:
        assert np.array_equal(perm, np.arange(n))
    # chunk length is the longest row
    dr = np.zeros(n_c * C, dtype=np.int64)
    dr[:n] = deg[perm]
    assert np.array_equal(cl, dr.reshape(n_c, C).max(axis=1))
    if sigma >= n:  # Section III-A: total storage <= nnz + C * max degree
        assert P <= C * int(deg.max())
    # split table covers every chunk exactly once, in order
    items = L["items"]
    for ci in range(n_c):
        it = items[items[:, 0] == ci]
        assert it[0, 1] == 0 and it[-1, 2] == cl[ci]
        assert np.all(it[1:, 1] == it[:-1, 2])
        if split_w > 0:
            assert np.all(it[:, 2] - it[:, 1] <= max(split_w, 0) if cl[ci] > split_w else True)
    return L


@pytest.mark.parametrize("C", [4, 8, 32])
@pytest.mark.parametrize("sigma_kind", ["one", "small", "full"])
def test_layout_rules_kronecker(C, sigma_kind):
    g = gg.kronecker(8, seed=5)
    sigma = {"one": 1, "small": 4 * C, "full": g.n}[sigma_kind]
    check_layout(g, C, sigma, split_w=16)


def test_layout_ragged_tail_and_lattice():
    g = gg.lattice(13, 0.1, seed=2)  # n = 169, not a multiple of C
    for C in (8, 16, 64):
        check_layout(g, C, g.n, split_w=3)
        check_layout(g, C, 40)


def test_full_sort_reduces_padding():
    g = gg.kronecker(10, seed=1)
    P1 = oracle.slimsell_layout(g.row_ptr, g.col, 32, 1)["padding"]
    Pn = oracle.slimsell_layout(g.row_ptr, g.col, 32, g.n)["padding"]
    assert Pn < P1
    # sigma smaller than C reorders rows inside windows but cannot beat the full sort
    Ps = oracle.slimsell_layout(g.row_ptr, g.col, 32, 8)["padding"]
    assert Ps >= Pn
