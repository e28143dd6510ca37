"""Host logic of the layout autotuner (no GPU): the library's cache key
(slimsell_tune_signature) and match rule (slimsell_tune_match) group graphs of
one family and size and separate other sizes and shapes; the key's values are
pinned by hand on small graphs."""
import numpy as np
import pytest

import graphgen as gg
import paper_2010_09913_gb300 as ss


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ss.build()


def sig(g):
    return ss.slimsell_tune_signature(g.row_ptr)


def test_signature_by_hand():
    # star with 5 leaves: degrees 5 (bucket floor(log2 5) = 2) and 1 (bucket 0)
    s = sig(gg.from_edges(6, [(0, i) for i in range(1, 6)]))
    assert s.n == 6 and s.nnz_rounded == 10
    hist = list(s.hist)
    assert hist[0] == 42 and hist[2] == 8  # 50 * 5/6 = 41.7 and 50 * 1/6 = 8.3, rounded
    assert sum(hist) == 50
    # ten isolated vertices: nothing counted
    s = ss.slimsell_tune_signature(np.zeros(11, dtype=np.int64))
    assert s.n == 10 and s.nnz_rounded == 0 and sum(s.hist) == 0


@pytest.mark.parametrize("nnz,want", [(99, 99), (100, 100), (12345, 12000), (12567, 13000), (995, 1000)])
def test_nnz_rounded_to_two_digits(nnz, want):
    rp = np.array([0, nnz], dtype=np.int64)  # one vertex carrying every entry
    assert ss.slimsell_tune_signature(rp).nnz_rounded == want


def test_match_groups_seeds_of_one_family_and_size():
    base = sig(gg.kronecker(12, seed=1))
    for seed in (2, 3, 4):
        assert ss.slimsell_tune_match(base, sig(gg.kronecker(12, seed=seed)))


def test_match_separates_size_and_shape():
    base = sig(gg.kronecker(12, seed=1))
    assert not ss.slimsell_tune_match(base, sig(gg.kronecker(13, seed=1)))
    lat = sig(gg.lattice(64, 0.05, seed=1))  # n = 4096 like Kronecker 12, another shape
    assert lat.n == base.n
    assert not ss.slimsell_tune_match(base, lat)


def test_match_tolerance_is_three_units():
    a = sig(gg.kronecker(12, seed=1))
    b = sig(gg.kronecker(12, seed=1))
    b.hist[3] += 2
    b.hist[7] -= 1
    assert ss.slimsell_tune_match(a, b)       # L1 distance 3
    b.hist[9] += 1
    assert not ss.slimsell_tune_match(a, b)   # 4
    c = sig(gg.kronecker(12, seed=1))
    c.n += 1
    assert not ss.slimsell_tune_match(a, c)
