"""Input generators: cleaned symmetric CSR, determinism, family shapes (no GPU)."""
import numpy as np

import graphgen as gg


def check_clean(g):
    deg = g.degrees()
    src = np.repeat(np.arange(g.n), deg)
    assert np.all(src != g.col), "self-loop"
    for v in range(0, g.n, max(1, g.n // 200)):
        row = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.all(np.diff(row) > 0), "unsorted or duplicate row"
    # symmetric: the multiset of (u, v) equals the multiset of (v, u)
    a = np.sort(src.astype(np.int64) * g.n + g.col)
    b = np.sort(g.col.astype(np.int64) * g.n + src)
    assert np.array_equal(a, b)


def test_kronecker_clean_deterministic():
    g1 = gg.kronecker(12, seed=3)
    g2 = gg.kronecker(12, seed=3)
    g3 = gg.kronecker(12, seed=4)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col, g2.col)
    assert not np.array_equal(g1.col[:1000], g3.col[:1000])
    check_clean(g1)
    assert g1.n == 4096 and 0 < g1.nnz <= 2 * 16 * 4096
    # skewed degrees: the largest degree is far above the mean
    assert g1.degrees().max() > 20 * g1.degrees().mean()


def test_kronecker_quadrant_frequencies():
    # fraction of generated (u, v) bit pairs per quadrant approaches (a, b, c, d)
    g = gg.kronecker(10, seed=9, permute=False)
    check_clean(g)
    deg = g.degrees()
    # with d = 0.05 the low ids (bit 0) dominate: vertex 0 is the hub before permutation
    assert int(np.argmax(deg)) == 0


def test_lattice_and_er():
    L = 30
    full = gg.lattice(L, 0.0, seed=1)
    assert full.nnz == 4 * L * (L - 1)
    check_clean(full)
    cut = gg.lattice(L, 0.05, seed=1)
    kept = cut.nnz / full.nnz
    assert 0.9 < kept < 0.99
    er = gg.erdos_renyi(20000, 16.0, seed=2)
    check_clean(er)
    assert abs(er.nnz / er.n - 16.0) < 0.5


def test_roots_have_degree():
    g = gg.kronecker(10, seed=2)
    r = gg.roots(g, 50, seed=3)
    assert len(set(r.tolist())) == 50
    assert np.all(g.degrees()[r] >= 1)
    assert np.array_equal(r, gg.roots(g, 50, seed=3))


def test_permutation_is_bijection():
    p = gg.permutation(1000, 5)
    assert np.array_equal(np.sort(p), np.arange(1000))
