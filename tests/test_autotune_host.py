"""Host logic of the layout autotuner (no GPU): the cache key and its tolerant
lookup group graphs of one family and size and separate other sizes, shapes,
semirings and policies."""
import numpy as np

import graphgen as gg
from paper_2010_09913_gb300 import autotune


def key(g, sr="tropical", pol="slimwork"):
    return (autotune.signature(g.row_ptr), sr, pol)


def test_lookup_groups_seeds_of_one_family_and_size():
    cache = {key(gg.kronecker(12, seed=1)): "k12"}
    for seed in (2, 3, 4):  # seed 2's histogram sits across a bucket edge from seed 1's
        assert autotune.lookup(cache, key(gg.kronecker(12, seed=seed))) == "k12"


def test_lookup_separates_size_shape_semiring_and_policy():
    cache = {key(gg.kronecker(12, seed=1)): "k12"}
    assert autotune.lookup(cache, key(gg.kronecker(13, seed=1))) is None
    lat = gg.lattice(64, 0.05, seed=1)  # n = 4096 like Kronecker 12, another shape
    assert autotune.signature(lat.row_ptr)[0] == 4096
    assert autotune.lookup(cache, key(lat)) is None
    g = gg.kronecker(12, seed=1)
    assert autotune.lookup(cache, key(g, sr="real")) is None
    assert autotune.lookup(cache, key(g, pol="heuristic")) is None


def test_lookup_prefers_exact_then_closest():
    g = gg.kronecker(12, seed=1)
    (n, nnz, hist), sr, pol = key(g)
    near = (n, nnz, tuple(h + (1 if i == 0 else 0) for i, h in enumerate(hist)))
    far = (n, nnz, tuple(h + (3 if i == 0 else 0) for i, h in enumerate(hist)))
    cache = {(far, sr, pol): "far", (near, sr, pol): "near"}
    assert autotune.lookup(cache, key(g)) == "near"
    cache[key(g)] = "exact"
    assert autotune.lookup(cache, key(g)) == "exact"


def test_signature_of_degree_free_graph():
    rp = np.zeros(11, dtype=np.int64)  # ten isolated vertices
    n, nnz, hist = autotune.signature(rp)
    assert n == 10 and nnz == 0 and sum(hist) == 0 and len(hist) == 24


def test_lookup_keeps_grids_apart():
    g = gg.kronecker(12, seed=1)
    small = autotune.grid_key({"C": (16, 32), "sigma": (1, "n"), "split_w": (256,)})
    cache = {key(g) + (autotune.grid_key(autotune.GRID),): "full grid"}
    assert autotune.lookup(cache, key(g) + (small,)) is None
    assert autotune.lookup(cache, key(gg.kronecker(12, seed=2)) + (autotune.grid_key(autotune.GRID),)) == "full grid"
