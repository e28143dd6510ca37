"""The allocation-free degree sort agrees with the ordering slimsell_build uses.

slimsell_sigma_sort_noalloc serves callers that must not allocate device
memory (device memory fully reserved by another allocator, or loops that cannot
pay for cudaMalloc's synchronisation); it keeps its scratch in one fixed device
array shared by all calls.  These tests call it through the C ABI twice in a
row and compare each result with the permutation exported from a handle built
by slimsell_build, exactly (the permutation is integer data); the cases at the
array's size limit (n = 2^19, the widest keys) are also compared with the
oracle's layout.  They pass both alone in a fresh process and after the rest of
the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2010_09913_gb300 as ss

pytestmark = pytest.mark.gpu

MAX_N = 1 << 19


def reference_perm(g, sigma):
    # C = 8: every sigma below is a multiple of 8, so slimsell_build keeps it as given
    G = ss.SlimSellGraph.from_host(g.row_ptr, g.col, C=8, sigma=sigma, split_w=0)
    perm = G.export_layout()["perm"][: g.n].cpu().numpy()
    G.close()
    return perm


def noalloc_perm(g, sigma):
    lib = ss.lib()
    rp = torch.from_numpy(g.row_ptr).cuda()
    out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    status = lib.slimsell_sigma_sort_noalloc(rp.data_ptr(), g.n, sigma, out.data_ptr(), stream)
    assert status == 0, ss.slimsell_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_sort_matches_build_on_two_calls_in_a_row():
    ss.build()
    big = gg.kronecker(13, seed=6)      # n = 8192
    small = gg.lattice(37, 0.05, seed=3)  # n = 1369, different degree range
    cases = [(big, big.n), (small, 128), (big, 1000), (big, 1)]
    for g, sigma in cases:
        want = reference_perm(g, sigma)
        first = noalloc_perm(g, sigma)
        second = noalloc_perm(g, sigma)  # the shared scratch keeps the last call's contents
        np.testing.assert_array_equal(first, want)
        np.testing.assert_array_equal(second, want)


def test_noalloc_sort_at_the_size_limit():
    """n = 2^19 exactly: the scratch offsets (histograms of 128 tiles, the scan's
    partials) at their largest; sigma = 8 gives 65,536 windows, so the keys carry
    19 + 16 bits and the sort makes five passes."""
    ss.build()
    g = gg.kronecker(19, seed=2)
    assert g.n == MAX_N
    for sigma in (g.n, 8):
        want = oracle.slimsell_layout(g.row_ptr, g.col, 8, sigma)["perm"]
        np.testing.assert_array_equal(reference_perm(g, sigma), want)
        first = noalloc_perm(g, sigma)
        second = noalloc_perm(g, sigma)
        np.testing.assert_array_equal(first, want)
        np.testing.assert_array_equal(second, want)


def test_noalloc_rejects_sizes_beyond_its_array():
    ss.build()
    lib = ss.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.slimsell_sigma_sort_noalloc(fake, MAX_N + 1, 4, fake, None) == 1
    assert str(MAX_N) in ss.slimsell_last_error()
    assert lib.slimsell_sigma_sort_noalloc(fake, 0, 4, fake, None) == 1
    assert lib.slimsell_sigma_sort_noalloc(fake, 100, 0, fake, None) == 1
