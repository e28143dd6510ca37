"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument checks reject bad calls before any device work (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2010_09913_gb300 as ss


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(slimsell_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    ss.build()
    return ss.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "slimsell_build" in names and "slimsell_bfs" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(ss.exported_symbols()) <= set(names)


def test_version_and_error_strings(lib):
    assert "sm_103a" in ss.slimsell_version()
    assert isinstance(ss.slimsell_last_error(), str)


def test_build_rejects_bad_arguments_on_host(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    # bad C
    assert lib.slimsell_build(fake, fake, 10, 20, 12, 10, 0, None, ctypes.byref(h)) == 1
    assert "C must be" in ss.slimsell_last_error()
    assert h.value is None
    # n < 1, negative nnz, sigma < 1, split_w < 0, NULL row_ptr
    assert lib.slimsell_build(fake, fake, 0, 20, 32, 10, 0, None, ctypes.byref(h)) == 1
    assert lib.slimsell_build(fake, fake, 10, -1, 32, 10, 0, None, ctypes.byref(h)) == 1
    assert lib.slimsell_build(fake, fake, 10, 20, 32, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.slimsell_build(fake, fake, 10, 20, 32, 10, -5, None, ctypes.byref(h)) == 1
    assert lib.slimsell_build(None, fake, 10, 20, 32, 10, 0, None, ctypes.byref(h)) == 1
    assert lib.slimsell_build(fake, fake, 10, 20, 32, 10, 0, None, None) == 1


def test_null_handle_rejected(lib):
    assert lib.slimsell_bfs(None, 0, 0, 1, None, None, None) == 1
    assert lib.slimsell_get_info(None, None) == 1
    assert lib.slimsell_set_profiling(None, 1) == 1
    lib.slimsell_destroy(None)  # no-op


def test_extension_entry_points_reject_null_on_host(lib):
    """Multi-source BFS (with and without parents), the format comparison and
    betweenness centrality refuse a NULL handle or output before any CUDA call."""
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert lib.slimsell_bfs_multi(None, fake, 4, 1, None, None) == 1
    assert lib.slimsell_bfs_multi_parents(None, fake, 4, 1, None, fake, None) == 1
    assert lib.slimsell_bfs_multi_parents(fake, None, 4, 1, None, None, None) == 1
    assert "NULL" in ss.slimsell_last_error()
    assert lib.slimsell_bfs_spmv(None, 0, 0, 0, fake, None, None) == 1
    assert lib.slimsell_bfs_spmv(fake, 0, 0, 0, None, None, None) == 1
    assert lib.slimsell_bc(None, fake, 1, fake, None, None) == 1
    assert lib.slimsell_bc(fake, None, 1, fake, None, None) == 1
    assert lib.slimsell_bc(fake, fake, 1, None, None, None) == 1
    assert lib.slimsell_get_values(None, fake, None) == 1
    assert lib.slimsell_get_values(fake, None, None) == 1
    assert "NULL" in ss.slimsell_last_error()
