"""CPU oracle for SlimSell BFS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it; it exists to say what the right answer is.

* ``bfs_queue``      traditional queue BFS (Section II-C).
* ``dp``             DP transformation p = DP(d) (Section II-C), max-id tie-break.
* ``bfs_semiring``   algebraic BFS over the tropical, real, boolean and sel-max
                     semirings on the plain CSR (Section III-A), dense vectors.
* ``bfs_multi``      k independent queue BFS runs (multi-source extension).
* ``bc``             betweenness centrality over a set of sources (Brandes'
                     dependency accumulation; the paper's future-work algorithms).
* ``slimsell_layout`` Sell-C-sigma / SlimSell layout (Sections II-D and III-B):
                     sigma-window degree sort, chunk tables cs/cl, column-major
                     col with -1 padding, SlimChunk split table (Section III-D).
* ``mlp_*``          fp64 reference of the variant-selector MLP (extension).

Parity status: all functions are pinned by ``tests/test_oracle_*.py`` against
brute force, closed forms, library routines and the BFS invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TROPICAL, REAL, BOOLEAN, SELMAX = 0, 1, 2, 3
SEMIRINGS = {"tropical": TROPICAL, "real": REAL, "boolean": BOOLEAN, "selmax": SELMAX}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (serial C, -O2)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"],
                   check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_bfs_queue.restype = ctypes.c_int64
    lib.oracle_bfs_queue.argtypes = [ctypes.c_int32, i64p, i32p, ctypes.c_int32, i32p]
    lib.oracle_dp.restype = None
    lib.oracle_dp.argtypes = [ctypes.c_int32, i64p, i32p, i32p, ctypes.c_int32, i32p]
    lib.oracle_bfs_semiring.restype = ctypes.c_int64
    lib.oracle_bfs_semiring.argtypes = [ctypes.c_int32, i64p, i32p, ctypes.c_int32, ctypes.c_int32,
                                        i32p, i32p, f64p, i64p, ctypes.c_int32]
    lib.oracle_bfs_multi.restype = ctypes.c_int64
    lib.oracle_bfs_multi.argtypes = [ctypes.c_int32, i64p, i32p, i32p, ctypes.c_int32, i32p]
    lib.oracle_bc.restype = ctypes.c_int32
    lib.oracle_bc.argtypes = [ctypes.c_int32, i64p, i32p, i32p, ctypes.c_int32, f64p]
    _lib = lib
    return lib


def _csr(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return row_ptr, col


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def bfs_queue(row_ptr, col, root: int) -> np.ndarray:
    """Traditional queue BFS: int32 distances, -1 for unreached vertices."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.shape[0] - 1
    dist = np.empty(max(n, 1), dtype=np.int32)
    r = lib.oracle_bfs_queue(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32), int(root),
                             _p(dist, ctypes.c_int32))
    if r < 0:
        raise ValueError(f"oracle_bfs_queue: bad root {root}")
    return dist[:n]


def dp(row_ptr, col, dist, root: int) -> np.ndarray:
    """DP transformation: parent = max-id neighbour one level closer to the root."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.shape[0] - 1
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    parent = np.empty(max(n, 1), dtype=np.int32)
    lib.oracle_dp(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                  _p(dist, ctypes.c_int32), int(root), _p(parent, ctypes.c_int32))
    return parent[:n]


def bfs_semiring(row_ptr, col, root: int, semiring, with_counts: bool = False):
    """Algebraic BFS over one semiring.

    Returns ``(dist, parent, fval, iterations, level_counts)``; ``fval`` holds
    the real-semiring value with which each vertex entered the frontier (the
    number of shortest paths from the root), 1.0 for boolean / sel-max.
    """
    lib = _load()
    if isinstance(semiring, str):
        semiring = SEMIRINGS[semiring]
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.shape[0] - 1
    dist = np.empty(max(n, 1), dtype=np.int32)
    parent = np.empty(max(n, 1), dtype=np.int32)
    fval = np.empty(max(n, 1), dtype=np.float64)
    cap = n + 2
    counts = np.zeros(cap, dtype=np.int64)
    it = lib.oracle_bfs_semiring(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32), int(root),
                                 int(semiring), _p(dist, ctypes.c_int32), _p(parent, ctypes.c_int32),
                                 _p(fval, ctypes.c_double), _p(counts, ctypes.c_int64), cap)
    if it < 0:
        raise ValueError(f"oracle_bfs_semiring failed ({it})")
    levels = counts[: max(int(it), 1)]
    return dist[:n], parent[:n], fval[:n], int(it), levels


def bfs_multi(row_ptr, col, roots) -> np.ndarray:
    """k independent BFS runs; returns dist as a (k, n) int32 array."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.shape[0] - 1
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    k = roots.shape[0]
    dist = np.empty((k, max(n, 1)), dtype=np.int32)
    r = lib.oracle_bfs_multi(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                             _p(roots, ctypes.c_int32), k, _p(dist, ctypes.c_int32))
    if r < 0:
        raise ValueError("oracle_bfs_multi: bad root")
    return dist[:, :n]


def reached_edges(row_ptr, dist) -> int:
    """Undirected edges with an endpoint in the reached set (each counted once).

    In an undirected graph every neighbour of a reached vertex is reached, so
    this is half the degree sum over reached vertices.
    """
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return int(deg[np.asarray(dist) >= 0].sum() // 2)


def bc(row_ptr, col, sources) -> np.ndarray:
    """Betweenness centrality summed over ``sources`` (fp64, Brandes):
    bc[v] = sum over s in sources, t != s, v of sigma_st(v) / sigma_st."""
    lib = _load()
    row_ptr, col = _csr(row_ptr, col)
    n = row_ptr.shape[0] - 1
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.float64)
    r = lib.oracle_bc(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32), _p(src, ctypes.c_int32),
                      int(src.shape[0]), _p(out, ctypes.c_double))
    if r != 0:
        raise ValueError("oracle_bc: bad source")
    return out[:n]


def slimsell_layout(row_ptr, col, C: int, sigma: int, split_w: int = 0):
    """SlimSell layout by definition (Sections II-D, III-B, III-D).

    * Rows are sorted by descending degree inside windows [j*sigma, (j+1)*sigma),
      ties by ascending vertex id; sigma <= 1 keeps the identity order, and any
      other sigma is first rounded up to a multiple of C (the paper takes sigma
      as a multiple of C, Section IV).
    * ``perm[r]`` = vertex stored at row position r; ``invperm[v]`` = its position.
    * Chunk i holds rows [i*C, (i+1)*C); rows beyond n are empty padding rows.
    * ``cl[i]`` = longest row of chunk i; ``cs`` = exclusive prefix sum of C*cl.
    * ``col_s[cs[i] + j*C + l]`` = relabelled id of the j-th neighbour (in
      descending original id order) of row i*C + l, or -1 for padding.
    * Split table: chunk i with cl[i] > split_w (split_w > 0) becomes the items
      (i, j0, min(j0 + split_w, cl[i])) for j0 = 0, split_w, ...; other chunks
      are single items (i, 0, cl[i]).
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int32)
    n = row_ptr.shape[0] - 1
    deg = np.diff(row_ptr)
    ids = np.arange(n, dtype=np.int64)
    if sigma <= 1:
        perm = ids.copy()
    else:
        sigma = -(-int(sigma) // C) * C  # rounded up to a multiple of C
        window = ids // sigma
        perm = np.lexsort((ids, -deg, window))  # primary key: window, then -deg, then id
    invperm = np.empty(n, dtype=np.int64)
    invperm[perm] = ids
    n_c = (n + C - 1) // C
    deg_rows = np.zeros(n_c * C, dtype=np.int64)
    deg_rows[:n] = deg[perm]
    cl = deg_rows.reshape(n_c, C).max(axis=1) if n_c > 0 else np.zeros(0, dtype=np.int64)
    cs = np.zeros(n_c + 1, dtype=np.int64)
    cs[1:] = np.cumsum(C * cl)
    col_s = np.full(int(cs[-1]), -1, dtype=np.int64)
    owner = np.repeat(ids, deg)                       # vertex owning each CSR entry
    e = np.arange(col.shape[0], dtype=np.int64)
    j = row_ptr[owner + 1] - 1 - e                    # position in descending-id order
    r = invperm[owner]
    i, l = r // C, r % C
    col_s[cs[i] + j * C + l] = invperm[col]
    items = []
    for ci in range(n_c):
        L = int(cl[ci])
        if split_w > 0 and L > split_w:
            for j0 in range(0, L, split_w):
                items.append((ci, j0, min(j0 + split_w, L)))
        else:
            items.append((ci, 0, L))
    return {
        "perm": perm.astype(np.int32), "invperm": invperm.astype(np.int32),
        "cl": cl.astype(np.int32), "cs": cs, "col": col_s.astype(np.int32),
        "items": np.asarray(items, dtype=np.int32).reshape(-1, 3),
        "n_c": n_c, "padding": int(cs[-1]) - int(col.shape[0]),
    }
