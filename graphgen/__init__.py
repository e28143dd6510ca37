"""Seeded synthetic graph inputs (Kronecker, lattice, Erdos-Renyi) as cleaned CSR.

Input preparation shared by the CPU oracle, the tests and the benchmark.  It
holds none of the BFS method's arithmetic: edges are drawn from a
counter-based generator, labels are permuted, and the edge list is
symmetrised, stripped of self-loops and duplicates and stored as CSR
(``row_ptr`` int64[n+1], ``col`` int32[nnz], rows sorted by ascending id).

The graph families follow the evaluation setup of Section IV ("Selection of
Benchmarks and Parameters"): Graph500-style Kronecker graphs with initiator
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05) and Erdos-Renyi graphs; 2-D lattices
with random edge deletion stand in for high-diameter road networks
(Table "graphs", rca).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

STREAM_ROOT = 5


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
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
    lib.gg_rand.restype = ctypes.c_uint64
    lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    lib.gg_kronecker_edges.restype = ctypes.c_int
    lib.gg_kronecker_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                       i32p, i32p]
    lib.gg_permutation.restype = ctypes.c_int
    lib.gg_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p]
    lib.gg_lattice_edges.restype = ctypes.c_int64
    lib.gg_lattice_edges.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, i32p, i32p]
    lib.gg_er_edges.restype = ctypes.c_int
    lib.gg_er_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
    lib.gg_edges_to_csr.restype = ctypes.c_int64
    lib.gg_edges_to_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i64p,
                                    i32p, ctypes.c_int64]
    lib.gg_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


@dataclass
class Graph:
    """Cleaned undirected graph in CSR form (both directions stored)."""
    n: int
    row_ptr: np.ndarray  # int64[n + 1]
    col: np.ndarray      # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        """Undirected edges (nnz / 2)."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def edges_to_csr(n: int, src: np.ndarray, dst: np.ndarray, relabel: np.ndarray | None = None,
                 name: str = "") -> Graph:
    """Symmetrise, drop self-loops and duplicates, and build CSR."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cap = 2 * m
    col = np.empty(max(cap, 1), dtype=np.int32)
    rl = None
    if relabel is not None:
        relabel = np.ascontiguousarray(relabel, dtype=np.int32)
        rl = _p32(relabel)
    nnz = lib.gg_edges_to_csr(n, m, _p32(src), _p32(dst), rl, _p64(row_ptr), _p32(col), cap)
    if nnz < 0:
        raise RuntimeError(f"gg_edges_to_csr failed ({nnz})")
    col = col[:nnz].copy() if nnz < col.shape[0] else col
    return Graph(n=n, row_ptr=row_ptr, col=col, name=name)


def permutation(n: int, seed: int) -> np.ndarray:
    lib = _load()
    perm = np.empty(max(n, 1), dtype=np.int32)
    if lib.gg_permutation(n, seed, _p32(perm)) != 0:
        raise RuntimeError("gg_permutation failed")
    return perm[:n]


def kronecker(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19,
              c: float = 0.19, seed: int = 1, permute: bool = True) -> Graph:
    """Graph500-style Kronecker graph: 2^scale vertices, edgefactor * 2^scale draws."""
    lib = _load()
    n = 1 << scale
    m = edgefactor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if lib.gg_kronecker_edges(scale, m, a, b, c, seed, _p32(src), _p32(dst)) != 0:
        raise RuntimeError("gg_kronecker_edges failed")
    relabel = permutation(n, seed) if permute else None
    g = edges_to_csr(n, src, dst, relabel, name=f"kron{scale}-ef{edgefactor}-s{seed}")
    del src, dst
    return g


def lattice(L: int, p_del: float = 0.05, seed: int = 1, permute: bool = False) -> Graph:
    """L x L four-neighbour lattice with each edge deleted with probability p_del."""
    lib = _load()
    cap = max(2 * L * (L - 1), 1)
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    kept = lib.gg_lattice_edges(L, p_del, seed, _p32(src), _p32(dst))
    if kept < 0:
        raise RuntimeError("gg_lattice_edges failed")
    n = L * L
    relabel = permutation(n, seed) if permute else None
    return edges_to_csr(n, src[:kept], dst[:kept], relabel, name=f"lattice{L}-p{p_del}-s{seed}")


def erdos_renyi(n: int, mean_degree: float = 16.0, seed: int = 1) -> Graph:
    """G(n, M) with M = n * mean_degree / 2 endpoint-pair draws before cleaning."""
    lib = _load()
    M = int(round(n * mean_degree / 2))
    src = np.empty(max(M, 1), dtype=np.int32)
    dst = np.empty(max(M, 1), dtype=np.int32)
    if lib.gg_er_edges(n, M, seed, _p32(src), _p32(dst)) != 0:
        raise RuntimeError("gg_er_edges failed")
    return edges_to_csr(n, src[:M], dst[:M], None, name=f"er{n}-d{mean_degree}-s{seed}")


def from_edges(n: int, edges, name: str = "") -> Graph:
    """Small hand-made graphs from an iterable of (u, v) pairs."""
    e = np.asarray(list(edges), dtype=np.int32).reshape(-1, 2)
    return edges_to_csr(n, e[:, 0], e[:, 1], None, name=name)


def roots(g: Graph, k: int, seed: int, distinct: bool = True) -> np.ndarray:
    """k roots drawn from (seed, root stream) among vertices of degree >= 1."""
    lib = _load()
    deg = g.degrees()
    if not np.any(deg > 0):
        raise ValueError("graph has no edges")
    out, seen, ctr = [], set(), 0
    while len(out) < k:
        r = int(lib.gg_rand(seed, STREAM_ROOT, ctr) % g.n)
        ctr += 1
        if deg[r] < 1 or (distinct and r in seen):
            continue
        seen.add(r)
        out.append(r)
    return np.asarray(out, dtype=np.int32)


def mlp_weights(seed: int, scale: float = 0.3) -> np.ndarray:
    """Seeded fp32 parameters for the 16-64-64-4 selector MLP (5508 values, in the
    order W1[16][64], b1, W2[64][64], b2, W3[64][4], b3); He-style normal weights
    times `scale`, biases drawn small."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, scale * np.sqrt(2.0 / 16), (16, 64)), rng.normal(0, 0.05, 64),
             rng.normal(0, scale * np.sqrt(2.0 / 64), (64, 64)), rng.normal(0, 0.05, 64),
             rng.normal(0, scale * np.sqrt(2.0 / 64), (64, 4)), rng.normal(0, 0.05, 4)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def num_threads() -> int:
    return int(_load().gg_num_threads())
