"""Autotuner for the layout parameters (chunk height C, sorting scope sigma,
SlimChunk width w) of a graph: builds the layout for every point of a grid,
times BFS on sample roots with CUDA events (device-side loops), and keeps the
fastest.  Results are cached by a graph signature (n, nnz, log2 degree
histogram), so graphs of the same family and size reuse one search.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (POLICIES, SEMIRINGS, slimsell_bfs, slimsell_build, slimsell_destroy)

GRID = {"C": (8, 16, 32, 64), "sigma": (1, 256, 4096, "n"), "split_w": (256, 1024, 4096)}

_cache: dict = {}


def signature(row_ptr: np.ndarray) -> tuple:
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    hist = np.bincount(np.floor(np.log2(deg[deg > 0])).astype(np.int64), minlength=24)[:24]
    n, nnz = len(deg), int(deg.sum())
    # bucket the histogram coarsely so same-family graphs of one size share a key
    return (n, round(nnz, -max(0, len(str(nnz)) - 2)), tuple(int(round(h / max(1, n) * 50)) for h in hist))


def tune(row_ptr: np.ndarray, col: np.ndarray, roots, semiring: str = "tropical",
         policy: str = "slimwork", grid=GRID, repeats: int = 2, use_cache: bool = True,
         device="cuda"):
    """Returns (best {C, sigma, split_w}, [(params, ms per BFS), ...])."""
    key = (signature(row_ptr), semiring, policy)
    if use_cache and key in _cache:
        return _cache[key]
    n = len(row_ptr) - 1
    rp = torch.from_numpy(np.asarray(row_ptr, dtype=np.int64)).to(device)
    cl = torch.from_numpy(np.asarray(col, dtype=np.int32)).to(device)
    sr, pol = SEMIRINGS[semiring], POLICIES[policy]
    stream = torch.cuda.current_stream()
    table = []
    for C in grid["C"]:
        for sigma in grid["sigma"]:
            s = n if sigma == "n" else int(sigma)
            for w in grid["split_w"]:
                h = slimsell_build(rp, cl, n, int(cl.numel()), C, s, w, stream)
                for r in roots[:1]:  # warm-up: builds the loop graph
                    slimsell_bfs(h, int(r), sr, pol, None, None, stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(repeats):
                    for r in roots:
                        slimsell_bfs(h, int(r), sr, pol, None, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / (repeats * len(roots))
                slimsell_destroy(h)
                table.append(({"C": C, "sigma": sigma, "split_w": w}, ms))
    best = min(table, key=lambda t: t[1])[0]
    _cache[key] = (best, table)
    return best, table
