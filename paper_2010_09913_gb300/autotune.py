"""Autotuner for the layout parameters (chunk height C, sorting scope sigma,
SlimChunk width w) of a graph: builds the layout for every point of a grid,
times BFS on sample roots with CUDA events (device-side loops), and keeps the
fastest.  Results are cached by a graph signature (n, nnz, log2 degree
histogram); a graph reuses a cached search when its n and rounded nnz match and
its histogram is within HIST_TOLERANCE (L1, in histogram units) of the cached
one, so graphs of the same family and size share one search even where the
coarse histogram buckets of two seeds fall on opposite sides of a bucket edge.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (POLICIES, SEMIRINGS, slimsell_bfs, slimsell_build, slimsell_destroy)

GRID = {"C": (8, 16, 32, 64), "sigma": (1, 256, 4096, "n"), "split_w": (256, 1024, 4096)}

_cache: dict = {}
HIST_TOLERANCE = 3


def signature(row_ptr: np.ndarray) -> tuple:
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64))
    hist = np.bincount(np.floor(np.log2(deg[deg > 0])).astype(np.int64), minlength=24)[:24]
    n, nnz = len(deg), int(deg.sum())
    # bucket the histogram coarsely so same-family graphs of one size share a key
    return (n, round(nnz, -max(0, len(str(nnz)) - 2)), tuple(int(round(h / max(1, n) * 50)) for h in hist))


def grid_key(grid) -> tuple:
    return tuple(sorted((k, tuple(v)) for k, v in grid.items()))


def lookup(cache: dict, key):
    """The cached entry for `key` = (signature, semiring, policy[, grid key]): an
    exact match, else the closest cached signature with the same n, rounded nnz
    and the same remaining fields whose histogram differs by at most
    HIST_TOLERANCE (L1); None if none."""
    if key in cache:
        return cache[key]
    (n, nnz, hist), rest = key[0], key[1:]
    best, best_d = None, HIST_TOLERANCE + 1
    for k, entry in cache.items():
        sig = k[0]
        if k[1:] != rest or sig[0] != n or sig[1] != nnz:
            continue
        d = sum(abs(a - b) for a, b in zip(sig[2], hist))
        if d < best_d:
            best, best_d = entry, d
    return best


def tune(row_ptr: np.ndarray, col: np.ndarray, roots, semiring: str = "tropical",
         policy: str = "slimwork", grid=GRID, repeats: int = 2, use_cache: bool = True,
         device="cuda"):
    """Returns (best {C, sigma, split_w}, [(params, ms per BFS), ...])."""
    key = (signature(row_ptr), semiring, policy, grid_key(grid))
    if use_cache:
        hit = lookup(_cache, key)
        if hit is not None:
            return hit
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
