"""Layout autotuner (C x sigma x split width), marshalling only: the grid
search, its CUDA-event timing and the signature cache run in the library
(``slimsell_autotune`` in include/slimsell.h).  A grid is a dict of tuples;
sigma "n" means a global sort."""
from __future__ import annotations

import numpy as np
import torch

from . import POLICIES, SEMIRINGS, slimsell_autotune

GRID = {"C": (8, 16, 32, 64), "sigma": (1, 256, 4096, "n"), "split_w": (256, 1024, 4096)}


def _sigma_out(s: int):
    return "n" if s == 0 else int(s)


def tune(row_ptr: np.ndarray, col: np.ndarray, roots, semiring: str = "tropical",
         policy: str = "slimwork", grid=GRID, repeats: int = 2, use_cache: bool = True,
         device="cuda", with_result: bool = False):
    """Returns (best {C, sigma, split_w}, [(params, ms per BFS), ...]) and, with
    with_result, the library's result record as a third element (cached flag,
    points timed)."""
    n = len(row_ptr) - 1
    rp = torch.from_numpy(np.asarray(row_ptr, dtype=np.int64)).to(device)
    cl = torch.from_numpy(np.asarray(col, dtype=np.int32)).to(device)
    if cl.numel() == 0:
        cl = torch.zeros(1, dtype=torch.int32, device=device)[:0]
    sigmas = [0 if s == "n" else int(s) for s in grid["sigma"]]
    res, pts = slimsell_autotune(rp, cl, n, int(np.asarray(col).size), SEMIRINGS[semiring],
                                 POLICIES[policy], roots, grid["C"], sigmas, grid["split_w"],
                                 repeats, use_cache)
    table = [({"C": p.C, "sigma": _sigma_out(p.sigma), "split_w": p.split_w}, p.ms) for p in pts]
    b = res.best
    best = {"C": b.C, "sigma": _sigma_out(b.sigma), "split_w": b.split_w}
    return (best, table, res) if with_result else (best, table)
