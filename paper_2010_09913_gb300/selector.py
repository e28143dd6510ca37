"""Training and evaluation of the per-iteration variant selector (an extension).

The selector is a 16-64-64-4 MLP evaluated on the device before every BFS
iteration (``policy="learned"``); its outputs predict the log-time of the four
iteration variants (full pull, SlimWork pull, push, filtered pull) and the
iteration runs the argmin.  Schedules never change BFS results, only time.

* ``collect`` runs every variant as a fixed policy on the same roots, with
  CUDA-event timing of each iteration's kernels, and pairs the features the
  device logged before iteration k with the measured log-times of iteration k
  (all variants follow the same level trajectory, so iteration k is the same
  frontier expansion in every run).
* ``train`` fits the MLP with the library's GPU train-step kernel (masked MSE on
  log-microseconds, Adam); minibatches are contiguous slices of a host-shuffled
  copy, so no tensor arithmetic happens outside the library.
* ``evaluate`` reports the measured cost of the learned, heuristic and fixed
  schedules next to the per-iteration best schedule (the regret baseline).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (N_OUTPUTS, N_PARAMS, OPT_PROFILE_QUEUE, slimsell_get_features,
               slimsell_mlp_train_step, slimsell_selector_load, slimsell_set_option,
               slimsell_set_profiling)

VARIANTS = ["full", "slimwork", "push", "pull_filtered"]


def _profiled_run(G, root: int, semiring: str, policy: str):
    """One BFS with per-iteration kernel times; returns (ns[k], variant[k], features[k]).
    Every variant is timed the same way, one launch and one counter read per
    iteration (the adaptive push cannot be queued ahead), so that the labels
    compare like with like."""
    slimsell_set_profiling(G.h, True)
    slimsell_set_option(G.h, OPT_PROFILE_QUEUE, 0)
    G.bfs(int(root), semiring, policy, want_parent=False)
    st, its = G.run_stats(cap=65536)
    iters = st.iterations
    ns = np.array([its[k].kernel_ns for k in range(1, iters + 1)], dtype=np.float64)
    var = np.array([its[k].variant for k in range(1, iters + 1)], dtype=np.int32)
    feats = slimsell_get_features(G.h, iters + 1)[1:iters + 1]
    slimsell_set_option(G.h, OPT_PROFILE_QUEUE, 1)
    slimsell_set_profiling(G.h, False)
    return ns, var, feats


def collect(G, roots, semiring: str = "tropical", repeats: int = 3, max_per_root: int = 0):
    """Features X [N, 16], log-microsecond targets T [N, 4] and masks M [N, 4].

    max_per_root > 0 keeps that many evenly spaced iterations of each run, so
    that a high-diameter graph (thousands of levels) does not drown the others."""
    xs, ts, ms = [], [], []
    for r in roots:
        per_var, feats = [], None
        for vi, v in enumerate(VARIANTS):
            runs = [_profiled_run(G, int(r), semiring, v) for _ in range(repeats)]
            ns = np.median(np.stack([x[0] for x in runs]), axis=0)
            executed = runs[0][1]
            ok = (executed == vi) | ((vi == 2) & (executed == 4))  # 4: cluster push
            per_var.append((ns, ok))
            if v == "pull_filtered":
                feats = runs[0][2]
        iters = len(per_var[0][0])
        T = np.zeros((iters, N_OUTPUTS), dtype=np.float32)
        M = np.zeros((iters, N_OUTPUTS), dtype=np.float32)
        for vi, (ns, ok) in enumerate(per_var):
            T[:, vi] = np.log(ns / 1000.0 + 1.0)
            M[:, vi] = ok.astype(np.float32)
        keep = np.arange(iters)
        if max_per_root > 0 and iters > max_per_root:
            keep = np.unique(np.linspace(0, iters - 1, max_per_root).round().astype(np.int64))
        xs.append(feats.astype(np.float32)[keep])
        ts.append(T[keep])
        ms.append(M[keep])
    return np.concatenate(xs), np.concatenate(ts), np.concatenate(ms)


def train(X, T, M, steps: int = 3000, lr: float = 3e-3, batch: int = 128, seed: int = 0,
          init=None, device="cuda"):
    """Fit the selector on the GPU; returns (weights float32[5508], final loss)."""
    rng = np.random.default_rng(seed)
    if init is None:
        # He-style initialisation, small biases
        parts = [rng.normal(0, math.sqrt(2.0 / 16), (16, 64)), np.zeros(64),
                 rng.normal(0, math.sqrt(2.0 / 64), (64, 64)), np.zeros(64),
                 rng.normal(0, math.sqrt(2.0 / 64), (64, 4)), np.full(4, float(T[M > 0].mean()) if M.sum() else 0.0)]
        init = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    w = torch.from_numpy(np.asarray(init, dtype=np.float32).copy()).to(device)
    m = torch.zeros(N_PARAMS, device=device)
    v = torch.zeros(N_PARAMS, device=device)
    loss = torch.zeros(1, device=device)
    n = X.shape[0]
    b = min(batch, n)
    step, last = 0, float("nan")
    while step < steps:
        order = rng.permutation(n)
        xd = torch.from_numpy(np.ascontiguousarray(X[order], dtype=np.float32)).to(device)
        td = torch.from_numpy(np.ascontiguousarray(T[order], dtype=np.float32)).to(device)
        md = torch.from_numpy(np.ascontiguousarray(M[order], dtype=np.float32)).to(device)
        for s0 in range(0, n - b + 1, b):
            step += 1
            slimsell_mlp_train_step(w, m, v, step, xd[s0:s0 + b], td[s0:s0 + b], md[s0:s0 + b], lr,
                                    None, loss)
            if step >= steps:
                break
    torch.cuda.synchronize()
    last = float(loss.item())
    return w.cpu().numpy(), last


def evaluate(G, roots, semiring: str = "tropical", weights=None, repeats: int = 3):
    """Measured iteration-kernel time (ms, summed over roots) of each schedule.

    Returns a dict with one entry per fixed variant, 'heuristic', 'learned'
    (if weights are given) and 'best' (the per-iteration minimum over the fixed
    variants' measured times: what a perfect selector could reach).
    """
    if weights is not None:
        slimsell_selector_load(G.h, weights)
    out = {v: 0.0 for v in VARIANTS}
    out.update({"heuristic": 0.0, "best": 0.0})
    if weights is not None:
        out["learned"] = 0.0
    for r in roots:
        per_var = []
        for v in VARIANTS:
            ns = np.median(np.stack([_profiled_run(G, int(r), semiring, v)[0] for _ in range(repeats)]),
                           axis=0)
            per_var.append(ns)
            out[v] += ns.sum() / 1e6
        out["best"] += np.min(np.stack(per_var), axis=0).sum() / 1e6
        for pol in ["heuristic"] + (["learned"] if weights is not None else []):
            out[pol] += np.median([_profiled_run(G, int(r), semiring, pol)[0].sum()
                                   for _ in range(repeats)]) / 1e6
    return out


def device_times(G, roots, semiring: str, policies, reps: int = 15):
    """Whole-run device time (ms, summed over roots) of each policy with the
    device-side loop: CUDA events around every run, the median of `reps` runs
    per root (one warm-up run per policy first)."""
    from . import POLICIES, SEMIRINGS, slimsell_bfs
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for pol in policies:
        slimsell_bfs(G.h, int(roots[0]), SEMIRINGS[semiring], POLICIES[pol], None, None, stream)
        total = 0.0
        for r in roots:
            ts = []
            for _ in range(reps):
                e0.record(stream)
                slimsell_bfs(G.h, int(r), SEMIRINGS[semiring], POLICIES[pol], None, None, stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            total += float(np.median(ts))
        out[pol] = total
    return out
