"""Python binding of libslimsell (GB300 SlimSell BFS), marshalling only.

Every function here is a thin ctypes wrapper of the C entry point with the same
name in ``include/slimsell.h``; all computation runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors) and streams.  There is no
CPU fallback: if ``libslimsell.so`` is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB, build  # noqa: F401  (build() compiles the library)

TROPICAL, REAL, BOOLEAN, SELMAX = 0, 1, 2, 3
SEMIRINGS = {"tropical": TROPICAL, "real": REAL, "boolean": BOOLEAN, "selmax": SELMAX}
V_FULL, V_SLIMWORK, V_PUSH, V_PULL_FILTERED, V_HEURISTIC, V_LEARNED = range(6)
VARIANT_PUSH_LOCAL = 4  # executed-variant id of the cluster push (iteration stats only)
FORMAT_SLIMSELL, FORMAT_SELL = 0, 1  # storage formats of slimsell_bfs_spmv
FORMATS = {"slimsell": FORMAT_SLIMSELL, "sell": FORMAT_SELL}
POLICIES = {"full": V_FULL, "slimwork": V_SLIMWORK, "push": V_PUSH,
            "pull_filtered": V_PULL_FILTERED, "heuristic": V_HEURISTIC, "learned": V_LEARNED}
STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID", 2: "SS_ERR_OOM", 3: "SS_ERR_CUDA",
          4: "SS_ERR_TIMEOUT", 5: "SS_ERR_UNSUPPORTED"}


class SlimSellError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class ss_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("C", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("split_w", ctypes.c_int32), ("n_chunks", ctypes.c_int32),
                ("n_items", ctypes.c_int32), ("n_split_chunks", ctypes.c_int32),
                ("max_degree", ctypes.c_int32), ("nnz", ctypes.c_int64), ("slots", ctypes.c_int64),
                ("padding", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class ss_iter_stats(ctypes.Structure):
    _fields_ = [("frontier", ctypes.c_int64), ("frontier_degree", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("active_chunks", ctypes.c_int64),
                ("variant", ctypes.c_int32), ("kernel_ns", ctypes.c_int32)]


class ss_run_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("semiring", ctypes.c_int32),
                ("reached", ctypes.c_int64), ("reached_degree", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("dp_slots", ctypes.c_int64),
                ("iter_kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class ss_tune_point(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int32), ("sigma", ctypes.c_int32), ("split_w", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class ss_tune_result(ctypes.Structure):
    _fields_ = [("best", ss_tune_point), ("points", ctypes.c_int32), ("cached", ctypes.c_int32)]


class ss_tune_signature(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz_rounded", ctypes.c_int64), ("hist", ctypes.c_int32 * 24)]


_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load libslimsell.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing; run paper_2010_09913_gb300.build.build() first")
    L = ctypes.CDLL(LIB)
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sigs = {
        "slimsell_build": (i32, [_VP, _VP, i32, i64, i32, i32, i32, _VP, ctypes.POINTER(_VP)]),
        "slimsell_bfs": (i32, [_VP, i32, i32, i32, _VP, _VP, _VP]),
        "slimsell_get_values": (i32, [_VP, _VP, _VP]),
        "slimsell_bfs_multi": (i32, [_VP, _VP, i32, i32, _VP, _VP]),
        "slimsell_bfs_multi_parents": (i32, [_VP, _VP, i32, i32, _VP, _VP, _VP]),
        "slimsell_bfs_spmv": (i32, [_VP, i32, i32, i32, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
        "slimsell_bc": (i32, [_VP, _VP, i32, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
        "slimsell_get_info": (i32, [_VP, ctypes.POINTER(ss_info)]),
        "slimsell_get_run_stats": (i32, [_VP, ctypes.POINTER(ss_run_stats),
                                         ctypes.POINTER(ss_iter_stats), i32]),
        "slimsell_set_profiling": (i32, [_VP, i32]),
        "slimsell_set_option": (i32, [_VP, i32, i64]),
        "slimsell_export_layout": (i32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
        "slimsell_destroy": (None, [_VP]),
        "slimsell_sigma_sort_noalloc": (i32, [_VP, i32, i32, _VP, _VP]),
        "slimsell_selector_load": (i32, [_VP, _VP, i64]),
        "slimsell_get_features": (i32, [_VP, _VP, i32]),
        "slimsell_mlp_forward": (i32, [_VP, _VP, i32, _VP, _VP]),
        "slimsell_mlp_train_step": (i32, [_VP, _VP, _VP, i32, _VP, _VP, _VP, i32, ctypes.c_float,
                                          _VP, _VP, _VP]),
        "slimsell_batch_create": (i32, [_VP, i32, i32, i32, ctypes.POINTER(_VP)]),
        "slimsell_batch_run": (i32, [_VP, _VP, _VP, _VP, _VP]),
        "slimsell_batch_get_stats": (i32, [_VP, ctypes.POINTER(ss_run_stats)]),
        "slimsell_batch_destroy": (None, [_VP]),
        "slimsell_autotune": (i32, [_VP, _VP, i32, i64, i32, i32, _VP, i32, _VP, i32, _VP, i32, _VP, i32,
                                    i32, i32, ctypes.POINTER(ss_tune_result), _VP, i32, _VP]),
        "slimsell_tune_signature": (i32, [_VP, i32, ctypes.POINTER(ss_tune_signature)]),
        "slimsell_tune_match": (i32, [ctypes.POINTER(ss_tune_signature), ctypes.POINTER(ss_tune_signature)]),
        "slimsell_last_error": (ctypes.c_char_p, []),
        "slimsell_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    return ["slimsell_build", "slimsell_bfs", "slimsell_bfs_multi", "slimsell_bfs_multi_parents",
            "slimsell_bfs_spmv", "slimsell_bc", "slimsell_get_values",
            "slimsell_get_info", "slimsell_get_run_stats",
            "slimsell_set_profiling", "slimsell_set_option", "slimsell_export_layout",
            "slimsell_destroy",
            "slimsell_sigma_sort_noalloc", "slimsell_selector_load", "slimsell_get_features",
            "slimsell_mlp_forward", "slimsell_mlp_train_step", "slimsell_batch_create",
            "slimsell_batch_run", "slimsell_batch_get_stats", "slimsell_batch_destroy",
            "slimsell_autotune", "slimsell_tune_signature", "slimsell_tune_match",
            "slimsell_last_error", "slimsell_version"]


def _check(fn: str, status: int):
    if status != 0:
        raise SlimSellError(fn, status, lib().slimsell_last_error().decode())


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None, dtype: torch.dtype, name: str):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t.data_ptr()


# ---- C entry points, same names -------------------------------------------------------

def slimsell_build(row_ptr: torch.Tensor, col: torch.Tensor, n: int, nnz: int, C: int, sigma: int,
                   split_w: int, stream=None) -> int:
    h = _VP()
    _check("slimsell_build", lib().slimsell_build(
        _ptr(row_ptr, torch.int64, "row_ptr"), _ptr(col, torch.int32, "col"), int(n), int(nnz),
        int(C), int(sigma), int(split_w), _stream(stream), ctypes.byref(h)))
    return h.value


def slimsell_bfs(h: int, root: int, semiring: int, policy: int, dist: torch.Tensor | None,
                 parent: torch.Tensor | None, stream=None) -> None:
    _check("slimsell_bfs", lib().slimsell_bfs(
        h, int(root), int(semiring), int(policy), _ptr(dist, torch.int32, "dist"),
        _ptr(parent, torch.int32, "parent"), _stream(stream)))


def slimsell_get_values(h: int, out: torch.Tensor, stream=None) -> None:
    _check("slimsell_get_values", lib().slimsell_get_values(h, _ptr(out, torch.float32, "out"),
                                                            _stream(stream)))


def slimsell_bfs_multi(h: int, roots: torch.Tensor, policy: int, dist: torch.Tensor | None,
                       stream=None) -> None:
    _check("slimsell_bfs_multi", lib().slimsell_bfs_multi(
        h, _ptr(roots, torch.int32, "roots"), int(roots.numel()), int(policy),
        _ptr(dist, torch.int32, "dist"), _stream(stream)))


def slimsell_bfs_multi_parents(h: int, roots: torch.Tensor, policy: int, dist: torch.Tensor | None,
                               parent: torch.Tensor | None, stream=None) -> None:
    _check("slimsell_bfs_multi_parents", lib().slimsell_bfs_multi_parents(
        h, _ptr(roots, torch.int32, "roots"), int(roots.numel()), int(policy),
        _ptr(dist, torch.int32, "dist"), _ptr(parent, torch.int32, "parent"), _stream(stream)))


def slimsell_bfs_spmv(h: int, root: int, semiring: int, fmt: int, dist: torch.Tensor,
                      stream=None, timed: bool = False):
    """Value-vector BFS-SpMV in the SlimSell or Sell-C-sigma format; returns the
    summed device time of its kernels in ms when timed, else None."""
    ms = ctypes.c_double(0.0)
    _check("slimsell_bfs_spmv", lib().slimsell_bfs_spmv(
        h, int(root), int(semiring), int(fmt), _ptr(dist, torch.int32, "dist"),
        ctypes.byref(ms) if timed else None, _stream(stream)))
    return ms.value if timed else None


def slimsell_bc(h: int, sources: torch.Tensor, bc: torch.Tensor, stream=None, timed: bool = False):
    """Betweenness centrality over `sources` into `bc` (float64, length n);
    returns the summed device time of its kernels in ms when timed, else None."""
    ms = ctypes.c_double(0.0)
    _check("slimsell_bc", lib().slimsell_bc(
        h, _ptr(sources, torch.int32, "sources"), int(sources.numel()), _ptr(bc, torch.float64, "bc"),
        ctypes.byref(ms) if timed else None, _stream(stream)))
    return ms.value if timed else None


def slimsell_get_info(h: int) -> ss_info:
    out = ss_info()
    _check("slimsell_get_info", lib().slimsell_get_info(h, ctypes.byref(out)))
    return out


def slimsell_get_run_stats(h: int, cap: int = 0):
    out = ss_run_stats()
    arr = (ss_iter_stats * cap)() if cap > 0 else None
    _check("slimsell_get_run_stats", lib().slimsell_get_run_stats(h, ctypes.byref(out), arr, int(cap)))
    return out, arr


def slimsell_set_profiling(h: int, on: bool) -> None:
    _check("slimsell_set_profiling", lib().slimsell_set_profiling(h, 1 if on else 0))


OPT_DP_PASS, OPT_SMEM_BYTES, OPT_DEVICE_LOOP, OPT_SELECTOR_MARGIN, OPT_PROFILE_QUEUE = 1, 2, 3, 4, 5
OPT_PUSH_BLOCKS, OPT_FORMAT = 6, 8


def slimsell_set_option(h: int, option: int, value: int) -> None:
    _check("slimsell_set_option", lib().slimsell_set_option(h, int(option), int(value)))


def slimsell_export_layout(h: int, perm, cl, cs, col, items, stream=None) -> None:
    _check("slimsell_export_layout", lib().slimsell_export_layout(
        h, _ptr(perm, torch.int32, "perm"), _ptr(cl, torch.int32, "cl"), _ptr(cs, torch.int64, "cs"),
        _ptr(col, torch.int32, "col"), _ptr(items, torch.int32, "items"), _stream(stream)))


def slimsell_sigma_sort_noalloc(row_ptr: torch.Tensor, n: int, sigma: int, perm: torch.Tensor,
                                stream=None) -> None:
    """Allocation-free degree sort; see include/slimsell.h for its limits."""
    _check("slimsell_sigma_sort_noalloc", lib().slimsell_sigma_sort_noalloc(
        _ptr(row_ptr, torch.int64, "row_ptr"), int(n), int(sigma), _ptr(perm, torch.int32, "perm"),
        _stream(stream)))


N_FEATURES, N_OUTPUTS, N_PARAMS = 16, 4, 5508


def slimsell_selector_load(h: int, weights) -> None:
    """weights: 5508 float32 values (numpy array or CPU tensor), or None to unload."""
    if weights is None:
        _check("slimsell_selector_load", lib().slimsell_selector_load(h, None, 0))
        return
    import numpy as np
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
    _check("slimsell_selector_load", lib().slimsell_selector_load(
        h, w.ctypes.data_as(ctypes.c_void_p), int(w.size)))


def slimsell_get_features(h: int, cap: int):
    import numpy as np
    out = np.zeros((cap, N_FEATURES), dtype=np.float32)
    _check("slimsell_get_features", lib().slimsell_get_features(
        h, out.ctypes.data_as(ctypes.c_void_p), int(cap)))
    return out


def slimsell_mlp_forward(w: torch.Tensor, x: torch.Tensor, y: torch.Tensor, stream=None) -> None:
    _check("slimsell_mlp_forward", lib().slimsell_mlp_forward(
        _ptr(w, torch.float32, "w"), _ptr(x, torch.float32, "x"), int(x.shape[0]),
        _ptr(y, torch.float32, "y"), _stream(stream)))


def slimsell_mlp_train_step(w, m, v, step, x, t, mask, lr, grad=None, loss=None, stream=None) -> None:
    _check("slimsell_mlp_train_step", lib().slimsell_mlp_train_step(
        _ptr(w, torch.float32, "w"), _ptr(m, torch.float32, "m") if m is not None else None,
        _ptr(v, torch.float32, "v") if v is not None else None, int(step),
        _ptr(x, torch.float32, "x"), _ptr(t, torch.float32, "t"), _ptr(mask, torch.float32, "mask"),
        int(x.shape[0]), float(lr), _ptr(grad, torch.float32, "grad") if grad is not None else None,
        _ptr(loss, torch.float32, "loss") if loss is not None else None, _stream(stream)))


def slimsell_autotune(row_ptr: torch.Tensor, col: torch.Tensor, n: int, nnz: int, semiring: int,
                      policy: int, roots, Cs, sigmas, split_ws, repeats: int = 2, use_cache: bool = True,
                      stream=None):
    """Layout autotuner; returns (ss_tune_result, [ss_tune_point, ...] in grid order)."""
    import numpy as np
    r = np.ascontiguousarray(np.asarray(roots, dtype=np.int32))
    gc = np.ascontiguousarray(np.asarray(Cs, dtype=np.int32))
    gs = np.ascontiguousarray(np.asarray(sigmas, dtype=np.int32))
    gw = np.ascontiguousarray(np.asarray(split_ws, dtype=np.int32))
    total = gc.size * gs.size * gw.size
    table = (ss_tune_point * total)()
    res = ss_tune_result()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check("slimsell_autotune", lib().slimsell_autotune(
        _ptr(row_ptr, torch.int64, "row_ptr"), _ptr(col, torch.int32, "col"), int(n), int(nnz),
        int(semiring), int(policy), p(r), int(r.size), p(gc), int(gc.size), p(gs), int(gs.size),
        p(gw), int(gw.size), int(repeats), 1 if use_cache else 0, ctypes.byref(res), table, total,
        _stream(stream)))
    return res, list(table)


def slimsell_tune_signature(row_ptr) -> ss_tune_signature:
    """Cache key of a graph from host row offsets (numpy int64)."""
    import numpy as np
    rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int64))
    out = ss_tune_signature()
    _check("slimsell_tune_signature", lib().slimsell_tune_signature(
        rp.ctypes.data_as(ctypes.c_void_p), int(rp.size - 1), ctypes.byref(out)))
    return out


def slimsell_tune_match(a: ss_tune_signature, b: ss_tune_signature) -> bool:
    return bool(lib().slimsell_tune_match(ctypes.byref(a), ctypes.byref(b)))


def slimsell_batch_create(handles, semiring: int, policy: int) -> int:
    arr = (_VP * len(handles))(*handles)
    b = _VP()
    _check("slimsell_batch_create", lib().slimsell_batch_create(
        arr, len(handles), int(semiring), int(policy), ctypes.byref(b)))
    return b.value


def slimsell_batch_run(b: int, roots: torch.Tensor, dists=None, parents=None, stream=None) -> None:
    """roots: int32 CUDA tensor [g]; dists / parents: lists of int32 CUDA tensors (or None)."""
    def ptrs(ts):
        if ts is None:
            return None
        return (_VP * len(ts))(*[(_ptr(t, torch.int32, "output") if t is not None else None) for t in ts])
    _check("slimsell_batch_run", lib().slimsell_batch_run(
        b, _ptr(roots, torch.int32, "roots"), ptrs(dists), ptrs(parents), _stream(stream)))


def slimsell_batch_get_stats(b: int, g: int):
    out = (ss_run_stats * g)()
    _check("slimsell_batch_get_stats", lib().slimsell_batch_get_stats(b, out))
    return list(out)


def slimsell_batch_destroy(b: int) -> None:
    if b:
        lib().slimsell_batch_destroy(b)


def slimsell_destroy(h: int) -> None:
    if h:
        lib().slimsell_destroy(h)


def slimsell_last_error() -> str:
    return lib().slimsell_last_error().decode()


def slimsell_version() -> str:
    return lib().slimsell_version().decode()


# ---- convenience wrapper ---------------------------------------------------------------

class SlimSellGraph:
    """Owns one built handle; tensors stay on the caller's device."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, C: int = 32, sigma: int | None = None,
                 split_w: int = 1024, stream=None):
        n = row_ptr.numel() - 1
        self.n = n
        self.h = slimsell_build(row_ptr, col, n, col.numel(), C, n if sigma is None else sigma,
                                split_w, stream)

    @classmethod
    def wrap(cls, h: int, n: int):
        """View an existing handle (not owned: close() leaves it alone)."""
        obj = cls.__new__(cls)
        obj.h, obj.n, obj._owned = h, n, False
        return obj

    @classmethod
    def from_host(cls, row_ptr, col, device="cuda", **kw):
        rp = torch.as_tensor(row_ptr, dtype=torch.int64).to(device)
        c = torch.as_tensor(col, dtype=torch.int32).to(device)
        if c.numel() == 0:
            c = torch.zeros(1, dtype=torch.int32, device=device)[:0]
        return cls(rp, c, **kw)

    def info(self) -> ss_info:
        return slimsell_get_info(self.h)

    def set_option(self, option: int, value: int) -> None:
        slimsell_set_option(self.h, option, value)

    def bfs(self, root: int, semiring="tropical", policy="slimwork", dist=None, parent=None,
            want_parent: bool = True, stream=None):
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
        pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
        dev = torch.device("cuda", torch.cuda.current_device())
        if dist is None:
            dist = torch.empty(self.n, dtype=torch.int32, device=dev)
        if parent is None and want_parent:
            parent = torch.empty(self.n, dtype=torch.int32, device=dev)
        slimsell_bfs(self.h, root, sr, pol, dist, parent, stream)
        return dist, parent

    def values(self, out=None, stream=None):
        """Path counts of the last real-semiring bfs() (float32, original vertex order)."""
        if out is None:
            out = torch.empty(self.n, dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
        slimsell_get_values(self.h, out, stream)
        return out

    def bfs_multi(self, roots, policy="slimwork", dist=None, want_dist: bool = True, stream=None):
        """k-source BFS; returns dist as an (n, k) int32 tensor (vertex-major)."""
        pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
        dev = torch.device("cuda", torch.cuda.current_device())
        r = torch.as_tensor(roots, dtype=torch.int32).to(dev)
        if dist is None and want_dist:
            dist = torch.empty((self.n, r.numel()), dtype=torch.int32, device=dev)
        slimsell_bfs_multi(self.h, r, pol, dist, stream)
        return dist

    def bfs_spmv(self, root: int, semiring="tropical", fmt="slimsell", dist=None, stream=None):
        """Plain value-vector BFS-SpMV in either storage format; returns dist."""
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
        f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        if dist is None:
            dist = torch.empty(self.n, dtype=torch.int32, device=torch.device("cuda", torch.cuda.current_device()))
        slimsell_bfs_spmv(self.h, root, sr, f, dist, stream)
        return dist

    def bc(self, sources, stream=None):
        """Betweenness centrality summed over `sources`; returns a float64 tensor."""
        dev = torch.device("cuda", torch.cuda.current_device())
        src = torch.as_tensor(sources, dtype=torch.int32).to(dev)
        out = torch.empty(self.n, dtype=torch.float64, device=dev)
        slimsell_bc(self.h, src, out, stream)
        return out

    def bfs_multi_parents(self, roots, policy="slimwork", dist=None, parent=None,
                          want_dist: bool = True, stream=None):
        """k-source BFS with largest-id parents; returns (dist, parent), both (n, k)
        int32 tensors (vertex-major; dist None when want_dist is False)."""
        pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
        dev = torch.device("cuda", torch.cuda.current_device())
        r = torch.as_tensor(roots, dtype=torch.int32).to(dev)
        if dist is None and want_dist:
            dist = torch.empty((self.n, r.numel()), dtype=torch.int32, device=dev)
        if parent is None:
            parent = torch.empty((self.n, r.numel()), dtype=torch.int32, device=dev)
        slimsell_bfs_multi_parents(self.h, r, pol, dist, parent, stream)
        return dist, parent

    def run_stats(self, cap: int = 0):
        return slimsell_get_run_stats(self.h, cap)

    def export_layout(self):
        inf = self.info()
        dev = torch.device("cuda", torch.cuda.current_device())
        perm = torch.empty(inf.n_chunks * inf.C, dtype=torch.int32, device=dev)
        cl = torch.empty(inf.n_chunks, dtype=torch.int32, device=dev)
        cs = torch.empty(inf.n_chunks + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(inf.slots, 1), dtype=torch.int32, device=dev)
        items = torch.empty(max(inf.n_items, 1) * 4, dtype=torch.int32, device=dev)
        slimsell_export_layout(self.h, perm, cl, cs, col, items)
        return {"perm": perm, "cl": cl, "cs": cs, "col": col[: inf.slots],
                "items": items[: inf.n_items * 4].view(-1, 4)}

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            slimsell_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
