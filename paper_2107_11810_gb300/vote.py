"""Python binding of libvote.so (argument marshalling only).

Every step of the search runs in the CUDA library; this module converts torch
tensors and numpy arrays to pointers and sizes and raises on error codes.  There
is no CPU fallback: if the library is missing, :func:`load` raises.

Names follow the C ABI in ``include/vote.h``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .inputs import LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, FAMILY_DK

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvote.so")
_lock = threading.Lock()
_lib = None

VOTE_OPT_PRECISION, VOTE_OPT_PRUNE, VOTE_OPT_CHUNK_RECORDS = 1, 2, 3
VOTE_OPT_TRACE_CAP, VOTE_OPT_GROUP, VOTE_OPT_FAULT_ALLOC_AT = 4, 5, 6
VOTE_OPT_INITIAL_LB, VOTE_OPT_KERNEL_TIMING, VOTE_OPT_BATCH_WORKERS = 7, 8, 10
VOTE_OPT_DIVE, VOTE_OPT_SPIN_LIMIT = 11, 12
KERNEL_CLASSES = ["lift", "cell_geo", "test_count", "test_emit", "children", "replay", "group", "spare"]
STATUS = {0: "VOTE_OK", 1: "VOTE_EINVAL", 2: "VOTE_ENOMEM", 3: "VOTE_ECUDA", 4: "VOTE_ECAPACITY",
          5: "VOTE_ETIMEOUT", 6: "VOTE_EUNSUPPORTED", 7: "VOTE_EINTERNAL"}
NPARAM = {LINE2D: 2, PLANE3D_SPH: 3, POSE3DOF: 4, POSE6DOF: 5, RAYS3D: 4, POINTSET2D: 4, AFFINE4D: 4, RADIAL5DOF: 5}
# essential parameters (record coefficients) per family
NESSENTIAL = {LINE2D: 1, PLANE3D_SPH: 3, POSE3DOF: 2, POSE6DOF: 11, RAYS3D: 2, POINTSET2D: 2, AFFINE4D: 3,
              RADIAL5DOF: 7}
EXPORTS = ["vote_create", "vote_set_option", "vote_set_stream", "vote_solve", "vote_solve_host",
           "vote_cell_counts", "vote_levels", "vote_get_trace", "vote_get_stats", "vote_get_kernel_times",
           "vote_get_level_stats", "vote_cell_counts_noalloc", "vote_softscore_fwd", "vote_softscore_bwd",
           "vote_refine", "vote_solve_batched", "vote_leaf_box", "vote_level_constants",
           "vote_last_error", "vote_destroy"]


class VoteError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("cells", ctypes.c_int64), ("records", ctypes.c_int64),
                ("tests", ctypes.c_int64), ("rechecks", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("leaves", ctypes.c_int64), ("peak_records", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def load(path: str | None = None):
    """Load libvote.so (build it first with ``paper_2107_11810_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libvote.so not found at {p}; run paper_2107_11810_gb300.build.build()")
            lib = ctypes.CDLL(p)
            P, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.vote_create.argtypes = [i32, i32, i32, P, P, ctypes.POINTER(ctypes.c_void_p)]
            lib.vote_set_option.argtypes = [P, i32, d]
            lib.vote_set_stream.argtypes = [P, P]
            lib.vote_solve.argtypes = [P, P, i64, P, P, P, P]
            lib.vote_solve_host.argtypes = [P, P, i64, P, P, P, P]
            lib.vote_cell_counts.argtypes = [P, P, i64, i32, P, P, P, P]
            lib.vote_levels.argtypes = [P, P, P]
            lib.vote_leaf_box.argtypes = [P, P, P, P]
            lib.vote_level_constants.argtypes = [i32, i32, i32, P, P, P, P, P, P, P]
            lib.vote_get_trace.argtypes = [P, i64, P, P, P, P, P]
            lib.vote_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
            lib.vote_get_kernel_times.argtypes = [P, P, P, P]
            lib.vote_get_level_stats.argtypes = [P, P, P, P, P]
            lib.vote_cell_counts_noalloc.argtypes = [i32, i32, i32, P, P, P, i64, i32, P, P, P, P, P]
            lib.vote_softscore_fwd.argtypes = [P, P, i64, P, P, P, P]
            lib.vote_softscore_bwd.argtypes = [P, P, i64, P, P, P, P, P, P]
            lib.vote_refine.argtypes = [P, P, i64, P, P, P, P, i32, P, P]
            lib.vote_solve_batched.argtypes = [P, P, P, i32, P, P, P, P, P]
            lib.vote_last_error.restype = ctypes.c_char_p
            lib.vote_last_error.argtypes = []
            lib.vote_destroy.argtypes = [P]
            lib.vote_destroy.restype = None
            for name in EXPORTS:
                if name not in ("vote_last_error", "vote_destroy"):
                    getattr(lib, name).restype = i32
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        raise VoteError(rc, load().vote_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def check_surfaces(surfaces, nparam: int):
    """A device surface array must be a contiguous CUDA float64 tensor [nparam, n]:
    anything else would hand the library a pointer it reads out of bounds or in
    the wrong format."""
    import torch
    if not isinstance(surfaces, torch.Tensor):
        raise ValueError("surfaces must be a torch tensor on a CUDA device")
    if surfaces.ndim != 2 or surfaces.shape[0] != nparam:
        raise ValueError(f"surfaces must be [{nparam}, n], got {tuple(surfaces.shape)}")
    if not (surfaces.is_cuda and surfaces.dtype == torch.float64 and surfaces.is_contiguous()):
        raise ValueError("surfaces must be a contiguous CUDA float64 tensor")


def check_words(buf, n: int, device, name: str):
    """A device bit-mask buffer: CUDA int32 tensor with at least (n + 31) // 32 words,
    contiguous, on the surfaces' device."""
    import torch
    if buf is None:
        return
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or buf.dtype != torch.int32 or not buf.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA int32 tensor")
    if buf.numel() < (n + 31) // 32:
        raise ValueError(f"{name} needs at least {(n + 31) // 32} words, has {buf.numel()}")
    if buf.device != device:
        raise ValueError(f"{name} must be on {device}, is on {buf.device}")


class Solver:
    """One voting problem shape: family, per-coordinate eps, domain bounds.

    ``solve(surfaces)`` takes a CUDA float64 tensor [P, n] (structure of arrays)
    and returns the best leaf centre, its integer coordinates, the depth and the
    inlier mask (CUDA int32 tensor holding the uint32 words)."""

    def __init__(self, family: int, eps, bounds, precision: int = 1, prune: bool = True,
                 chunk_records: int | None = None, trace_cap: int = 0, stream=None):
        self.lib = load()
        self.family = family
        self.d, self.k = FAMILY_DK[family]
        self.np = NPARAM[family]
        e = np.ascontiguousarray(eps, dtype=np.float64).reshape(self.d)
        b = np.ascontiguousarray(bounds, dtype=np.float64).reshape(2 * self.d)
        h = ctypes.c_void_p()
        _check(self.lib.vote_create(family, self.d, self.k, _ptr(e), _ptr(b), ctypes.byref(h)))
        self.eps, self.bounds = e, b
        self.h = h
        self.set_option(VOTE_OPT_PRECISION, precision)
        self.set_option(VOTE_OPT_PRUNE, 1 if prune else 0)
        if chunk_records:
            self.set_option(VOTE_OPT_CHUNK_RECORDS, chunk_records)
        if trace_cap:
            self.set_option(VOTE_OPT_TRACE_CAP, trace_cap)
        if stream is not None:
            self.set_stream(stream)

    def set_option(self, key: int, value: float):
        _check(self.lib.vote_set_option(self.h, key, float(value)))

    def set_stream(self, stream):
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self.lib.vote_set_stream(self.h, ctypes.c_void_p(handle)))

    def levels(self):
        L = ctypes.c_int()
        Lj = np.zeros(self.d, np.int32)
        _check(self.lib.vote_levels(self.h, ctypes.byref(L), _ptr(Lj)))
        return L.value, Lj

    def _check_surfaces(self, surfaces):
        check_surfaces(surfaces, self.np)

    def solve(self, surfaces, want_mask: bool = True):
        import torch
        self._check_surfaces(surfaces)
        n = surfaces.shape[1]
        bp = np.zeros(self.d)
        bl = np.zeros(self.d, np.int64)
        dep = np.zeros(1, np.int64)
        mask = torch.zeros(max((n + 31) // 32, 1), dtype=torch.int32, device=surfaces.device) if want_mask else None
        _check(self.lib.vote_solve(self.h, _ptr(surfaces), n, _ptr(bp), _ptr(bl), _ptr(dep), _ptr(mask)))
        out = dict(best_point=bp, best_leaf=bl, depth=int(dep[0]))
        if want_mask:
            out["mask"] = mask[: (n + 31) // 32]
        return out

    def solve_host(self, surfaces, want_mask: bool = True):
        """Host buffers in and out (copies inside the call)."""
        if hasattr(surfaces, "data_ptr"):
            import torch
            if surfaces.is_cuda or not surfaces.is_contiguous() or surfaces.dtype != torch.float64:
                raise ValueError("surfaces must be a contiguous CPU float64 tensor")
        else:
            surfaces = np.ascontiguousarray(surfaces, dtype=np.float64)
        if surfaces.ndim != 2 or surfaces.shape[0] != self.np:
            raise ValueError(f"surfaces must be [{self.np}, n]")
        n = surfaces.shape[1]
        bp = np.zeros(self.d)
        bl = np.zeros(self.d, np.int64)
        dep = np.zeros(1, np.int64)
        mask = np.zeros(max((n + 31) // 32, 1), np.uint32) if want_mask else None
        _check(self.lib.vote_solve_host(self.h, _ptr(surfaces), n, _ptr(bp), _ptr(bl), _ptr(dep), _ptr(mask)))
        out = dict(best_point=bp, best_leaf=bl, depth=int(dep[0]))
        if want_mask:
            out["mask"] = mask[: (n + 31) // 32]
        return out

    def cell_counts(self, surfaces, level: int, coords, want_reach: bool = False):
        import torch
        self._check_surfaces(surfaces)
        n = surfaces.shape[1]
        c = np.ascontiguousarray(coords, dtype=np.int64).reshape(self.d)
        ub = np.zeros(1, np.int64)
        lb = np.zeros(1, np.int64)
        reach = torch.zeros(max((n + 31) // 32, 1), dtype=torch.int32, device=surfaces.device) if want_reach else None
        check_words(reach, n, surfaces.device, "reach")
        _check(self.lib.vote_cell_counts(self.h, _ptr(surfaces), n, int(level), _ptr(c), _ptr(ub), _ptr(lb),
                                         _ptr(reach)))
        if want_reach:
            return int(ub[0]), int(lb[0]), reach[: (n + 31) // 32]
        return int(ub[0]), int(lb[0])

    def trace(self, cap: int):
        lv = np.zeros(max(cap, 1), np.int32)
        co = np.zeros((max(cap, 1), self.d), np.int64)
        ub = np.zeros(max(cap, 1), np.int64)
        lb = np.zeros(max(cap, 1), np.int64)
        cnt = np.zeros(1, np.int64)
        _check(self.lib.vote_get_trace(self.h, cap, _ptr(lv), _ptr(co), _ptr(ub), _ptr(lb), _ptr(cnt)))
        m = int(cnt[0])
        return dict(level=lv[:m], coords=co[:m], ub=ub[:m], lb=lb[:m])

    def kernel_times(self) -> dict:
        """{class: (ms, launches, algorithmic bytes)} of the last solve (needs
        VOTE_OPT_KERNEL_TIMING = 1)."""
        ms = np.zeros(8)
        nl = np.zeros(8, np.int64)
        by = np.zeros(8)
        _check(self.lib.vote_get_kernel_times(self.h, _ptr(ms), _ptr(nl), _ptr(by)))
        return {k: (float(ms[i]), int(nl[i]), float(by[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def level_stats(self) -> dict:
        """Per level of the last solve: cells expanded, record slots tested, and with
        grouping on the records entering the grouping and the canonical records
        leaving it (merge fraction = 1 - grouped_out / grouped_in)."""
        L, _ = self.levels()
        a = {k: np.zeros(max(L, 1), np.int64) for k in ("cells", "records", "grouped_in", "grouped_out")}
        _check(self.lib.vote_get_level_stats(self.h, _ptr(a["cells"]), _ptr(a["records"]), _ptr(a["grouped_in"]),
                                             _ptr(a["grouped_out"])))
        return {k: v[:L] for k, v in a.items()}

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib.vote_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def solve_batched(self, blocks, want_mask: bool = True):
        """Solve independent problems.  ``blocks``: CUDA float64 tensor holding the
        problems' [P, n_b] blocks back to back (see pack_batch) and ``offsets``.
        Returns dict of best_points [B, d], best_leaves, depths [B], masks (CUDA
        int32 words, problem b at word_offsets[b]), latency_ms [B]."""
        import torch
        data, offsets = blocks
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        B = len(offs) - 1
        if not (isinstance(data, torch.Tensor) and data.is_cuda and data.dtype == torch.float64
                and data.is_contiguous() and data.numel() >= self.np * int(offs[-1])):
            raise ValueError(f"batched surfaces must be a contiguous CUDA float64 tensor of at least "
                             f"{self.np} x {int(offs[-1])} values")
        ns = np.diff(offs)
        wo = np.concatenate([[0], np.cumsum((ns + 31) // 32)]).astype(np.int64)
        bp = np.zeros((max(B, 1), self.d))
        bl = np.zeros((max(B, 1), self.d), np.int64)
        dep = np.zeros(max(B, 1), np.int64)
        lat = np.zeros(max(B, 1))
        masks = torch.zeros(max(int(wo[-1]), 1), dtype=torch.int32, device=data.device) if want_mask else None
        _check(self.lib.vote_solve_batched(self.h, _ptr(data), _ptr(offs), B, _ptr(bp), _ptr(bl), _ptr(dep),
                                           _ptr(masks), _ptr(lat)))
        return dict(best_points=bp[:B], best_leaves=bl[:B], depths=dep[:B], masks=masks, word_offsets=wo,
                    latency_ms=lat[:B])

    def refine(self, surfaces, mask, cell_lo, cell_hi, point, tol=None, iters: int = 50):
        """Projected gradient ascent of the soft inlier score inside a cell; returns
        (point, score)."""
        self._check_surfaces(surfaces)
        n = surfaces.shape[1]
        check_words(mask, n, surfaces.device, "mask")
        lo = np.ascontiguousarray(cell_lo, dtype=np.float64).reshape(self.d)
        hi = np.ascontiguousarray(cell_hi, dtype=np.float64).reshape(self.d)
        pt = np.array(point, dtype=np.float64).reshape(self.d)
        tl = None if tol is None else np.ascontiguousarray(tol, dtype=np.float64).reshape(self.d - self.k)
        sc = np.zeros(1)
        _check(self.lib.vote_refine(self.h, _ptr(surfaces), n, _ptr(mask), _ptr(lo), _ptr(hi), _ptr(tl), int(iters),
                                    _ptr(pt), _ptr(sc)))
        return pt, float(sc[0])

    def leaf_box(self, leaf):
        """(lo, hi) of a leaf cell given its integer coordinates (vote_leaf_box)."""
        lf = np.ascontiguousarray(leaf, dtype=np.int64).reshape(self.d)
        lo = np.zeros(self.d)
        hi = np.zeros(self.d)
        _check(self.lib.vote_leaf_box(self.h, _ptr(lf), _ptr(lo), _ptr(hi)))
        return lo, hi

    def close(self):
        if getattr(self, "h", None):
            self.lib.vote_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_batch(param_list):
    """Concatenate [P, n_b] float64 arrays into the batched layout: a flat array with
    problem b's [P, n_b] block at element P * offsets[b]; returns (flat, offsets)."""
    offs = np.concatenate([[0], np.cumsum([p.shape[1] for p in param_list])]).astype(np.int64)
    flat = np.concatenate([np.ascontiguousarray(p, dtype=np.float64).ravel() for p in param_list]) \
        if param_list else np.zeros(0)
    return flat, offs


def cell_counts_noalloc(family: int, eps, bounds, surfaces, level: int, coords, reach=None, stream=None):
    """UB and LB of one cell through the entry point that allocates no device memory
    (its scratch is a fixed array inside the library).  ``surfaces``: CUDA float64
    [P, n]; ``reach``: optional CUDA int32 tensor of (n+31)//32 words to receive the
    reach mask.  Calls that may overlap on the GPU must be serialised by the caller."""
    lib = load()
    d, k = FAMILY_DK[family]
    check_surfaces(surfaces, NPARAM[family])
    check_words(reach, surfaces.shape[1], surfaces.device, "reach")
    e = np.ascontiguousarray(eps, dtype=np.float64).reshape(d)
    b = np.ascontiguousarray(bounds, dtype=np.float64).reshape(2 * d)
    c = np.ascontiguousarray(coords, dtype=np.int64).reshape(d)
    ub = np.zeros(1, np.int64)
    lb = np.zeros(1, np.int64)
    handle = None
    if stream is not None:
        handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.vote_cell_counts_noalloc(family, d, k, _ptr(e), _ptr(b), _ptr(surfaces), surfaces.shape[1],
                                        int(level), _ptr(c), _ptr(ub), _ptr(lb), _ptr(reach), handle))
    return int(ub[0]), int(lb[0])


def level_constants(family: int, eps, bounds) -> dict:
    """The level structure without a context or a device (vote_level_constants): L,
    Lj [d], s_f [d-k], s_t [L, le] (essential-parameter snap steps per level) and
    A [L, d-k] (accumulated canonization error bound after each level's snap)."""
    lib = load()
    d, k = FAMILY_DK[family]
    le = NESSENTIAL[family]
    e = np.ascontiguousarray(eps, dtype=np.float64).reshape(d)
    b = np.ascontiguousarray(bounds, dtype=np.float64).reshape(2 * d)
    L = ctypes.c_int()
    Lj = np.zeros(d, np.int32)
    s_f = np.zeros(d - k)
    s_t = np.zeros(31 * le)
    A = np.zeros(31 * (d - k))
    _check(lib.vote_level_constants(family, d, k, _ptr(e), _ptr(b), ctypes.byref(L), _ptr(Lj), _ptr(s_f),
                                    _ptr(s_t), _ptr(A)))
    n = L.value
    return dict(L=n, Lj=Lj, s_f=s_f, s_t=s_t[: n * le].reshape(n, le), A=A[: n * (d - k)].reshape(n, d - k))


def mask_words_to_numpy(mask) -> np.ndarray:
    """CUDA int32 tensor of mask words -> numpy uint32."""
    if hasattr(mask, "cpu"):
        mask = mask.cpu().numpy()
    return np.asarray(mask).view(np.uint32)
