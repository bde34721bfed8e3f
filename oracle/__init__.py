"""Oracle for approximate max-depth general voting (arXiv 2107.11810, Algorithm 2).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  The product path
(``paper_2107_11810_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``gv_oracle.c`` (plain recursive FP64 C, one IEEE
operation at a time, compiled with ``-ffp-contract=off``); this module compiles it
with gcc on first use and exposes it through ctypes.

Functions and the passages they follow:
  * :func:`solve` -- SurfaceConsensus (Algorithm 2) with canonization
    (Sec. 3.2, "Canonization") and bound-based pruning (Sec. 3.3, B&B combined
    with canonization); returns the best leaf, its depth and the inlier mask.
  * :func:`solve_parallel` -- the same search on several host threads (the
    multi-core CPU baseline); identical results.
  * :func:`cell_counts` -- upper/lower bound of one cell by replaying every
    original surface from the root (merge tracking, Sec. 3.2).
  * :func:`levels` -- level structure, snap steps and accumulated canonization
    error (Sec. 3.2, "Canonization" and the eps-update discussion).
  * :func:`vsin` / :func:`vcos` -- the sine/cosine used for cell-centre basis
    values (Taylor series with Cody-Waite reduction).
  * :func:`oracle.naive.naive_voting` -- naive voting (Algorithm 1) on the leaf
    grid, every family (the comparator's definition).
  * :func:`sigma`, :func:`lipschitz`, :func:`path_records` -- the margin functions
    behind the canonization error bound and the surface-box test (Sec. 3.2), and
    the canonical records of one surface along a root-to-cell path, exported so
    that tests can check them against the surface equations.

Pins (tests/test_oracle_*.py): brute-force depth on dense grids, the exact
arrangement maximum for lines, planted inliers, the approximation guarantee,
pruning/order/grouping invariance, special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgvoracle.so")
_lock = threading.Lock()
_lib = None

LINE2D, PLANE3D_SPH, POSE3DOF, POSE6DOF, RAYS3D, POINTSET2D, AFFINE4D, RADIAL5DOF, POSE7DOF = range(1, 10)
NO_MERGE, NO_PRUNE, REVERSE = 1, 2, 4
FAMILY_SHAPE = {LINE2D: (2, 1, 1, 2), PLANE3D_SPH: (3, 2, 3, 3), POSE3DOF: (3, 1, 2, 4), POSE6DOF: (6, 4, 11, 5),
                RAYS3D: (3, 1, 2, 4), POINTSET2D: (4, 2, 2, 4), AFFINE4D: (4, 3, 3, 4), RADIAL5DOF: (5, 4, 7, 5),
                POSE7DOF: (7, 5, 11, 5)}
"""family -> (d, k, number of essential params, number of input params)"""

_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile gv_oracle.c into oracle/_build/libgvoracle.so (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _declare(lib):
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int
    lib.gvo_vsin.restype = ctypes.c_double
    lib.gvo_vsin.argtypes = [ctypes.c_double]
    lib.gvo_vcos.restype = ctypes.c_double
    lib.gvo_vcos.argtypes = [ctypes.c_double]
    lib.gvo_levels.restype = i32
    lib.gvo_levels.argtypes = [i32, i32, i32, P, P, P, P, P, P, P]
    lib.gvo_root_records.restype = i32
    lib.gvo_root_records.argtypes = [i32, i32, i32, P, P, P, i64, P, P]
    lib.gvo_solve.restype = i32
    lib.gvo_solve.argtypes = [i32, i32, i32, P, P, P, i64, i32, P, P, P, P, P, i64, P, P, P, P, P, P]
    lib.gvo_cell_counts.restype = i32
    lib.gvo_cell_counts.argtypes = [i32, i32, i32, P, P, P, i64, i32, P, P, P, P]
    lib.gvo_solve_parallel.restype = i32
    lib.gvo_solve_parallel.argtypes = [i32, i32, i32, P, P, P, i64, i32, P, P, P, P, P]
    lib.gvo_sigma.restype = i32
    lib.gvo_sigma.argtypes = [i32, i32, i32, P, P, P]
    lib.gvo_lipschitz.restype = i32
    lib.gvo_lipschitz.argtypes = [i32, i32, i32, P, P, P]
    lib.gvo_path_records.restype = i32
    lib.gvo_path_records.argtypes = [i32, i32, i32, P, P, P, i64, i64, i32, P, P, P]
    lib.gvo_rotation.restype = None
    lib.gvo_rotation.argtypes = [P, P]
    return lib


def load_variant(source: str, tag: str):
    """Compile a modified copy of the oracle source (used by the mutation tests to
    check that the pins catch planted mistakes) and return the loaded library."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"variant_{tag}.c")
    lib = os.path.join(_BUILD, f"libgvoracle_{tag}.so")
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", *_CFLAGS, "-o", lib, src, "-lm"], check=True)
    return _declare(ctypes.CDLL(lib))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(family, eps, bounds, params):
    d, k, le, npar = FAMILY_SHAPE[family]
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(d)
    bounds = np.ascontiguousarray(bounds, dtype=np.float64).reshape(2 * d)
    params = np.ascontiguousarray(params, dtype=np.float64)
    if params.ndim != 2 or params.shape[0] != npar:
        raise ValueError(f"params must be SoA [{npar}, n]")
    return d, k, le, eps, bounds, params


def vsin(x: float) -> float:
    return _load().gvo_vsin(float(x))


def vcos(x: float) -> float:
    return _load().gvo_vcos(float(x))


def rotation(ph, lib=None) -> np.ndarray:
    """The 3x3 rotation matrix of axis-angle vector ph that the POSE6DOF family's
    basis uses (Rodrigues' formula by power series in |ph|^2)."""
    ph = np.ascontiguousarray(ph, dtype=np.float64).reshape(3)
    out = np.zeros(9)
    (lib or _load()).gvo_rotation(_ptr(ph), _ptr(out))
    return out.reshape(3, 3)


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def levels(family, eps, bounds, lib=None):
    """Level structure: dict with L, Lj[d], h[L+1, d], s_f[d-k], s_t[L, le], A[L+1, d-k]."""
    d, k, le, _ = FAMILY_SHAPE[family]
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    bounds = np.ascontiguousarray(bounds, dtype=np.float64)
    Lj = np.zeros(d, np.int32)
    lib = lib or _load()
    L = lib.gvo_levels(family, d, k, _ptr(eps), _ptr(bounds), _ptr(Lj), None, None, None, None)
    if L < 0:
        raise ValueError("invalid problem")
    h = np.zeros((L + 1, d))
    s_f = np.zeros(d - k)
    s_t = np.zeros((max(L, 1), le))
    A = np.zeros((L + 1, d - k))
    lib.gvo_levels(family, d, k, _ptr(eps), _ptr(bounds), _ptr(Lj), _ptr(h), _ptr(s_f), _ptr(s_t), _ptr(A))
    return dict(L=L, Lj=Lj, h=h, s_f=s_f, s_t=s_t[:L], A=A)


def root_records(family, eps, bounds, params):
    d, k, le, eps, bounds, params = _prep(family, eps, bounds, params)
    n = params.shape[1]
    f = np.zeros((d - k, n))
    t = np.zeros((le, n))
    if _load().gvo_root_records(family, d, k, _ptr(eps), _ptr(bounds), _ptr(params), n, _ptr(f), _ptr(t)):
        raise ValueError("invalid problem")
    return f, t


def solve(family, eps, bounds, params, flags=0, trace_cap=0, members=False, lib=None):
    """Run SurfaceConsensus.  Returns a dict with best_point[d], best_leaf[d],
    depth, mask (uint32 words), stats (tests, cells, leaves, L), and optionally
    the trace (level, coords, ub, lb of every tested child) and the best leaf's
    members (only with NO_MERGE)."""
    d, k, le, eps, bounds, params = _prep(family, eps, bounds, params)
    n = params.shape[1]
    best_point = np.zeros(d)
    best_leaf = np.zeros(d, np.int64)
    depth = np.zeros(1, np.int64)
    mask = np.zeros(max((n + 31) // 32, 1), np.uint32)
    stats = np.zeros(4, np.int64)
    tl = np.zeros(max(trace_cap, 1), np.int32)
    tc = np.zeros((max(trace_cap, 1), d), np.int64)
    tu = np.zeros(max(trace_cap, 1), np.int64)
    tb = np.zeros(max(trace_cap, 1), np.int64)
    tn = np.zeros(1, np.int64)
    mem = np.full(max(n, 1), -1, np.int64) if members else None
    rc = (lib or _load()).gvo_solve(family, d, k, _ptr(eps), _ptr(bounds), _ptr(params), n, flags,
                           _ptr(best_point), _ptr(best_leaf), _ptr(depth), _ptr(mask), _ptr(stats),
                           trace_cap, _ptr(tl), _ptr(tc), _ptr(tu), _ptr(tb), _ptr(tn), _ptr(mem))
    if rc:
        raise ValueError("invalid problem")
    out = dict(best_point=best_point, best_leaf=best_leaf, depth=int(depth[0]),
               mask=mask[: (n + 31) // 32], stats=stats)
    if trace_cap:
        m = int(tn[0])
        out["trace"] = dict(level=tl[:m].copy(), coords=tc[:m].copy(), ub=tu[:m].copy(), lb=tb[:m].copy())
    if members:
        out["members"] = np.sort(mem[: int(depth[0])])
    return out


def solve_parallel(family, eps, bounds, params, threads=None, lib=None):
    """The same search on several host threads (OpenMP over the subtrees below a
    split level, sharing the best bound between subtrees); depth, best leaf and
    mask equal :func:`solve`'s.  stats: tests, cells, leaves, L, threads, tasks."""
    d, k, le, eps, bounds, params = _prep(family, eps, bounds, params)
    n = params.shape[1]
    threads = threads or os.cpu_count() or 1
    best_point = np.zeros(d)
    best_leaf = np.zeros(d, np.int64)
    depth = np.zeros(1, np.int64)
    mask = np.zeros(max((n + 31) // 32, 1), np.uint32)
    stats = np.zeros(6, np.int64)
    if (lib or _load()).gvo_solve_parallel(family, d, k, _ptr(eps), _ptr(bounds), _ptr(params), n, int(threads),
                                            _ptr(best_point), _ptr(best_leaf), _ptr(depth), _ptr(mask),
                                            _ptr(stats)):
        raise ValueError("invalid problem")
    return dict(best_point=best_point, best_leaf=best_leaf, depth=int(depth[0]), mask=mask[: (n + 31) // 32],
                stats=stats)


def cell_counts(family, eps, bounds, params, level, coords, want_reach=False):
    """(UB, LB[, reach mask]) of one cell by replay of every original surface."""
    d, k, le, eps, bounds, params = _prep(family, eps, bounds, params)
    n = params.shape[1]
    coords = np.ascontiguousarray(coords, dtype=np.int64).reshape(d)
    ub = np.zeros(1, np.int64)
    lb = np.zeros(1, np.int64)
    reach = np.zeros(max((n + 31) // 32, 1), np.uint32) if want_reach else None
    if _load().gvo_cell_counts(family, d, k, _ptr(eps), _ptr(bounds), _ptr(params), n, int(level),
                               _ptr(coords), _ptr(ub), _ptr(lb), _ptr(reach)):
        raise ValueError("invalid cell")
    if want_reach:
        return int(ub[0]), int(lb[0]), reach[: (n + 31) // 32]
    return int(ub[0]), int(lb[0])


def mask_to_indices(mask: np.ndarray, n: int) -> np.ndarray:
    bits = np.unpackbits(mask.view(np.uint8), bitorder="little")[:n]
    return np.nonzero(bits)[0]


def _bounds_arg(bounds, d):
    return None if bounds is None else np.ascontiguousarray(bounds, dtype=np.float64).reshape(2 * d)


def sigma(family, h, bounds=None, lib=None):
    """sigma_m: the oracle's bound on the change of basis function m across a cell
    of half-widths h[d] (it sets the essential-parameter snap steps and the
    canonization error bound, Sec. 3.2).  ``bounds`` (the domain, lo/hi per
    coordinate) is needed where the bound depends on it (7DoF)."""
    d, k, le, _ = FAMILY_SHAPE[family]
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(d)
    out = np.zeros(le)
    if (lib or _load()).gvo_sigma(family, d, k, _ptr(_bounds_arg(bounds, d)), _ptr(h), _ptr(out)):
        raise ValueError("invalid family or domain")
    return out


def lipschitz(family, t, bounds=None, lib=None):
    """Lambda[j, i]: the oracle's bound on |dF_j/dx_i| for essential parameters t
    (the free-coordinate term of the surface-box test, Sec. 3.2); ``bounds`` as for
    :func:`sigma`."""
    d, k, le, _ = FAMILY_SHAPE[family]
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(le)
    out = np.zeros((d - k) * k)
    if (lib or _load()).gvo_lipschitz(family, d, k, _ptr(_bounds_arg(bounds, d)), _ptr(t), _ptr(out)):
        raise ValueError("invalid family or domain")
    return out.reshape(d - k, k)


def path_records(family, eps, bounds, params, i, level, coords, lib=None):
    """Canonical record (f[d-k], t[le]) of original surface i after the snap at each
    level of the path from the root to cell (level, coords), as long as the record
    reaches that level's cell.  Returns (f[m, d-k], t[m, le]), m <= level."""
    d, k, le, eps, bounds, params = _prep(family, eps, bounds, params)
    n = params.shape[1]
    coords = np.ascontiguousarray(coords, dtype=np.int64).reshape(d)
    f = np.zeros((max(level, 1), d - k))
    t = np.zeros((max(level, 1), le))
    m = (lib or _load()).gvo_path_records(family, d, k, _ptr(eps), _ptr(bounds), _ptr(params), n, int(i),
                                           int(level), _ptr(coords), _ptr(f), _ptr(t))
    if m < 0:
        raise ValueError("invalid input")
    return f[:m], t[:m]
