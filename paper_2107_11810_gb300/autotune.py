"""Autotuner for the solver's runtime settings.

The search's launch shapes are fixed per kernel (warp tiles of 32 records, blocks
of 8 warps), but how much work one expansion step takes (chunk size) and how many
host workers a batched solve uses depend on the family, the problem size and the
GPU.  The autotuner
times a few candidate settings on a representative problem, keeps the fastest,
and caches the choice in a JSON file keyed by (family, d, n bucket, GPU name).
Results never depend on these settings (they are tested bit-identical), only the
time does.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import vote

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gv_gb300_autotune.json")
CANDIDATES = [
    dict(chunk_records=1 << 23),
    dict(chunk_records=1 << 25),
    dict(chunk_records=1 << 26),
    dict(chunk_records=1 << 27),
]


def n_bucket(n: int) -> int:
    """Power-of-4 bucket of the problem size."""
    return 0 if n <= 1 else int(math.log(n, 4))


def cache_key(family: int, d: int, n: int, gpu: str) -> str:
    return f"{family}:{d}:{n_bucket(n)}:{gpu}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(solver: "vote.Solver", setting: dict) -> None:
    solver.set_option(vote.VOTE_OPT_CHUNK_RECORDS, setting["chunk_records"])
    if "batch_workers" in setting:
        solver.set_option(vote.VOTE_OPT_BATCH_WORKERS, setting["batch_workers"])


def tune(solver: "vote.Solver", surfaces, candidates=None, reps: int = 1, timer=None, gpu: str | None = None,
         cache_path: str | None = DEFAULT_CACHE) -> dict:
    """Time each candidate setting on ``surfaces`` (after one warm-up solve), apply
    the fastest to ``solver`` and record it in the cache.  ``timer(solver, surfaces)``
    returns seconds for one solve (default: wall clock around a synchronised
    solve).  Returns {"best": setting, "times": [(setting, seconds), ...]}."""
    candidates = candidates or CANDIDATES
    if timer is None:
        import torch

        def timer(s, x):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.solve(x, want_mask=False)
            torch.cuda.synchronize()
            return time.perf_counter() - t0
    if gpu is None:
        import torch
        gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    times = []
    for c in candidates:
        apply(solver, c)
        timer(solver, surfaces)                                  # warm-up (allocations)
        t = min(timer(solver, surfaces) for _ in range(reps))
        times.append((c, t))
    best = min(times, key=lambda x: x[1])[0]
    apply(solver, best)
    if cache_path:
        cache = load_cache(cache_path)
        cache[cache_key(solver.family, solver.d, surfaces.shape[1], gpu)] = dict(best, seconds=min(t for _, t in times))
        save_cache(cache, cache_path)
    return dict(best=best, times=times)


def apply_cached(solver: "vote.Solver", n: int, gpu: str, cache_path: str = DEFAULT_CACHE) -> bool:
    """Apply a cached setting for this (family, d, n bucket, GPU); False if none."""
    entry = load_cache(cache_path).get(cache_key(solver.family, solver.d, n, gpu))
    if not entry:
        return False
    apply(solver, entry)
    return True
