"""Launch-shape autotuner for the formal-solution march.

The march's work per voxel is split into 8 fixed direction slots; the one
free launch parameter is how many thread blocks share the slots of a voxel
tile ("direction groups", 1, 2, 4 or 8).  More groups give more, shorter
blocks (better balance of the depth-dependent characteristic lengths and
of the transmission cutoff), fewer groups give fewer blocks that re-read
less.  J does not depend on the choice (fixed summation order), so the
tuner only times it: each candidate runs a few formal solutions with CUDA
events on the launching stream (the library's profiling counters), and the
fastest mean wins.  Results are cached in a JSON file keyed by grid shape,
direction count, precision and SM count.
"""

from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Tuple

CANDIDATES = (1, 2, 4, 8)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rt3d_autotune.json")


def cache_key(nx: int, ny: int, nz: int, ndir: int, precision: int, sms: int) -> str:
    return f"{nx}x{ny}x{nz}:d{ndir}:p{precision}:sm{sms}"


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: Dict[str, dict]) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings: Dict[int, float]) -> int:
    """Fastest candidate; ties go to fewer groups (fewer blocks)."""
    return min(timings, key=lambda g: (timings[g], g))


def tune(key: str, time_candidate: Callable[[int], float],
         candidates: Iterable[int] = CANDIDATES, cache_path: Optional[str] = DEFAULT_CACHE,
         refresh: bool = False) -> Tuple[int, Dict[int, float]]:
    """Return (best groups, {groups: ms}) for `key`, from the cache unless
    `refresh`; `time_candidate(g)` returns the mean ms of the march with g
    groups."""
    cache = load_cache(cache_path) if cache_path else {}
    if not refresh and key in cache and "groups" in cache[key]:
        return int(cache[key]["groups"]), {int(k): v for k, v in cache[key].get("ms", {}).items()}
    timings = {int(g): float(time_candidate(int(g))) for g in candidates}
    best = pick(timings)
    if cache_path:
        cache[key] = {"groups": best, "ms": {str(k): v for k, v in timings.items()}}
        save_cache(cache_path, cache)
    return best, timings


def time_solver_fs(R, ctx, J_dev: int, groups: int, repeats: int = 2) -> float:
    """Mean device time (ms) of the march kernel over `repeats` formal
    solutions of context `ctx` with `groups` direction groups (J_dev: a
    device buffer for the results)."""
    lib = R.load()
    R.rt_set_direction_groups(ctx, groups)
    R.rt_set_profiling(ctx, True)
    R.rt_reset_stats(ctx)
    for _ in range(repeats):
        rc = lib.rt_formal_solution_dev(ctx, None, J_dev, None)
        if rc != 0:
            raise R.RtError(rc, R.rt_last_error(ctx))
    st = R.rt_get_stats(ctx)
    R.rt_set_profiling(ctx, False)
    return st["fs_ms"] / max(st["fs_launches"], 1)


def autotune_solver(solver, cache_path: Optional[str] = DEFAULT_CACHE, refresh: bool = False,
                    repeats: int = 2) -> int:
    """Tune and apply the direction groups of a ``rt3d.Solver``."""
    import torch
    from . import rt3d as R
    p = solver.p
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = cache_key(p.nx, p.ny, p.nz, p.ndir, solver.precision, sms)
    buf = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float64, device="cuda")
    R.load().rt_formal_solution_dev(solver.ctx, None, buf.data_ptr(), None)  # warm-up
    best, _ = tune(key, lambda g: time_solver_fs(R, solver.ctx, buf.data_ptr(), g, repeats),
                   CANDIDATES, cache_path, refresh)
    R.rt_set_direction_groups(solver.ctx, best)
    return best
