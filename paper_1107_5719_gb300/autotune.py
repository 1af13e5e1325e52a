"""Launch-shape autotuner for the formal-solution march.

The march's work per voxel is split into 8 fixed direction slots.  Free
launch parameters: how many thread blocks share the slots of a voxel tile
("direction groups", 1, 2, 4 or 8) and, for the FP32-sweep march, the
threads per block (64, 128 or 256: the tile width, at about the same
resident threads per SM) and the block order (tile- or plane-major).  More groups give more, shorter blocks (better balance of
the depth-dependent characteristic lengths and of the transmission cutoff),
fewer groups give fewer blocks that re-read less; narrower blocks give a
finer last wave.  J does not depend on either choice (fixed summation
order), so the tuner only times them: each candidate runs a few formal
solutions (or batch iterations) with CUDA events on the launching stream
(the library's profiling counters), and the fastest mean wins.  Results are
cached in a JSON file keyed by grid shape, direction count, precision and
SM count (and the batch size for batches).  Every direction sums into its
slot whatever its sign, so each thread already marches both members of a
mirror pair mu, -mu (k0 and nz-1-k0 steps): the per-thread work is balanced
across planes without a separate pairing knob.
"""

from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Tuple

CANDIDATES = (1, 2, 4, 8)
# (groups, threads per block, block order) of the FP32-sweep march; block
# order 1 = the tiles of a plane consecutive, 2 = the planes of a tile
CANDIDATES_FP32 = tuple((g, t, o) for o in (1, 2) for t in (64, 128, 256) for g in (1, 2, 4, 8))
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


def pick(timings: Dict) -> object:
    """Fastest candidate; ties go to the smaller one (fewer groups, then
    fewer threads per block, then the lower block order)."""
    return min(timings, key=lambda g: (timings[g], g))


def _enc(c):
    """Cache form of a candidate: an int, or "groups x threads x order"."""
    return "x".join(str(v) for v in c) if isinstance(c, tuple) else int(c)


def _dec(s):
    s = str(s)
    return tuple(int(v) for v in s.split("x")) if "x" in s else int(s)


def tune(key: str, time_candidate: Callable, candidates: Iterable = CANDIDATES,
         cache_path: Optional[str] = DEFAULT_CACHE, refresh: bool = False) -> Tuple[object, Dict]:
    """Return (best candidate, {candidate: ms}) for `key`, from the cache
    unless `refresh`; `time_candidate(c)` returns the mean ms of the march
    with candidate c (a group count, or a (groups, threads, order) tuple)."""
    cache = load_cache(cache_path) if cache_path else {}
    if not refresh and key in cache and "groups" in cache[key]:
        return _dec(cache[key]["groups"]), {_dec(k): v for k, v in cache[key].get("ms", {}).items()}
    cands = [tuple(c) if isinstance(c, (tuple, list)) else int(c) for c in candidates]
    timings = {c: float(time_candidate(c)) for c in cands}
    best = pick(timings)
    if cache_path:
        cache[key] = {"groups": _enc(best), "ms": {str(_enc(k)): v for k, v in timings.items()}}
        save_cache(cache_path, cache)
    return best, timings


def _apply(R, ctx, cand):
    if isinstance(cand, tuple):
        R.rt_set_direction_groups(ctx, cand[0])
        R.rt_set_block_threads(ctx, cand[1])
        if len(cand) > 2:
            R.rt_set_block_order(ctx, cand[2])
    else:
        R.rt_set_direction_groups(ctx, cand)


def _apply_batch(R, b, cand):
    R.rt_batch_set_direction_groups(b, cand[0])
    R.rt_batch_set_block_threads(b, cand[1])
    if len(cand) > 2:
        R.rt_batch_set_block_order(b, cand[2])


def time_solver_fs(R, ctx, J_dev: int, cand, repeats: int = 2) -> float:
    """Mean device time (ms) of the march kernel over `repeats` formal
    solutions of context `ctx` with launch shape `cand` (J_dev: a device
    buffer for the results)."""
    lib = R.load()
    _apply(R, ctx, cand)
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
                    repeats: int = 2):
    """Tune and apply the launch shape of a ``rt3d.Solver`` (direction
    groups; for the FP32 sweep also threads per block and block order)."""
    import torch
    from . import rt3d as R
    p = solver.p
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = cache_key(p.nx, p.ny, p.nz, p.ndir, solver.precision, sms)
    cands = CANDIDATES_FP32 if solver.precision == R.RT_FP32_SWEEP else CANDIDATES
    buf = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float64, device="cuda")
    R.load().rt_formal_solution_dev(solver.ctx, None, buf.data_ptr(), None)  # warm-up
    best, _ = tune(key, lambda c: time_solver_fs(R, solver.ctx, buf.data_ptr(), c, repeats),
                   cands, cache_path, refresh)
    _apply(R, solver.ctx, best)
    return best


def time_batch_fs(R, b, nprob: int, cand, iters: int = 1) -> float:
    """Mean device time (ms) of the fused FP32 march of a batch over `iters`
    outer iterations from J = B with launch shape `cand` = (groups, threads,
    block order);
    the batch is reset afterwards (Lambda* kept)."""
    _apply_batch(R, b, cand)
    R.rt_batch_reset(b)
    R.rt_batch_reset_stats(b)
    R.rt_batch_set_profiling(b, True)
    R.rt_batch_solve(b, nprob, tol=0.0, max_iter=iters)
    st = R.rt_batch_get_stats(b)
    R.rt_batch_set_profiling(b, False)
    R.rt_batch_reset(b)
    return st["fs_ms"] / max(st["fs_launches"], 1)


def autotune_batch(b, problems, cache_path: Optional[str] = DEFAULT_CACHE, refresh: bool = False,
                   iters: int = 1):
    """Tune and apply the fused launch shape, (groups, threads per block,
    block order), of
    an FP32-sweep batch, keyed by the largest grid, direction count, batch
    size and SM count."""
    import torch
    from . import rt3d as R
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    big = max(problems, key=lambda p: p.nvox)
    key = cache_key(big.nx, big.ny, big.nz, big.ndir, R.RT_FP32_SWEEP, sms) + f":b{len(problems)}"
    R.rt_batch_solve(b, len(problems), tol=0.0, max_iter=1)          # warm-up, builds Lambda*
    best, _ = tune(key, lambda c: time_batch_fs(R, b, len(problems), c, iters),
                   CANDIDATES_FP32, cache_path, refresh)
    _apply_batch(R, b, best)
    R.rt_batch_reset(b)
    return best
