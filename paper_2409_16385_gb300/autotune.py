"""Launch-shape autotuner for the kernels whose best shape depends on the workload: the
per-pair barrier evaluation (threads per block, grid cap in blocks per SM, register
budget), the pair tile of its work queue and of the CCD advancement's (items a warp claims
at a time), the BVH traversal (threads per block, grid cap, register budget) and the BVH
refit (how its bottom-up arrival counters are ordered).

Results never depend on the shape: every kernel is a grid-stride loop over a device-side
count, and every reduction order is fixed by sort keys, not by the launch.  So the tuner
is free to pick on time alone.  It times each candidate with the library's per-kernel
CUDA-event timers on the caller's own stage (one call of `stage()` runs the workload once),
takes the median of a few repetitions, and keeps the fastest.  Choices are cached in a
JSON file keyed by device name, compute capability and a workload key chosen by the
caller, so later runs on the same kind of GPU and workload skip the search.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Tuple

EVAL_SPACE: Tuple[Tuple[int, int, int], ...] = tuple(
    (threads, bps, variant) for threads in (64, 128) for bps in (2, 3, 4, 6, 8, 16) for variant in (2, 3, 4))
# items a warp claims from the evaluation's / CCD advancement's work queue at a time
TILE_SPACE: Tuple[Tuple[int, int, int], ...] = tuple((items, 1, 0) for items in (32, 64, 128, 256))
QUERY_SPACE: Tuple[Tuple[int, int, int], ...] = tuple(
    (threads, bps, variant) for threads in (64, 128, 256) for bps in (2, 4, 8, 12, 16, 24, 32) for variant in (2, 3))

REFIT_SPACE: Tuple[Tuple[int, int, int], ...] = ((256, 8, 0), (256, 8, 1), (256, 8, 2))

SPACES = {"eval_barrier": EVAL_SPACE, "bvh_query": QUERY_SPACE, "bvh_refit": REFIT_SPACE, "eval_tile": TILE_SPACE,
          "ccd_tile": TILE_SPACE}
# the library timer that brackets each tunable kernel's launches
TIMERS = {"eval_barrier": "eval_barrier", "bvh_query": "bvh_query", "bvh_refit": "bvh_build",
          "eval_tile": "eval_barrier", "ccd_tile": "ccd_advance"}


def default_cache_path() -> str:
    return os.environ.get("EMBIPC_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm_{p.major}{p.minor}|{p.multi_processor_count}sm"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_kernel(cs, stage: Callable[[], None], kernel: str, reps: int = 3) -> float:
    """Median over `reps` calls of stage() of the summed device time of `kernel`'s
    launches in one call (ms)."""
    import torch
    cs.timing_enable([kernel])
    samples = []
    for _ in range(reps):
        stage()
        torch.cuda.synchronize()
        ms, n = cs.timing_read().get(kernel, (0.0, 0))
        samples.append(ms)
    cs.timing_enable([])
    samples.sort()
    return samples[len(samples) // 2]


def tune(cs, stage: Callable[[], None], workload_key: str,
         kernels: Iterable[str] = ("eval_barrier", "eval_tile", "bvh_query", "bvh_refit", "ccd_tile"),
         cache_path: Optional[str] = None, reps: int = 3, force: bool = False) -> Dict[str, dict]:
    """Chooses and applies a launch shape for each kernel on `cs` (a ContactScene).

    stage() must run the workload once on torch's current stream (it is called about
    (1 + reps) times per candidate).  Returns {kernel: {"shape": [threads, bps, variant],
    "ms": best, "default_ms": time of the library default, "cached": bool}}."""
    path = cache_path or default_cache_path()
    table = _load(path)
    key = f"{device_key()}|{workload_key}"
    entry = table.get(key, {})
    out = {}
    for kernel in kernels:
        if not force and kernel in entry:
            shape = entry[kernel]["shape"]
            cs.set_launch(kernel, *shape)
            out[kernel] = dict(entry[kernel], cached=True)
            continue
        timer = TIMERS[kernel]
        stage()                                   # warm: hierarchies built, caches primed
        default_ms = time_kernel(cs, stage, timer, reps)
        best, best_ms, seen = None, float("inf"), {}
        for shape in SPACES[kernel]:
            cs.set_launch(kernel, *shape)
            stage()
            ms = time_kernel(cs, stage, timer, reps)
            seen["x".join(map(str, shape))] = ms
            if ms < best_ms:
                best, best_ms = shape, ms
        cs.set_launch(kernel, *best)
        entry[kernel] = dict(shape=list(best), ms=best_ms, default_ms=default_ms, candidates=seen)
        out[kernel] = dict(entry[kernel], cached=False)
    table[key] = entry
    _store(path, table)
    return out
