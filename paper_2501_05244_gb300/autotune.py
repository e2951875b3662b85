"""Autotuner of a plan's launch shapes (the spread's tile height, the batched form's grouping and stream count).

The tunables change only speed: every setting computes the same operator (up to FP32 summation
order).  :func:`autotune` times a caller-supplied step -- one call of the operation being tuned, on
representative inputs -- for each candidate value of each tunable in turn (coordinate descent,
holding the others at their best so far), keeps the fastest, and caches the choice in a JSON file
keyed by the GPU's name, the plan's shape and a caller-supplied workload tag (for example the sample
count range of a batch).  A cached choice is applied without timing.
"""
from __future__ import annotations

import json
import os
import tempfile
from typing import Callable, Dict, Iterable, Optional

from .nursd import NursdError

#: candidate values of each tunable
DEFAULT_SPACE: Dict[str, Iterable[int]] = {"batch_grouped": (1, 0), "spread_rows": (4, 8, 16),
                                           "batch_streams": (1, 2, 4, 8, 16)}


def default_cache_path() -> str:
    """$NURSD_TUNE_CACHE, else ~/.cache/nursd/tune.json."""
    return os.environ.get("NURSD_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "nursd",
                                                               "tune.json")


def gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device())


def shape_key(plan, workload: str = "", gpu: Optional[str] = None) -> str:
    """Cache key: GPU name, plan shape (N, F, Z, T) and the caller's workload tag."""
    return f"{gpu if gpu is not None else gpu_name()}|N={plan.N}|F={plan.F}|Z={plan.Z}|T={plan.T}|{workload}"


def cuda_event_timer(step: Callable[[], object], reps: int, warmup: int) -> float:
    """Mean milliseconds of `step` over `reps` calls after `warmup`, CUDA events on the current stream."""
    import torch

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(plan, step: Callable[[], object], workload: str = "", space: Optional[Dict[str, Iterable[int]]] = None,
             cache_path: Optional[str] = None, use_cache: bool = True, reps: int = 5, warmup: int = 2,
             timer: Callable[[Callable[[], object], int, int], float] = cuda_event_timer,
             gpu: Optional[str] = None) -> dict:
    """Choose the fastest value of each tunable for `step` on `plan`, apply it, and cache it.

    Returns {"key", "choice", "cached", "results" (ms of every timed setting), "ms" (best)}.
    """
    space = space if space is not None else DEFAULT_SPACE
    path = cache_path or default_cache_path()
    key = shape_key(plan, workload, gpu)
    cache = _load(path)
    if use_cache and key in cache:
        for name, value in cache[key]["choice"].items():
            plan.tune(name, value)
        return {"key": key, "choice": dict(cache[key]["choice"]), "cached": True,
                "results": cache[key].get("results", {}), "ms": cache[key].get("ms")}
    results = {}
    best_ms = None
    for name, values in space.items():
        best = None
        for v in values:
            try:
                plan.tune(name, v)
            except NursdError:  # not applicable to this plan's shape
                continue
            ms = float(timer(step, reps, warmup))
            results[f"{name}={v}"] = ms
            if best is None or ms < best[1]:
                best = (v, ms)
        if best is not None:
            plan.tune(name, best[0])
            best_ms = best[1]
    choice = {name: plan.tuning()[name] for name in space}
    cache = _load(path)  # another process may have written meanwhile
    cache[key] = {"choice": choice, "results": results, "ms": best_ms}
    _store(path, cache)
    return {"key": key, "choice": choice, "cached": False, "results": results, "ms": best_ms}
