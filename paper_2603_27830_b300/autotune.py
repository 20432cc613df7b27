"""Autotuner for the batched persistent launch.

The tunable shape is the work tile: how many consecutive states (a run along the
time axis of one satellite, then the next satellites of the same request) a block
takes from the tile counter at a time, and the persistent grid size.  Small tiles
balance uneven requests better; large tiles cost fewer counter atomics and record
reloads.  ``tune_batch`` times each candidate on the caller's own batch with CUDA
events and keeps the fastest; results are cached in a JSON file keyed by the
device, the precision and a coarse signature of the batch (request count, total
states and mean grid length, each bucketed to a power of two).

Cache file: $SGP4_AUTOTUNE_CACHE, else ~/.cache/sgp4_b300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import numpy as np
import torch

from .api import BatchPlan, Records, plan_batch, sgp4_propagate_batched

TILE_CANDIDATES = (256, 512, 1024, 2048, 4096, 8192)
GRID_WAVES = (0,)          # 0 = one full wave (resident blocks x SMs)
DEFAULT_TILE = 1024

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("SGP4_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sgp4_b300",
                                       "autotune.json"))


def _bucket(x: float) -> int:
    return int(round(math.log2(max(1.0, float(x)))))


def signature(requests: np.ndarray, precision: str, device=None) -> str:
    req = np.asarray(requests, dtype=np.int64).reshape(-1, 5)
    states = int((req[:, 1] * req[:, 3]).sum())
    mean_t = float(req[:, 3].mean()) if len(req) else 0.0
    name = torch.cuda.get_device_name(device)
    return f"{name}|{precision}|req2^{_bucket(len(req))}|states2^{_bucket(states)}|T2^{_bucket(mean_t)}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_plan(plan: BatchPlan, records: Records, tsince: torch.Tensor, precision: str,
              out: tuple, reps: int = 3) -> float:
    """Median device time (ms) of one batched launch."""
    sgp4_propagate_batched(plan, records, tsince, precision, out=out)   # warm-up
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        sgp4_propagate_batched(plan, records, tsince, precision, out=out)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def tune_batch(requests, records: Records, tsince: torch.Tensor, precision: str = "fp32",
               out: tuple | None = None, candidates=TILE_CANDIDATES, reps: int = 3,
               use_cache: bool = True) -> tuple[BatchPlan, dict]:
    """Pick the tile size for this batch (cached); returns the plan and the record."""
    req = np.asarray(requests, dtype=np.int64).reshape(-1, 5)
    key = signature(req, precision, tsince.device)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        entry = cache[key]
        return plan_batch(req, entry["tile_states"], entry["grid_blocks"], tsince.device), entry
    if out is None:
        probe = plan_batch(req, DEFAULT_TILE, 0, tsince.device)
        dt = torch.float32 if precision == "fp32" else torch.float64
        S = int(probe.c.out_needed)
        out = (torch.empty((S, 3), dtype=dt, device=tsince.device),
               torch.empty((S, 3), dtype=dt, device=tsince.device),
               torch.empty((S,), dtype=torch.int32, device=tsince.device))
    trials = []
    for tile in candidates:
        for grid in GRID_WAVES:
            plan = plan_batch(req, tile, grid, tsince.device)
            trials.append((time_plan(plan, records, tsince, precision, out, reps), tile, grid))
    best_ms, tile, grid = min(trials)
    entry = {"tile_states": tile, "grid_blocks": grid, "ms": best_ms,
             "trials": [{"tile_states": t, "grid_blocks": g, "ms": m} for m, t, g in trials]}
    if use_cache:
        with _lock:
            cache = _load()
            cache[key] = entry
            _store(cache)
    return plan_batch(req, tile, grid, tsince.device), entry
