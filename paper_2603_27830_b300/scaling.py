"""Scaling sweep of the propagation on one GPU (the paper's scaling analysis, Sec. 3.2):
1 satellite x 1 .. 1e7 times, 1 .. 2e6 satellites x 1 time, and an N x T grid, on the
Starlink-shaped element generator with one-day grids.  For each point it reports the
time of one `sgp4_propagate` call (FP32 and FP64) and the states/s it implies.

Protocol (Sec. 3.1): records built and inputs resident on the device before timing,
warm-up excluded, each trial repeats the call until at least 0.2 s has passed, 5 trials,
the minimum time per call reported; CUDA events on the launching stream.  The time per
call includes the host side of the Python call, so the small sizes show the per-call
latency floor of the API.

Usage: python -m paper_2603_27830_b300.scaling [--out sweep.jsonl] [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import torch

from . import sgp4_init, sgp4_propagate
from . import workloads as W

STATE_BYTES = {"fp32": 28, "fp64": 52}


def _points(quick: bool):
    top_t = 10 ** (5 if quick else 7)
    top_n = 10 ** 5 if quick else 2_000_000
    pts = [("1xT", 1, 10 ** k) for k in range(int(math.log10(top_t)) + 1)]
    ns = [10 ** k for k in range(int(math.log10(top_n)) + 1)]
    if top_n not in ns:
        ns.append(top_n)
    pts += [("Nx1", n, 1) for n in ns]
    grid_n = [10 ** k for k in range(0, 5 if quick else 7)]
    grid_t = [10 ** k for k in range(0, 4 if quick else 5)]
    cap = 10 ** (7 if quick else 9)
    pts += [("NxT", n, t) for n in grid_n for t in grid_t if n * t <= cap]
    return pts


def time_call(fn, min_s: float = 0.2, trials: int = 5) -> float:
    """Minimum over `trials` of the mean time (ms) of `fn` repeated for >= min_s."""
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    one = max(a.elapsed_time(b), 1e-3)
    reps = max(1, int(math.ceil(min_s * 1e3 / one)))
    best = float("inf")
    for _ in range(trials):
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / reps)
    return best


def run(points, precisions=("fp32", "fp64"), out=None):
    dev = torch.device("cuda")
    rows = []
    for kind, n, t_count in points:
        w = W.config2(seed=0, n=n, t_count=t_count)
        el = torch.as_tensor(w.elements, device=dev)
        ts = torch.as_tensor(w.tsince, device=dev)
        recs, _ = sgp4_init(el)
        for prec in precisions:
            dt = torch.float32 if prec == "fp32" else torch.float64
            buf = (torch.empty((n, t_count, 3), dtype=dt, device=dev),
                   torch.empty((n, t_count, 3), dtype=dt, device=dev),
                   torch.empty((n, t_count), dtype=torch.int32, device=dev))
            ms = time_call(lambda: sgp4_propagate(recs, ts, prec, out=buf))
            states = n * t_count
            row = {"sweep": kind, "n_sats": n, "t_count": t_count, "states": states,
                   "precision": prec, "ms_per_call": ms, "states_per_s": states / (ms * 1e-3),
                   "output_gb_per_s": states * STATE_BYTES[prec] / (ms * 1e-3) / 1e9}
            rows.append(row)
            line = json.dumps(row)
            print(line, flush=True)
            if out:
                out.write(line + "\n")
                out.flush()
            del buf
        del recs, el, ts
        torch.cuda.empty_cache()
    return rows


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=None, help="also write the JSON lines to this file")
    ap.add_argument("--quick", action="store_true", help="sizes up to 1e7 states only")
    args = ap.parse_args(argv)
    out = open(args.out, "w") if args.out else None
    try:
        run(_points(args.quick), out=out)
    finally:
        if out:
            out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
