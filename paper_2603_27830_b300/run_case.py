"""Run one workload through sgp4_init + sgp4_propagate a few times (for profilers).

    python -m paper_2603_27830_b300.run_case --workload starlink --precision fp32 --reps 2

Workloads: near-earth (64 x 100), starlink (9,341 x 1,000), catalogue (1,000,000 x
100; ``--n`` shrinks it).  Prints the wall time of each repetition.
"""
from __future__ import annotations

import argparse
import time

import torch

from . import sgp4_init, sgp4_propagate
from . import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["near-earth", "starlink", "catalogue"],
                    default="starlink")
    ap.add_argument("--precision", choices=["fp32", "fp64", "both"], default="fp32")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--n", type=int, default=None)
    args = ap.parse_args()
    if args.workload == "near-earth":
        w = W.config1()
    elif args.workload == "starlink":
        w = W.config2()
    else:
        w = W.config3(n=args.n or 1_000_000)
    el = torch.as_tensor(w.elements, device="cuda")
    ts = torch.as_tensor(w.tsince, device="cuda")
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        for k in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            recs, _ = sgp4_init(el)
            r, v, st = sgp4_propagate(recs, ts, prec)
            torch.cuda.synchronize()
            print(f"{w.name} {prec} rep {k}: {1e3 * (time.perf_counter() - t0):.3f} ms")
            del r, v, st


if __name__ == "__main__":
    main()
