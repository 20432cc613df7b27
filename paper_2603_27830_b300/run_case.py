"""Run one workload through sgp4_init + sgp4_propagate a few times (for profilers).

    python -m paper_2603_27830_b300.run_case --workload starlink --precision fp32 --reps 2

Workloads: near-earth (64 x 100), starlink (9,341 x 1,000), catalogue (1,000,000 x
100; ``--n`` shrinks it), batch (64 uneven requests, N_i log-U[100,5e3], T_i
log-U[10,500]: the batched persistent launch), adjoint (the fitting workload,
10,000 x 500: one sgp4_adjoint call), fit (the same workload: one sgp4_fit_step call
against observations of the perturbed elements), jacobian (the same workload: one
sgp4_jacobian call with an element covariance), fit-forward (the same workload: init +
propagate), deep-space (10,000 deep-space satellites with their own epochs x 1,000 times
over seven days; ``--n`` shrinks it; ``--order-by-class`` groups its records by the
branches their states take).  Prints the wall time of each repetition.
"""
from __future__ import annotations

import argparse
import time

import torch

from . import sgp4_init, sgp4_propagate
from . import workloads as W


def _timed(label, fn, reps):
    for k in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        print(f"{label} rep {k}: {1e3 * (time.perf_counter() - t0):.3f} ms")


def run_batch(args):
    from . import make_batch, plan_batch, sgp4_propagate_batched
    reqs = W.config4(seed=0, n_requests=64, n_range=(100, 5000), t_range=(10, 500))
    b = make_batch([(q.elements, q.tsince) for q in reqs])
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    plan = plan_batch(b.requests, 2048)
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        out = sgp4_propagate_batched(plan, recs, ts, prec)
        _timed(f"batch {plan.total_states} states {prec}",
               lambda: sgp4_propagate_batched(plan, recs, ts, prec, out=out), args.reps)


def run_adjoint(args):
    from . import sgp4_adjoint
    w = W.config5(n=args.n or 10_000)
    el = torch.as_tensor(w.elements, device="cuda")
    ts = torch.as_tensor(w.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        dt = torch.float32 if prec == "fp32" else torch.float64
        g = torch.randn((w.n, w.t_count, 3), dtype=dt, device="cuda")
        _timed(f"adjoint {w.states} states {prec}",
               lambda: sgp4_adjoint(el, recs, ts, g, g, prec), args.reps)


def run_fit(args):
    from .fit import fit_step
    w = W.config5(n=args.n or 10_000)
    el = torch.as_tensor(w.elements, device="cuda")
    ts = torch.as_tensor(w.tsince, device="cuda")
    truth, _ = sgp4_init(torch.as_tensor(w.meta["truth"], device="cuda"))
    r_true = sgp4_propagate(truth, ts, "fp64")[0]
    r_obs = r_true + torch.as_tensor(w.meta["noise"](tuple(r_true.shape)), device="cuda")
    lam = torch.full((w.n,), 1e-3, dtype=torch.float64, device="cuda")
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        _timed(f"fit step {w.states} states {prec}",
               lambda: fit_step(el, ts, r_obs, lam, prec), args.reps)


def run_jacobian(args):
    from . import sgp4_jacobian
    w = W.config5(n=args.n or 10_000)
    el = torch.as_tensor(w.elements, device="cuda")
    ts = torch.as_tensor(w.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    cov = torch.diag_embed(torch.full((w.n, 7), 1e-10, dtype=torch.float64, device="cuda"))
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        _timed(f"jacobian {w.states} states {prec}",
               lambda: sgp4_jacobian(el, recs, ts, prec, cov=cov), args.reps)


def deep_class_order(elements):
    """Host-side order of deep-space elements [n, 7] grouped by the branches their states
    take: resonance (about one revolution a day; about two with e0 >= 0.5; none, from
    the Kozai mean motion), inclination below 0.2 rad (the Lyddane form of the
    periodics) and the Newton step count of e0.  Returns the permutation."""
    import math

    import numpy as np
    el = np.asarray(elements)
    rev = el[:, 0] * 1440.0 / (2.0 * math.pi)
    rez = np.where(np.abs(rev - 1.0027) < 0.1, 1,
                   np.where((rev > 1.9) & (rev < 2.1) & (el[:, 1] >= 0.5), 2, 0))
    e2 = el[:, 1] ** 2
    eb = sum((e2 > th).astype(int) for th in (1.5876e-10, 9.3e-5, 0.01664, 0.1347, 0.25))
    key = ((rez * 2 + (el[:, 2] < 0.2)) * 8 + eb)
    return np.argsort(key, kind="stable")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["near-earth", "starlink", "catalogue", "batch",
                                           "adjoint", "fit", "jacobian", "fit-forward",
                                           "deep-space"],
                    default="starlink")
    ap.add_argument("--precision", choices=["fp32", "fp64", "both"], default="fp32")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--order-by-class", action="store_true",
                    help="deep-space: group the records by class before sgp4_init")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "fit":
        return run_fit(args)
    if args.workload == "jacobian":
        return run_jacobian(args)
    if args.workload == "near-earth":
        w = W.config1()
    elif args.workload == "starlink":
        w = W.config2()
    elif args.workload == "fit-forward":
        w = W.config5(n=args.n or 10_000)
    elif args.workload == "deep-space":
        w = W.deep_space(n=args.n or 10_000)
    else:
        w = W.config3(n=args.n or 1_000_000)
    import numpy as np
    order = (deep_class_order(w.elements) if args.order_by_class
             else np.arange(len(w.elements)))
    el = torch.as_tensor(np.asarray(w.elements)[order], device="cuda")
    ts = torch.as_tensor(w.tsince, device="cuda")
    ep = {}
    if "epoch_day" in w.meta:
        ep = {"epoch_day": torch.as_tensor(np.asarray(w.meta["epoch_day"])[order], device="cuda"),
              "epoch_frac": torch.as_tensor(np.asarray(w.meta["epoch_frac"])[order],
                                            device="cuda")}
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        for k in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            recs, _ = sgp4_init(el, **ep)
            r, v, st = sgp4_propagate(recs, ts, prec)
            torch.cuda.synchronize()
            print(f"{w.name} {prec} rep {k}: {1e3 * (time.perf_counter() - t0):.3f} ms")
            del r, v, st


if __name__ == "__main__":
    main()
