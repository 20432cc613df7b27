"""FP32 vs FP64 position and velocity differences as a function of time since epoch
(the paper's precision study, Sec. 4), on one GPU.

For a synthetic element set (Starlink-shaped shells and a near-Earth catalogue draw) it
propagates the same records over 0 .. `days` days with the FP32 mixed-precision path and
the FP64 path, and reports per one-day bin the median, p99 and max of |r32 - r64| (km)
and |v32 - v64| (km/s) over the states both paths call valid (status 0 or 6).  The FP64
path agrees with the FP64 oracle to 1e-6 km (the parity tests), so these differences are
the FP32 path's errors to within that.

Usage: python -m paper_2603_27830_b300.precision_study [--days 14] [--out FILE.jsonl]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np
import torch

from . import sgp4_init, sgp4_propagate
from . import workloads as W


def study(name: str, elements: np.ndarray, days: float, per_day: int, out=None):
    dev = torch.device("cuda")
    t = np.linspace(0.0, days * 1440.0, int(days * per_day) + 1)
    el = torch.as_tensor(elements, device=dev)
    ts = torch.as_tensor(t, device=dev)
    recs, _ = sgp4_init(el)
    r32, v32, s32 = sgp4_propagate(recs, ts, "fp32")
    r64, v64, s64 = sgp4_propagate(recs, ts, "fp64")
    ok = ((s64 == 0) | (s64 == 6)) & (s32 == s64)
    dr = torch.linalg.vector_norm(r32.double() - r64, dim=-1)
    dv = torch.linalg.vector_norm(v32.double() - v64, dim=-1)
    mismatched = int((s32 != s64).sum())
    rows = []
    day_of = np.floor(t / 1440.0).astype(int)
    for d in range(int(np.ceil(days))):
        cols = torch.as_tensor(np.nonzero(day_of == d)[0], device=dev)
        m = ok[:, cols]
        a = dr[:, cols][m]
        b = dv[:, cols][m]
        if a.numel() == 0:
            continue
        qa = torch.quantile(a[:: max(1, a.numel() // 4_000_000)], torch.tensor(
            [0.5, 0.99], dtype=torch.float64, device=dev))
        qb = torch.quantile(b[:: max(1, b.numel() // 4_000_000)], torch.tensor(
            [0.5, 0.99], dtype=torch.float64, device=dev))
        row = {"set": name, "n_sats": int(el.shape[0]), "day": d, "states": int(a.numel()),
               "dr_median_km": float(qa[0]), "dr_p99_km": float(qa[1]),
               "dr_max_km": float(a.max()), "dv_median_kms": float(qb[0]),
               "dv_p99_kms": float(qb[1]), "dv_max_kms": float(b.max()),
               "status_mismatches": mismatched}
        rows.append(row)
        line = json.dumps(row)
        print(line, flush=True)
        if out:
            out.write(line + "\n")
    return rows


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--days", type=float, default=14.0)
    ap.add_argument("--per-day", type=int, default=144, help="times per day (default: 10 min)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    out = open(args.out, "w") if args.out else None
    try:
        study("starlink-9341", W.config2(seed=0).elements, args.days, args.per_day, out)
        rng = np.random.default_rng(14)
        study("catalogue-100000", W.catalogue_elements(rng, 100_000, invalid_frac=0.0),
              args.days, args.per_day, out)
    finally:
        if out:
            out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
