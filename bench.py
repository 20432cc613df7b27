#!/usr/bin/env python
"""Throughput benchmark of the SGP4 hot path: propagated states/s.

One step = sgp4_init (record build) + sgp4_propagate (secular update, long-period
terms, Kepler, short-period terms, TEME output) of the Starlink-shaped workload,
9,341 satellites x 1,000 times over one day, on the FP32 mixed-precision path;
the plain FP64 GPU path is timed beside it.  Inputs are resident in HBM when the
timed region starts; L2 is flushed (256 MB write) between timed steps.

Beside the headline the line carries the FP64 path, the batched uneven-request launch
(256 requests, CUDA-graph replay) and the adjoint / fitting workload (10,000 x 500:
sgp4_adjoint, one Levenberg-Marquardt step and the per-state Jacobians with covariance,
FP32 and FP64), each with its rate and roofline fraction.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (the
only reference this project has: the paper ships no runnable code here).
Under torchrun each rank propagates its own copy of the workload (independent
problems, no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "propagated states/s (sat x time) FP32 vs FP64 at stated max |dr| km; % roofline"
UNIT = "states/s"

# The paper's own figure for this workload and metric (Sec. 3.2): the full Starlink
# catalogue, 9,341 satellites x 1,000 times, FP32, record build + propagation, 3.8 ms
# on one A100.
PAPER_STATES_PER_S = 9341 * 1000 / 3.8e-3

# Per-state algorithmic output bytes (r, v as float32 x3 + int32 status; FP64: doubles).
BYTES_PER_STATE = {"fp32": 28, "fp64": 52}
# FP32 arithmetic + SFU operations per state of the FP32 formulation on the
# Starlink-shaped workload, counted with ncu on the current kernel: each packed
# instruction (FADD2, FMUL2, FFMA2) is two lane operations, one for each state of its
# pair: FADD 38.1 + FMUL 97.1 + FFMA 54.1 + SFU 18.1 per state (ncu's per-opcode and
# per-pipe instruction counts of one launch divided by the launch's states).
ALG_OPS_FP32 = 207
# DRAM bytes (read + write) of one launch of the FP32 propagate kernel on this workload,
# from an ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch after one warm-up launch): below the 28 B/state
# written because L2 still holds the tail of the output when the kernel ends.
TRAFFIC_FP32_BYTES = 203_369_984
# FP64 arithmetic (DADD + DMUL + DFMA thread instructions) per state of the FP64
# propagation on the Starlink-shaped workload, counted with ncu (DADD 15.0, DMUL 140.0,
# DFMA 210.0).
ALG_OPS_FP64 = 365
# Per state of the adjoint sweep on the fitting workload (10,000 x 500), counted with
# ncu: FP32 path FADD 78.4 + FMUL 221.6 + FFMA 169.9 + SFU 29.8 lane operations, the mix
# of the scalar sweep (one state per thread).  The packed sweep now run (two states per
# thread) executes 536 (FADD2/FMUL2/FFMA2 x 2 lanes + scalar FADD/FMUL/FFMA + SFU: the
# negations and sums of its packed form add some); the smaller count is the one used.
# FP64 path DADD + DMUL + DFMA.
ALG_OPS_ADJ_FP32 = 500
ALG_OPS_ADJ_FP64 = 707
# DADD + DMUL + DFMA per state of the FP64 Jacobian kernel (one forward and six reverse
# sweeps with the init Jacobian contraction and the covariance) and of the FP64 fit-step
# kernel (one forward and three reverse sweeps, the normal-equation sums), counted with
# ncu on 2,000 x 500 of the fitting workload.
ALG_OPS_JAC_FP64 = 3564
ALG_OPS_FIT_FP64 = 1823
# The same kernels in FP32 (FADD + FMUL + FFMA thread instructions and the SFU's, ncu on
# 2,000 x 500): Jacobian FADD 115.3, FMUL 1049.8, FFMA 2345.6, SFU 75.0; fit step FADD
# 130.5, FMUL 549.8, FFMA 1091.2, SFU 47.8.
ALG_OPS_JAC_FP32 = 3586
ALG_OPS_FIT_FP32 = 1819
# B300's FP64 unit: 2 lanes per SM per clock (one warp instruction per 64 cycles per
# SM sub-partition; ncu's fp64-pipe utilisation and instruction count give the rate).
FP64_LANES_PER_SM_CLK = 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def max_over_ranks(x: float, device) -> float:
    """Largest x over the ranks of the default process group (x when there is none):
    the job's time is that of its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Before each timed step the stream first runs a bounded GPU delay (PyTorch's clock-spin
# kernel, outside the timed region) while the host enqueues the step, so that the
# events time the GPU's work and not gaps in which the host had not yet submitted the
# next launch (on a slow host those gaps made a kernel's time exceed the whole step's).
# The lead must also cover the host while the NVML clock sampler's thread holds the
# interpreter: with 0.2 ms the headline step measured 0.120 ms under the sampler
# against 0.111 ms without it.
HOST_LEAD_CYCLES = 2_000_000    # about 1 ms at 2 GHz


def host_lead(torch) -> None:
    torch.cuda._sleep(HOST_LEAD_CYCLES)


def job_rate(states_per_rank: int, steps: int, world: int, ms_total: float) -> float:
    """Whole-job states/s: every rank propagates its own replica of the workload (the
    states are independent; there is no data-path collective)."""
    return world * states_per_rank * steps / (ms_total * 1e-3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class _Nvml:
    """Minimal ctypes binding of the NVML calls the clock sampler needs (the driver's
    libnvidia-ml.so.1; no Python package required)."""

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        self.reason_fn = None
        for name in ("nvmlDeviceGetCurrentClocksEventReasons",
                     "nvmlDeviceGetCurrentClocksThrottleReasons"):
            if hasattr(self.lib, name):
                self.reason_fn = getattr(self.lib, name)
                break

    def handle(self, pci_bus_id: str | None, index: int):
        h = self.c.c_void_p()
        if pci_bus_id:
            if self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(),
                                                         self.c.byref(h)) == 0:
                return h
        if self.lib.nvmlDeviceGetHandleByIndex_v2(index, self.c.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        return h

    def sm_clock(self, h, max_clock=False):
        v = self.c.c_uint()
        fn = self.lib.nvmlDeviceGetMaxClockInfo if max_clock else self.lib.nvmlDeviceGetClockInfo
        if fn(h, 1, self.c.byref(v)) != 0:      # NVML_CLOCK_SM = 1
            raise RuntimeError("clock query failed")
        return v.value

    def reasons(self, h):
        v = self.c.c_ulonglong()
        if self.reason_fn is None or self.reason_fn(h, self.c.byref(v)) != 0:
            return 0
        return v.value


class ClockSampler:
    """SM clock and throttle reasons sampled through NVML every 2 ms while the timed
    region runs (the region is only milliseconds long)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, pci_bus_id: str | None, index: int):
        self.pci = pci_bus_id
        self.idx = index
        self.samples = []
        self.max_mhz = None
        self._stop = None
        self._thread = None
        self.error = None

    def __enter__(self):
        import threading
        try:
            nv = _Nvml()
            h = nv.handle(self.pci, self.idx)
            self.max_mhz = nv.sm_clock(h, max_clock=True)
        except Exception as exc:  # no NVML: report it instead of clocks
            self.error = f"nvml unavailable: {exc}"
            return self
        self._stop = threading.Event()

        def poll():
            while not self._stop.is_set():
                try:
                    self.samples.append((nv.sm_clock(h), nv.reasons(h)))
                except Exception as exc:
                    self.error = str(exc)
                    return
                time.sleep(0.002)

        self._thread = threading.Thread(target=poll, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz,
                    "reasons": [self.error or "no samples"]}
        reasons = sorted({name for _, rs in self.samples for bit, name in self.REASONS.items()
                          if rs & bit})
        return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(self.samples)}


def time_oracle(elements, tsince, threads: int, trials: int = 5, min_trial_s: float = 0.2,
                epoch=None):
    """The paper's timing protocol (Sec. 3.1) applied to the FP64 oracle as it stands:
    one call propagates every satellite to every time; a trial repeats the call until
    it has run at least min_trial_s, and the best of `trials` trials (time per call) is
    reported.  Returns (states/s, seconds per call, calls per trial)."""
    import oracle
    oracle.load()
    states = elements.shape[0] * tsince.shape[-1]
    reps = 1
    while True:                      # find a repetition count that fills a trial
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.propagate(elements, tsince, threads=threads, epoch=epoch)
        dt = time.perf_counter() - t0
        if dt >= min_trial_s:
            break
        reps = max(reps * 2, int(reps * min_trial_s / max(dt, 1e-6)) + 1)
    best = dt / reps
    for _ in range(trials - 1):
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.propagate(elements, tsince, threads=threads, epoch=epoch)
        best = min(best, (time.perf_counter() - t0) / reps)
    return states / best, best, reps


def _errors(r_dev, v_dev, st_dev, rows, rr, vr, sr):
    """FP32/FP64 path vs the oracle on the sampled satellites `rows` (device outputs
    [n, T, 3] / [n, T]): status mismatches, max and p99 of |dr| (km) and |dv| (km/s)
    over the states with output."""
    import torch
    idx = torch.as_tensor(rows, device=st_dev.device)
    r = r_dev[idx].double().cpu().numpy()
    v = v_dev[idx].double().cpu().numpy()
    st = st_dev[idx].cpu().numpy()
    keep = (sr == 0) | (sr == 6)
    dr = np.linalg.norm(r[keep] - rr[keep], axis=-1)
    dv = np.linalg.norm(v[keep] - vr[keep], axis=-1)
    out = {"status_mismatches": int((st != sr).sum()), "states": int(st.size)}
    if dr.size:
        out.update({"states_over_1e-6_km": int((dr > 1e-6).sum()),
                    "max_dr_km": float(dr.max()), "p99_dr_km": float(np.percentile(dr, 99)),
                    "median_dr_km": float(np.median(dr)), "max_dv_kms": float(dv.max()),
                    "p99_dv_kms": float(np.percentile(dv, 99))})
    return out


# FP32 and FP64 arithmetic per state of the propagate kernels on each single-problem
# workload, counted with ncu on the current kernels the same way as ALG_OPS_FP32 and
# ALG_OPS_FP64 (the FP32 count includes the SFU operations).  The count depends on
# the workload: eccentric orbits take more Newton steps, simplified-drag records skip
# the D terms, guard-band states add FP64 work.
# Counted per workload (packed FADD2 / FMUL2 / FFMA2 from the per-opcode table, two
# lane operations each; scalar FADD / FMUL / FFMA and XU from the per-pipe counters):
# near-earth 221, catalogue (100,000 x 100 of the same draw) 229, fitting workload 219
# lane operations per state on the current kernel.  FP64: DADD + DMUL + DFMA of the
# FP64 kernel.  Deep space: the FP64 DADD + DMUL + DFMA of the deep-space pass (the
# propagation launch's last blocks), which computes every deep-space state in both
# precisions (2,000 x 1,000 of the same draw:
# 93.3 M + 427.1 M + 780.7 M thread instructions for 2e6 states = 651 per state; with
# the comparisons, conversions and roundings the FP64 pipe issues 1,069 per state and
# is 86% busy).
OPS_PER_STATE = {
    "near-earth-64x100": {"fp32": 221, "fp64": 379},
    "starlink-9341x1000": {"fp32": ALG_OPS_FP32, "fp64": ALG_OPS_FP64},
    "catalogue-1Mx100": {"fp32": 229, "fp64": 406},
    "fit-10000x500": {"fp32": 219, "fp64": 384},
    "deep-space-10000x1000": {"fp32": 651, "fp64": 651},
}


def _roofline(prec, workload, states, kern_ms, alu_peak, fp64_peak, hbm_peak):
    """Roofline of one propagate launch: arithmetic against its pipe's peak (FP32 lanes
    or the FP64 unit) and output bytes against HBM; the bound is the slower side."""
    sec = kern_ms * 1e-3
    gbs = BYTES_PER_STATE[prec] * states / sec / 1e9
    out = {"hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                   "bytes_per_state": BYTES_PER_STATE[prec]}}
    ops = OPS_PER_STATE.get(workload, {}).get(prec)
    if ops is None:
        out.update({"bound": "hbm", "frac": gbs / hbm_peak})
        return out
    # deep-space states run on the FP64 unit in both precisions
    fp64_unit = prec == "fp64" or workload.startswith("deep-space")
    peak = fp64_peak if fp64_unit else alu_peak
    gops = ops * states / sec / 1e9
    t_alu = ops * states / (peak * 1e9)
    t_hbm = BYTES_PER_STATE[prec] * states / (hbm_peak * 1e9)
    bound = ("fp64" if fp64_unit else "alu") if t_alu >= t_hbm else "hbm"
    out.update({"bound": bound, "achieved": gops, "peak": peak, "unit": "Gop/s",
                "ops_per_state": ops, "frac": (gops / peak) if bound != "hbm" else gbs / hbm_peak,
                "alu_frac": gops / peak})
    return out


def run_single_config(torch, dev, stream, flush, steps, w, precs, n_sample, threads,
                      alu_peak, fp64_peak, hbm_peak, time_cpu=True):
    """One single-problem workload: per precision the step (sgp4_init + sgp4_propagate)
    and the propagate launch alone, each the median of `steps` timed runs with L2
    flushed between them, the roofline of the launch, and the error against the FP64
    oracle over the whole horizon on a sample of satellites (all of them when n_sample
    is None; the sampled ones always include every deliberately invalid record)."""
    import oracle

    from paper_2603_27830_b300 import sgp4_init, sgp4_propagate
    n, T = w.n, w.t_count
    el = torch.as_tensor(w.elements, device=dev)
    ts = torch.as_tensor(w.tsince, device=dev)
    # records with their own epochs (the deep-space workload): the deep-space terms
    # depend on them
    ep_dev, ep_host = {}, None
    if "epoch_day" in w.meta:
        ep_dev = {"epoch_day": torch.as_tensor(w.meta["epoch_day"], device=dev),
                  "epoch_frac": torch.as_tensor(w.meta["epoch_frac"], device=dev)}
        ep_host = (w.meta["epoch_day"].astype(np.float64), w.meta["epoch_frac"])
    recs, ist = sgp4_init(el, **ep_dev)
    if n_sample is None or n_sample >= n:
        rows = np.arange(n)
        sample = f"all {n} satellites x {T} times"
    else:
        rng = np.random.default_rng(12345)
        rows = np.unique(np.concatenate([rng.choice(n, n_sample, replace=False),
                                         np.asarray(w.meta.get("invalid", []), dtype=np.int64)]))
        sample = (f"{len(rows)} of {n} satellites (random, plus every invalid record) x "
                  f"{T} times")
    ep_rows = None if ep_host is None else (ep_host[0][rows], ep_host[1][rows])
    rr, vr, sr, _ = oracle.propagate(w.elements[rows], w.tsince, threads=threads, epoch=ep_rows)
    res = {"workload": w.name, "n_sats": n, "t_count": T,
           "horizon_min": [float(w.tsince.min()), float(w.tsince.max())],
           "error_sample": sample}
    if time_cpu:
        rate, per_call, reps = time_oracle(w.elements[rows], w.tsince, threads, epoch=ep_rows)
        res["oracle"] = {"value": rate, "unit": UNIT, "cores": threads, "sample": sample,
                         "s_per_call": per_call, "calls_per_trial": reps,
                         "protocol": "best of 5 trials, each >= 0.2 s"}

    def median_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            host_lead(torch)
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    for prec in precs:
        dt = torch.float32 if prec == "fp32" else torch.float64
        out = (torch.empty((n, T, 3), dtype=dt, device=dev),
               torch.empty((n, T, 3), dtype=dt, device=dev),
               torch.empty((n, T), dtype=torch.int32, device=dev))
        reps = steps if prec == "fp32" else max(3, min(steps, 5))

        def step():
            sgp4_init(el, records=recs, init_status=ist, **ep_dev)
            sgp4_propagate(recs, ts, prec, out=out)

        step_ms = median_ms(step, reps)
        kern_ms = median_ms(lambda: sgp4_propagate(recs, ts, prec, out=out), reps)
        step()
        torch.cuda.synchronize()
        err = _errors(out[0], out[1], out[2], rows, rr, vr, sr)
        res[prec] = {"value": n * T / (step_ms * 1e-3), "unit": UNIT, "ms_per_step": step_ms,
                     "kernel_ms": kern_ms, "kernel_states_per_s": n * T / (kern_ms * 1e-3),
                     "roofline": _roofline(prec, w.name, n * T, kern_ms, alu_peak, fp64_peak,
                                           hbm_peak),
                     "vs_oracle": err}
        del out
    del recs, ist, el, ts
    torch.cuda.empty_cache()
    return res


def run_batched(torch, dev, stream, flush, steps, sample_requests=0, threads=1):
    """Time the 256-request uneven batch (graph replay of one persistent launch)."""
    from paper_2603_27830_b300 import BatchGraph, autotune, make_batch, sgp4_init
    from paper_2603_27830_b300 import workloads as W
    reqs = W.config4(seed=0)
    b = make_batch([(q.elements, q.tsince) for q in reqs])
    el = torch.as_tensor(b.elements, device=dev)
    ts = torch.as_tensor(b.tsince, device=dev)
    recs, _ = sgp4_init(el)
    S = int((b.requests[:, 1] * b.requests[:, 3]).sum())
    out = (torch.empty((S, 3), dtype=torch.float32, device=dev),
           torch.empty((S, 3), dtype=torch.float32, device=dev),
           torch.empty((S,), dtype=torch.int32, device=dev))
    plan, entry = autotune.tune_batch(b.requests, recs, ts, "fp32", out=out, reps=2)
    graph = BatchGraph(plan, recs, ts, "fp32", out=out)
    graph_out = out
    graph.replay(stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        host_lead(torch)
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay(stream)
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
    graph.close()
    med = statistics.median(ms)
    res = {"workload": "uneven-256-requests", "requests": len(reqs), "states": S,
           "value": S / (med * 1e-3), "unit": UNIT, "ms_per_launch": med,
           "tile_states": entry["tile_states"], "launches_per_step": 2,
           "note": "N_i log-U[100,5e4], T_i log-U[10,5e3], grids U[-720,2880] min; "
                   "one CUDA-graph replay (counter reset + persistent kernel)",
           "roofline": {"hbm": {"achieved": 28 * S / (med * 1e-3) / 1e9, "unit": "GB/s",
                                "bytes_per_state": 28}}}
    if sample_requests:
        # error against the oracle over each sampled request's whole grid, on up to 200
        # of its satellites (and every invalid record among them)
        import oracle
        rng = np.random.default_rng(4)
        r_all, v_all, s_all = graph_out
        el_s, st_ref, dr_all, dv_all = [], [], [], []
        mism = 0
        states_checked = 0
        for k in rng.choice(len(reqs), sample_requests, replace=False):
            sat0, n, t0, T, out0 = b.requests[k]
            pick = np.unique(np.concatenate([rng.choice(n, min(n, 200), replace=False),
                                             np.flatnonzero(reqs[k].elements[:, 1] >= 1.0)]))
            rr, vr, sr, _ = oracle.propagate(reqs[k].elements[pick], reqs[k].tsince,
                                             threads=threads)
            idx = torch.as_tensor((out0 + pick[:, None] * T + np.arange(T)[None, :]).reshape(-1),
                                  device=dev)
            rg = r_all[idx].double().cpu().numpy().reshape(len(pick), T, 3)
            vg = v_all[idx].double().cpu().numpy().reshape(len(pick), T, 3)
            sg = s_all[idx].cpu().numpy().reshape(len(pick), T)
            mism += int((sg != sr).sum())
            states_checked += sg.size
            keep = (sr == 0) | (sr == 6)
            dr_all.append(np.linalg.norm(rg[keep] - rr[keep], axis=-1))
            dv_all.append(np.linalg.norm(vg[keep] - vr[keep], axis=-1))
        dr = np.concatenate(dr_all)
        dv = np.concatenate(dv_all)
        res["vs_oracle"] = {"status_mismatches": mism, "states": states_checked,
                            "max_dr_km": float(dr.max()), "p99_dr_km": float(np.percentile(dr, 99)),
                            "median_dr_km": float(np.median(dr)), "max_dv_kms": float(dv.max()),
                            "p99_dv_kms": float(np.percentile(dv, 99))}
        res["error_sample"] = (f"{sample_requests} random requests, up to 200 satellites each "
                               f"(plus their invalid records), every time of their grids")
    del out, recs, el, ts
    torch.cuda.empty_cache()
    return res


def run_adjoint(torch, dev, stream, flush, steps, alu_peak, fp64_peak):
    """Adjoint and fitting workload (10,000 satellites x 500 times over one day): one
    sgp4_adjoint call (sweep kernel + init-Jacobian kernel) per step in FP32 and FP64,
    and one Levenberg-Marquardt step (sgp4_init + Jacobian + fit kernel)."""
    from paper_2603_27830_b300 import sgp4_adjoint, sgp4_init, sgp4_jacobian, sgp4_propagate
    from paper_2603_27830_b300 import workloads as W
    from paper_2603_27830_b300.fit import fit_step
    w = W.config5()
    states = w.n * w.t_count
    el = torch.as_tensor(w.elements, device=dev)
    ts = torch.as_tensor(w.tsince, device=dev)
    recs, _ = sgp4_init(el)
    truth, _ = sgp4_init(torch.as_tensor(w.meta["truth"], device=dev))
    r_true = sgp4_propagate(truth, ts, "fp64")[0]
    r_obs = r_true + torch.as_tensor(w.meta["noise"](tuple(r_true.shape)), device=dev)
    lam = torch.full((w.n,), 1e-3, dtype=torch.float64, device=dev)
    gen = torch.Generator(device=dev).manual_seed(0)
    g64 = torch.randn((w.n, w.t_count, 3), dtype=torch.float64, device=dev, generator=gen)
    sig = torch.tensor([1e-8, 1e-5, 1e-5, 1e-5, 1e-4, 1e-4, 1e-6], dtype=torch.float64,
                       device=dev)
    cov = torch.diag(sig * sig).expand(w.n, 7, 7).contiguous()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            host_lead(torch)
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            ms.append(a.elapsed_time(e))
        return statistics.median(ms)

    res = {"workload": w.name, "n_sats": w.n, "t_count": w.t_count}
    for prec, ops, peak, unit_kind in (("fp32", ALG_OPS_ADJ_FP32, alu_peak, "alu"),
                                       ("fp64", ALG_OPS_ADJ_FP64, fp64_peak, "fp64")):
        g = g64.float() if prec == "fp32" else g64
        ms = timed(lambda: sgp4_adjoint(el, recs, ts, g, g, prec))
        fit_ms = timed(lambda: fit_step(el, ts, r_obs, lam, prec))
        jac_ms = timed(lambda: sgp4_jacobian(el, recs, ts, prec, cov=cov))
        achieved = ops * states / (ms * 1e-3) / 1e9
        res[prec] = {"value": states / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms,
                     "roofline": {"bound": unit_kind, "achieved": achieved, "peak": peak,
                                  "unit": "Gop/s", "frac": achieved / peak,
                                  "ops_per_state": ops,
                                  "timed": "whole sgp4_adjoint call (sweep + init Jacobian)"},
                     "fit_step_ms": fit_ms, "fit_step_states_per_s": states / (fit_ms * 1e-3),
                     "jacobian_ms": jac_ms, "jacobian_states_per_s": states / (jac_ms * 1e-3),
                     "jacobian_note": "sgp4_jacobian: r, v, status, 6x7 J and 6x6 J C J^T "
                                      "per state"}
        jac_ops, fit_ops = ((ALG_OPS_JAC_FP64, ALG_OPS_FIT_FP64) if prec == "fp64"
                            else (ALG_OPS_JAC_FP32, ALG_OPS_FIT_FP32))
        for key, ops, ms_ in (("jacobian_roofline", jac_ops, jac_ms),
                              ("fit_step_roofline", fit_ops, fit_ms)):
            ach = ops * states / (ms_ * 1e-3) / 1e9
            res[prec][key] = {"bound": unit_kind, "achieved": ach, "peak": peak,
                              "unit": "Gop/s", "frac": ach / peak, "ops_per_state": ops,
                              "timed": "whole call (its small init and solve kernels "
                                       "included)"}
    del g64, r_obs, r_true, recs, truth, cov
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the headline workload
    (all 9,341 satellites x 1,000 times per step, or the first --ref-sats of them), on
    every host core.  Each step is one call of the oracle; the line's value is the
    states of all steps over their summed wall time."""
    import oracle
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2603_27830_b300 import workloads as W
    w = W.config2()
    threads = os.cpu_count() or 1
    n_sample = min(args.ref_sats, w.n)
    el = w.elements[:n_sample]
    oracle.load()
    for _ in range(args.warmup):
        oracle.propagate(el, w.tsince, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.propagate(el, w.tsince, threads=threads)
        times.append(time.perf_counter() - t0)
    states = n_sample * w.t_count
    value = states * args.steps / sum(times)
    sample = (f"all {w.n} satellites x {w.t_count} times per step" if n_sample == w.n else
              f"first {n_sample} of {w.n} satellites x {w.t_count} times per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n_sats": w.n, "t_count": w.t_count,
                   "precision": "fp64 (CPU oracle)"},
        "best_step_states_per_s": states / min(times),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2603_27830_b300 import sgp4_init, sgp4_propagate
    from paper_2603_27830_b300 import workloads as W

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_kind = _peaks()

    w = W.config2()
    n, T = w.n, w.t_count
    states = n * T
    el_h = torch.from_numpy(w.elements).pin_memory()
    ts_h = torch.from_numpy(w.tsince).pin_memory()
    el = el_h.to(dev)
    ts = ts_h.to(dev)
    recs, ist = sgp4_init(el)
    out32 = (torch.empty((n, T, 3), dtype=torch.float32, device=dev),
             torch.empty((n, T, 3), dtype=torch.float32, device=dev),
             torch.empty((n, T), dtype=torch.int32, device=dev))
    out64 = (torch.empty((n, T, 3), dtype=torch.float64, device=dev),
             torch.empty((n, T, 3), dtype=torch.float64, device=dev),
             torch.empty((n, T), dtype=torch.int32, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec, out):
        sgp4_init(el, records=recs, init_status=ist)
        sgp4_propagate(recs, ts, prec, out=out)

    def timed(prec, out, steps, warmup, kernel_only=False):
        for _ in range(warmup):   # the timed loop's own sequence, untimed
            host_lead(torch)
            flush.fill_(1.0)
            step(prec, out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        tot = 0.0
        per = []
        for _ in range(steps):
            host_lead(torch)
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            if kernel_only:
                sgp4_init(el, records=recs, init_status=ist)
                a.record(stream)
                sgp4_propagate(recs, ts, prec, out=out)
                b.record(stream)
            else:
                a.record(stream)
                step(prec, out)
                b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            per.append(ms)
            tot += ms
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return max_over_ranks(tot, dev), per

    # correctness spot check against the oracle (rank 0, before timing)
    max_dr_km = None
    if rank == 0:
        import oracle
        step("fp32", out32)
        torch.cuda.synchronize()
        k = 200
        rr, _, sr, _ = oracle.propagate(w.elements[:k], w.tsince)
        r32 = out32[0][:k].double().cpu().numpy()
        ok = sr == 0
        max_dr_km = float(np.linalg.norm(r32[ok] - rr[ok], axis=-1).max())

    props = torch.cuda.get_device_properties(dev)
    pci = None
    if hasattr(props, "pci_bus_id"):
        pci = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    with ClockSampler(pci, local) as clk:
        ms32, per32 = timed("fp32", out32, args.steps, args.warmup)
    clocks = clk.summary()
    ms32_k, per32_k = timed("fp32", out32, args.steps, 1, kernel_only=True)
    # the record build alone (the paper's JAX time included it; the headline step does)
    init_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        host_lead(torch)
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sgp4_init(el, records=recs, init_status=ist)
        b.record(stream)
        b.synchronize()
        init_ms.append(a.elapsed_time(b))
    ms64, _ = timed("fp64", out64, max(1, min(args.steps, 5)), 1)
    ms64_k, per64_k = timed("fp64", out64, max(1, min(args.steps, 5)), 1, kernel_only=True)

    value = job_rate(states, args.steps, world, ms32)
    fp64_value = job_rate(states, max(1, min(args.steps, 5)), world, ms64)

    # end to end through the public API with pinned host buffers
    r_h = torch.empty((n, T, 3), dtype=torch.float32).pin_memory()
    v_h = torch.empty((n, T, 3), dtype=torch.float32).pin_memory()
    s_h = torch.empty((n, T), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))

    def e2e_step():
        el_d = el_h.to(dev, non_blocking=True)
        ts_d = ts_h.to(dev, non_blocking=True)
        sgp4_init(el_d, records=recs, init_status=ist)
        sgp4_propagate(recs, ts_d, "fp32", out=out32)
        r_h.copy_(out32[0], non_blocking=True)
        v_h.copy_(out32[1], non_blocking=True)
        s_h.copy_(out32[2], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    b.synchronize()
    e2e_ms = a.elapsed_time(b)
    e2e_value = job_rate(states, e2e_steps, world, max_over_ranks(e2e_ms, dev))
    h2d = el_h.numel() * 8 + ts_h.numel() * 8
    d2h = (r_h.numel() + v_h.numel()) * 4 + s_h.numel() * 4

    # Roofline of the dominant kernel (the FP32 propagate), per launch.  It is bound by
    # FP32 arithmetic: ALG_OPS_FP32 operations per state (the formulation's FP32 and
    # SFU operations on this workload) against the FP32 lanes (148 SMs x 128 lanes x
    # SM clock).  Its HBM side (28 B per state of output) is reported beside it.
    kern_ms = statistics.mean(per32_k)
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e9          # Gop/s
    achieved_gops = ALG_OPS_FP32 * states / (kern_ms * 1e-3) / 1e9
    bytes_per_launch = BYTES_PER_STATE["fp32"] * states
    achieved_gbs = bytes_per_launch / (kern_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved_gops, "peak": alu_peak, "unit": "Gop/s",
                "frac": achieved_gops / alu_peak, "traffic": TRAFFIC_FP32_BYTES,
                "kernel": "propagate_kernel<fp32>", "kernel_ms": kern_ms,
                "timed": "the sgp4_propagate call: one launch of propagate_kernel<fp32>, whose "
                         "last blocks are the deep-space pass (no deep-space records here: "
                         "they read their flags)",
                "ops_per_state": ALG_OPS_FP32,
                "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
                "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved_gbs / peaks["hbm_gbs"], "peak_kind": peak_kind,
                        "bytes_per_state": BYTES_PER_STATE["fp32"]}}

    # The FP64 path is bound by B300's FP64 unit: ALG_OPS_FP64 operations per state
    # against 2 FP64 lanes per SM per clock.
    fp64_peak = n_sm * FP64_LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e9   # Gop/s
    kern64_ms = statistics.mean(per64_k)
    fp64_achieved = ALG_OPS_FP64 * states / (kern64_ms * 1e-3) / 1e9
    fp64_roofline = {"bound": "fp64", "achieved": fp64_achieved, "peak": fp64_peak,
                     "unit": "Gop/s", "frac": fp64_achieved / fp64_peak,
                     "kernel": "propagate_kernel<fp64>", "kernel_ms": kern64_ms,
                     "ops_per_state": ALG_OPS_FP64,
                     "peak_basis": f"{n_sm} SMs x {FP64_LANES_PER_SM_CLK} FP64 lanes x "
                                   f"{sm_mhz:.0f} MHz"}

    threads = os.cpu_count() or 1
    # Batched uneven requests: 256 requests, each with its own grid, in one persistent
    # launch replayed from a CUDA graph with the autotuned tile (FP32).
    batched = None
    if not args.no_batched:
        batched = run_batched(torch, dev, stream, flush, max(3, min(args.steps, 5)),
                              sample_requests=0 if args.no_configs else 16, threads=threads)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(torch, dev, stream, flush, max(3, min(args.steps, 5)), alu_peak,
                              fp64_peak)

    # Every workload: states/s of the step and of the launch in both precisions, the
    # launch's roofline, the error against the oracle over the whole horizon and the
    # oracle's own rate on the host cores.
    configs = None
    if rank == 0 and not args.no_configs:
        common = dict(threads=threads, alu_peak=alu_peak, fp64_peak=fp64_peak,
                      hbm_peak=peaks["hbm_gbs"], time_cpu=not args.no_cpu_baseline)
        cs = max(3, min(args.steps, 10))
        configs = {
            "1": run_single_config(torch, dev, stream, flush, cs, W.config1(), ("fp64", "fp32"),
                                   None, **common),
            "2": run_single_config(torch, dev, stream, flush, cs, W.config2(), ("fp32", "fp64"),
                                   None, **common),
            "3": run_single_config(torch, dev, stream, flush, cs, W.config3(), ("fp32", "fp64"),
                                   20_000, **common),
            "4": batched,
            "5": run_single_config(torch, dev, stream, flush, cs, W.config5(), ("fp32", "fp64"),
                                   None, **common),
            # deep space (SDP4), the branch the paper leaves for future work: FP64 states
            # in both precisions
            "deep": run_single_config(torch, dev, stream, flush, cs, W.deep_space(),
                                      ("fp64", "fp32"), 2_000, **common),
        }
        if adjoint is not None:
            configs["5"]["adjoint"] = "see the line's adjoint object (same workload)"

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, per_call, reps = time_oracle(w.elements, w.tsince, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"all {n} satellites x {T} times per call; best of 5 trials of "
                         f"{reps} call(s), {per_call:.2f} s per call on {threads} threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / PAPER_STATES_PER_S,
            "vs_baseline_basis": "the paper's 9,341 x 1,000 Starlink FP32 init + propagate in "
                                 "3.8 ms on one A100 (another GPU: context, not the target)",
            "dtype": "f32 (f64/double-float n*t phase)",
            "data": "synthetic",
            "config": {"workload": w.name, "n_sats": n, "t_count": T, "precision": "fp32",
                       "step": "sgp4_init + sgp4_propagate", "l2": "flushed between steps "
                       "(256 MB write)", "parallelism": f"replicas x{world}"},
            "fp32_max_dr_km_sample": max_dr_km,
            "init": {"ms": statistics.median(init_ms), "records": n,
                     "records_per_s": n / (statistics.median(init_ms) * 1e-3)},
            "propagate_fp32_kernel_ms": statistics.mean(per32_k),
            "step_ms": {"min": min(per32), "median": statistics.median(per32),
                        "max": max(per32)},
            "fp64": {"value": fp64_value, "unit": UNIT, "ms_per_step": ms64 / max(1, min(args.steps, 5)),
                     "kernel_ms": kern64_ms, "roofline": fp64_roofline},
            "roofline": roofline,
            "batched": batched,
            "adjoint": adjoint,
            "configs": configs,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per step: the record build and the FP32 propagation (whose launch also
            # carries the deep-space pass)
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-sats", type=int, default=9341)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
