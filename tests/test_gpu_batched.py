"""Batched persistent propagation: many uneven requests in one launch.

The batched kernel runs the same per-state code as sgp4_propagate: statuses equal
the per-request launches exactly and r, v to rounding (two kernels may be compiled
with different contractions), and its own outputs are bitwise independent of the
tile size; against the oracle the same bars hold as for single problems (status
bit-exact, FP64 within 1e-6 km)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import (FP32_TWO_DAY_KM, FP32_TWO_DAY_KMS, FP64_TOL_R_KM, ErrorStats,
                      assert_status_and_nan, device_state_errors, error_summary, state_errors)
from paper_2603_27830_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_batch(seed=0, n_req=30):
    from paper_2603_27830_b300 import make_batch
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n_req):
        n = int(rng.integers(0, 300)) if k % 7 else 0          # some empty requests
        T = int(rng.integers(0, 200)) if k % 11 else 0
        el = W.catalogue_elements(rng, max(n, 1), invalid_frac=0.03)[:n]
        probs.append((el, np.sort(rng.uniform(-720.0, 2880.0, T))))
    return make_batch(probs)


def _run_batched(b, precision, tile=1024, records=None):
    import torch

    from paper_2603_27830_b300 import plan_batch, sgp4_init, sgp4_propagate_batched
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs = records or sgp4_init(el)[0]
    plan = plan_batch(b.requests, tile)
    r, v, st = sgp4_propagate_batched(plan, recs, ts, precision)
    torch.cuda.synchronize()
    return r, v, st, recs


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_equals_per_request_launches(precision):
    import torch

    from paper_2603_27830_b300 import sgp4_init, sgp4_propagate
    b = _small_batch()
    r, v, st, _ = _run_batched(b, precision)
    for sat0, n, t0, T, out0 in b.requests:
        if n * T == 0:
            continue
        el = torch.as_tensor(b.elements[sat0:sat0 + n], device="cuda")
        ts = torch.as_tensor(b.tsince[t0:t0 + T], device="cuda")
        recs, _ = sgp4_init(el)
        r1, v1, s1 = sgp4_propagate(recs, ts, precision)
        sl = slice(out0, out0 + n * T)
        assert torch.equal(st[sl], s1.reshape(-1))
        # FP64: the same per-state code in two kernels (the compiler may contract
        # differently); FP32: both kernels run the same four-state units, but the Newton
        # step count is uniform over a warp and the warps cover different states in the
        # two launches, so they may differ by the FP32 path's rounding (metres; each is
        # within the FP32 bounds of the oracle tests)
        tol_r, tol_v = (1e-9, 1e-12) if precision == "fp64" else (0.02, 2e-5)
        dr = (r[sl] - r1.reshape(-1, 3)).nan_to_num(0.0).abs().max()
        dv = (v[sl] - v1.reshape(-1, 3)).nan_to_num(0.0).abs().max()
        assert float(dr) <= tol_r and float(dv) <= tol_v, (float(dr), float(dv))
        assert torch.equal(r[sl].isnan(), r1.reshape(-1, 3).isnan())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_against_oracle(precision):
    b = _small_batch(seed=1)
    r, v, st, _ = _run_batched(b, precision)
    r, v, st = r.double().cpu().numpy(), v.double().cpu().numpy(), st.cpu().numpy()
    for sat0, n, t0, T, out0 in b.requests:
        if n * T == 0:
            continue
        rr, vr, sr, _ = oracle.propagate(b.elements[sat0:sat0 + n], b.tsince[t0:t0 + T])
        sl = slice(out0, out0 + n * T)
        rg, vg, sg = r[sl].reshape(n, T, 3), v[sl].reshape(n, T, 3), st[sl].reshape(n, T)
        assert_status_and_nan(sg, sr, rg, vg)
        dr, dv = state_errors(rg, vg, rr, vr, sr)
        tol = FP64_TOL_R_KM if precision == "fp64" else FP32_TWO_DAY_KM
        if dr.size:
            assert dr.max() <= tol, error_summary(dr, dv)


def test_batched_guard_band_queue_overflow_fp32():
    """Requests whose every state is a guard-band state (inclination within 1e-5 rad
    of 180 degrees): tiles of 4,096 states overflow the block's 256-entry queue and are
    rescanned; tiles of 512 do not."""
    import math

    from paper_2603_27830_b300 import make_batch
    rng = np.random.default_rng(21)
    probs = []
    for k in range(6):
        n = int(rng.integers(50, 200))
        el = W.catalogue_elements(rng, n, invalid_frac=0.0)
        if k % 2 == 0:
            el[:, 2] = math.pi - 1e-5
            el[:, 1] = rng.uniform(0.03, 0.08, n)
        probs.append((el, np.sort(rng.uniform(-720.0, 2880.0, int(rng.integers(20, 120))))))
    b = make_batch(probs)
    for tile in (512, 4096):
        r, v, st, _ = _run_batched(b, "fp32", tile=tile)
        r, v, st = r.double().cpu().numpy(), v.double().cpu().numpy(), st.cpu().numpy()
        for sat0, n, t0, T, out0 in b.requests:
            rr, vr, sr, _ = oracle.propagate(b.elements[sat0:sat0 + n], b.tsince[t0:t0 + T])
            sl = slice(out0, out0 + n * T)
            rg, vg, sg = r[sl].reshape(n, T, 3), v[sl].reshape(n, T, 3), st[sl].reshape(n, T)
            assert_status_and_nan(sg, sr, rg, vg)
            dr, dv = state_errors(rg, vg, rr, vr, sr)
            if dr.size:
                assert dr.max() <= FP32_TWO_DAY_KM, error_summary(dr, dv)


def test_tile_size_does_not_change_results():
    import torch
    b = _small_batch(seed=2)
    ref = _run_batched(b, "fp32", tile=1024)
    for tile in (128, 384, 4096):
        out = _run_batched(b, "fp32", tile=tile, records=ref[3])
        for x, y in zip(out[:3], ref[:3]):
            assert torch.equal(x.nan_to_num(7.0), y.nan_to_num(7.0))


def test_reversed_outputs_with_gaps():
    """Outputs may be placed in any order with gaps: the gaps stay untouched."""
    import torch

    from paper_2603_27830_b300 import plan_batch, sgp4_init, sgp4_propagate_batched
    b = _small_batch(seed=3, n_req=8)
    req = b.requests.copy()
    off = 5
    for k in reversed(range(len(req))):
        req[k, 4] = off
        off += req[k, 1] * req[k, 3] + 3           # 3-state gap after each request
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    S = off
    r = torch.full((S, 3), 123.0, device="cuda")
    v = torch.full((S, 3), 123.0, device="cuda")
    st = torch.full((S,), 77, dtype=torch.int32, device="cuda")
    sgp4_propagate_batched(plan_batch(req, 256), recs, ts, "fp32", out=(r, v, st))
    ref_r, _, ref_st, _ = _run_batched(b, "fp32")
    written = torch.zeros(S, dtype=torch.bool, device="cuda")
    for (sat0, n, t0, T, o_new), o_ref in zip(req, b.requests[:, 4]):
        m = n * T
        written[o_new:o_new + m] = True
        assert torch.equal(st[o_new:o_new + m], ref_st[o_ref:o_ref + m])
        assert torch.equal(r[o_new:o_new + m].nan_to_num(7.0),
                           ref_r[o_ref:o_ref + m].nan_to_num(7.0))
    assert torch.all(st[~written] == 77) and torch.all(r[~written] == 123.0)


def test_graph_replay_equals_direct_launch():
    import torch

    from paper_2603_27830_b300 import BatchGraph, plan_batch, sgp4_init
    b = _small_batch(seed=4)
    ref = _run_batched(b, "fp32")
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    g = BatchGraph(plan_batch(b.requests, 1024), recs, ts, "fp32")
    for _ in range(2):
        for x in g.out:
            x.fill_(0)
        out = g.replay()
        torch.cuda.synchronize()
        for x, y in zip(out, ref[:3]):
            assert torch.equal(x.nan_to_num(7.0), y.nan_to_num(7.0))
    g.close()


def test_plan_init_page_locked_table_reused_on_return():
    """sgp4_batch_plan_init with a page-locked request table that the caller zeroes
    right after the call, while the stream is still busy: the plan keeps the table it
    was given (the call uploads its own checked copy)."""
    import ctypes

    import torch

    from paper_2603_27830_b300 import _lib, sgp4_init, sgp4_propagate_batched
    from paper_2603_27830_b300.api import BatchPlan
    b = _small_batch(seed=6, n_req=24)
    ref = _run_batched(b, "fp32", tile=512)
    lib = _lib.load()
    n = len(b.requests)
    table = torch.as_tensor(np.asarray(b.requests, dtype=np.int64)).pin_memory()
    nbytes = int(lib.sgp4_batch_workspace_bytes(n))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    plan = _lib.Sgp4BatchPlan()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    torch.cuda._sleep(20_000_000)             # keep the stream busy (about 10 ms)
    code = lib.sgp4_batch_plan_init(ctypes.c_void_p(table.data_ptr()), n, 512, 0,
                                    ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.byref(plan),
                                    ctypes.c_void_p(stream.cuda_stream))
    table.zero_()
    assert code == _lib.SGP4_OK
    r, v, st = sgp4_propagate_batched(BatchPlan(ws, plan, b.requests), ref[3],
                                      torch.as_tensor(b.tsince, device="cuda"), "fp32")
    torch.cuda.synchronize()
    for x, y in zip((r, v, st), ref[:3]):
        assert torch.equal(x.nan_to_num(7.0), y.nan_to_num(7.0))


def test_plan_larger_than_buffers_is_rejected():
    import torch

    from paper_2603_27830_b300 import _lib, plan_batch, sgp4_init, sgp4_propagate_batched
    b = _small_batch(seed=5, n_req=4)
    el = torch.as_tensor(b.elements[:-1], device="cuda")      # one satellite short
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    with pytest.raises(_lib.Sgp4Error) as ei:
        sgp4_propagate_batched(plan_batch(b.requests), recs, ts, "fp32")
    assert ei.value.code == _lib.SGP4_ERR_ARG


def test_uneven_requests_full_size_autotuned():
    """256 uneven requests (N log-U[100, 5e4], T log-U[10, 5e3], grids U[-720, 2880])
    in one autotuned persistent launch, FP32, against the oracle on every state of
    every request: statuses bit-exact, NaN where they say so, |dr| and |dv| within the
    two-day FP32 bound."""
    import json

    import torch

    from paper_2603_27830_b300 import autotune, make_batch, sgp4_init, sgp4_propagate_batched
    reqs = W.config4(seed=0)
    b = make_batch([(q.elements, q.tsince) for q in reqs])
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, ist = sgp4_init(el)
    S = int((b.requests[:, 1] * b.requests[:, 3]).sum())
    out = (torch.empty((S, 3), dtype=torch.float32, device="cuda"),
           torch.empty((S, 3), dtype=torch.float32, device="cuda"),
           torch.empty((S,), dtype=torch.int32, device="cuda"))
    plan, entry = autotune.tune_batch(b.requests, recs, ts, "fp32", out=out, reps=2,
                                      use_cache=False)
    r, v, st = sgp4_propagate_batched(plan, recs, ts, "fp32", out=out)
    torch.cuda.synchronize()
    ist_h = ist.cpu().numpy()
    stats = ErrorStats()
    checked = 0
    for k, (sat0, n, t0, T, out0) in enumerate(b.requests):
        if n * T == 0:
            continue
        step = max(1, 4_000_000 // T)                # satellites per oracle chunk
        for a in range(0, n, step):
            m = min(n, a + step) - a
            rr, vr, sr, isr = oracle.propagate(reqs[k].elements[a:a + m], reqs[k].tsince)
            np.testing.assert_array_equal(ist_h[sat0 + a:sat0 + a + m], isr)
            o = out0 + a * T
            dr, dv, keep = device_state_errors(r[o:o + m * T].view(m, T, 3),
                                               v[o:o + m * T].view(m, T, 3),
                                               st[o:o + m * T].view(m, T), rr, vr, sr)
            stats.add(dr[keep], dv[keep])
            checked += m * T
    assert checked == S
    summ = {"case": "uneven-256-requests-fp32", **stats.summary(),
            "tile_states": entry["tile_states"]}
    print(json.dumps(summ))
    assert summ["max_dr_km"] <= FP32_TWO_DAY_KM and summ["max_dv_kms"] <= FP32_TWO_DAY_KMS, summ
