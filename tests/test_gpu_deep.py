"""Deep-space (SDP4) states of the CUDA path against the FP64 oracle, through the C ABI.

Records with a period of 225 min or more take the deep-space branch: its record
constants must match the oracle's, every state's status bit for bit, FP64 states to
1e-6 km and 1e-9 km/s (or the oracle's own conditioning where that is larger), and
FP32 outputs (the deep-space states are computed in FP64 in both precisions) to the
float32 storage bar.  Single-problem, per-satellite-grid, absolute-time and batched
launches; mixed near-Earth and deep-space catalogues; the resonance's time limit;
code 3; and the differentiable entry points, which leave deep-space records out.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from gpu_util import (FP32_CATALOGUE_7D_KM, FP32_CATALOGUE_7D_KMS, FP32_STORE_REL,
                      FP64_TOL_R_KM, FP64_TOL_V_KMS, assert_fp64_within_conditioning,
                      device_state_errors, fp32_excess)
from paper_2603_27830_b300 import workloads as W

pytestmark = pytest.mark.gpu

REV = W.REV_PER_DAY
# Deep-space outputs of the FP32 path: FP64 states rounded to float32 (half an ulp of
# each component, ~6e-8 |r|), plus 1 mm for components near zero.
DEEP_FP32_ABS_KM = 1e-6
DEEP_FP32_ABS_KMS = 1e-9


def _records(el, day, frac):
    import torch

    from paper_2603_27830_b300 import sgp4_init
    return sgp4_init(torch.as_tensor(np.ascontiguousarray(el), device="cuda"),
                     epoch_day=torch.as_tensor(np.asarray(day, dtype=np.int32), device="cuda"),
                     epoch_frac=torch.as_tensor(np.asarray(frac, dtype=np.float64),
                                                device="cuda"))


def _propagate(el, t, day, frac, precision):
    import torch

    from paper_2603_27830_b300 import sgp4_propagate
    recs, ist = _records(el, day, frac)
    r, v, st = sgp4_propagate(recs, torch.as_tensor(np.ascontiguousarray(t), device="cuda"),
                              precision)
    torch.cuda.synchronize()
    return r, v, st, ist


def _compare(el, t, day, frac, precision, r, v, st, ist, near_bar=None):
    """Statuses bit for bit; FP64: the absolute bar or the oracle's conditioning; FP32:
    deep-space states within the storage bar, near-Earth ones within near_bar."""
    ep = (np.asarray(day, dtype=np.float64), np.asarray(frac))
    rr, vr, sr, isr = oracle.propagate(el, t, epoch=ep)
    np.testing.assert_array_equal(ist.cpu().numpy(), isr)
    dr, dv, keep, rn, vn = device_state_errors(r, v, st, rr, vr, sr, norms=True)
    deep = oracle.deep_records(el, epoch=ep)["deep"] >= 1
    if precision == "fp64":
        assert_fp64_within_conditioning(dr, dv, el, t, keep, epoch=ep)
        return dr, dv, keep, deep
    dk = keep & deep[:, None]
    bad_r = dk & (dr > DEEP_FP32_ABS_KM + FP32_STORE_REL * rn)
    bad_v = dk & (dv > DEEP_FP32_ABS_KMS + FP32_STORE_REL * vn)
    assert not bad_r.any() and not bad_v.any(), (float(dr[dk].max()), float(dv[dk].max()))
    if near_bar is not None:
        nk = keep & ~deep[:, None]
        n_bad, _ = fp32_excess(dr, dv, rn, vn, nk, *near_bar)
        assert n_bad == 0
    return dr, dv, keep, deep


# ------------------------------------------------------------------ record build
def test_deep_records_match_oracle():
    """The deep-space planes of the records (sidereal angle, lunar-solar rates and
    amplitudes, resonance terms) equal the oracle's to FP64 rounding."""
    wl = W.deep_space(seed=1, n=3000, t_count=2)
    el, day, frac = wl.elements, wl.meta["epoch_day"], wl.meta["epoch_frac"]
    recs, _ = _records(el, day, frac)
    import torch
    torch.cuda.synchronize()
    n = el.shape[0]
    stride = int(recs.c.stride)
    planes = recs.arena.cpu().numpy()[:82 * stride * 8].view(np.float64).reshape(82, stride)
    ref = oracle.deep_records(el, epoch=(day.astype(np.float64), frac))
    assert np.all(ref["deep"] >= 1)
    names = [k for k in oracle.DEEP_FIELDS if k != "irez"]
    for k, name in enumerate(names):
        got = planes[35 + k, :n]
        want = ref[name]
        if name in ("del1", "del2", "del3", "d2201", "d2211", "d3210", "d3222", "d4410",
                    "d4422", "d5220", "d5232", "d5421", "d5433", "lambda0", "xfact"):
            want = np.where(ref["irez"] > 0, want, 0.0)
        scale = np.abs(want).max() + 1e-300
        err = np.abs(got - want)
        if name in ("gsto", "lambda0", "sun_M0", "moon_M0"):
            # angles: the sidereal angle is a reduction of ~1e9 s of time (an ulp there
            # is 8.7e-12 rad), evaluated in another order by the record builder
            err = np.abs(np.remainder(got - want + math.pi, 2 * math.pi) - math.pi)
            scale = 50.0
        assert err.max() <= 1e-12 * scale, (name, float(err.max()), scale)


# ------------------------------------------------------------- single problem
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deep_space_catalogue_every_state(precision):
    """3,000 deep-space satellites (geosynchronous, Molniya, navigation, transfer and
    other orbits, own epochs) x 200 times over seven days, every state."""
    wl = W.deep_space(seed=2, n=3000, t_count=200)
    el, t, day, frac = wl.elements, wl.tsince, wl.meta["epoch_day"], wl.meta["epoch_frac"]
    r, v, st, ist = _propagate(el, t, day, frac, precision)
    _, _, keep, _ = _compare(el, t, day, frac, precision, r, v, st, ist)
    assert keep.mean() > 0.99


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_catalogue(precision):
    """Near-Earth and deep-space records interleaved in one record set: each class
    to its own bar, every status bit for bit (the propagation's blocks leave the
    deep-space states to the deep-space pass, the same launch's last blocks)."""
    rng = np.random.default_rng(7)
    near = W.catalogue_elements(rng, 4000)
    deep = W.deep_space_elements(rng, 1000)
    el = np.concatenate([near, deep])
    perm = rng.permutation(el.shape[0])
    el = el[perm]
    n = el.shape[0]
    day = rng.integers(2458000, 2462000, n).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, n)
    t = np.linspace(0.0, 10080.0, 64)
    r, v, st, ist = _propagate(el, t, day, frac, precision)
    _compare(el, t, day, frac, precision, r, v, st, ist,
             near_bar=(FP32_CATALOGUE_7D_KM, FP32_CATALOGUE_7D_KMS))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 5), (3, 1), (2500, 1), (40, 3000)])
def test_deep_pass_launch_shapes(precision, shape):
    """The deep-space pass at the launch shapes that size its share of the launch
    differently: one satellite, a few, many satellites at one time each (one grid part
    per work item), a long grid (many parts); deep-space and near-Earth records mixed."""
    n, T = shape
    rng = np.random.default_rng(100 + n)
    deep = W.deep_space_elements(rng, n)
    near = W.catalogue_elements(rng, n)
    pick = rng.random(n) < 0.5
    pick[0] = True                         # at least one deep-space record
    el = np.where(pick[:, None], deep, near)
    day = rng.integers(2458000, 2462000, n).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, n)
    t = np.sort(rng.uniform(-1440.0, 10080.0, T))
    r, v, st, ist = _propagate(el, t, day, frac, precision)
    _compare(el, t, day, frac, precision, r, v, st, ist,
             near_bar=(FP32_CATALOGUE_7D_KM, FP32_CATALOGUE_7D_KMS))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deep_per_satellite_grid_and_ragged(precision):
    """A grid per satellite (negative and positive times, T not a multiple of 4)."""
    rng = np.random.default_rng(8)
    el = W.deep_space_elements(rng, 301)
    day = rng.integers(2458000, 2462000, 301).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, 301)
    t = np.sort(rng.uniform(-4000.0, 12000.0, (301, 37)), axis=1)
    r, v, st, ist = _propagate(el, t, day, frac, precision)
    _compare(el, t, day, frac, precision, r, v, st, ist)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deep_absolute_times(precision):
    """sgp4_propagate_jd: each deep-space record from its own epoch to Julian dates."""
    import torch

    from paper_2603_27830_b300 import sgp4_propagate_jd
    rng = np.random.default_rng(9)
    el = W.deep_space_elements(rng, 500)
    day = rng.integers(2460000, 2460010, 500).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, 500)
    jd_day = np.repeat(np.arange(2460005, 2460015, dtype=np.int32), 4)
    jd_frac = np.tile(np.array([0.0, 0.25, 0.5, 0.875]), 10)
    recs, ist = _records(el, day, frac)
    r, v, st = sgp4_propagate_jd(recs, torch.as_tensor(jd_day, device="cuda"),
                                 torch.as_tensor(jd_frac, device="cuda"), precision)
    torch.cuda.synchronize()
    t = 1440.0 * ((jd_day[None, :] - day[:, None]).astype(np.float64) +
                  (jd_frac[None, :] - frac[:, None]))
    _compare(el, t, day, frac, precision, r, v, st, ist)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deep_batched(precision):
    """The persistent batched launch with deep-space and near-Earth requests (and a
    deep-space kernel after it, request by request)."""
    import torch

    from paper_2603_27830_b300 import make_batch, plan_batch, sgp4_init, sgp4_propagate_batched
    rng = np.random.default_rng(10)
    problems = []
    for k in range(6):
        el = (W.deep_space_elements(rng, 50 + 40 * k) if k % 2 == 0
              else W.catalogue_elements(rng, 60 + 30 * k))
        problems.append((el, np.sort(rng.uniform(-720.0, 4000.0, 20 + 7 * k))))
    batch = make_batch(problems)
    n = batch.elements.shape[0]
    # deep-space terms need an epoch: one per record
    day = rng.integers(2458000, 2462000, n).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, n)
    recs, _ = sgp4_init(torch.as_tensor(batch.elements, device="cuda"),
                        epoch_day=torch.as_tensor(day, device="cuda"),
                        epoch_frac=torch.as_tensor(frac, device="cuda"))
    plan = plan_batch(batch.requests, tile_states=512)
    r, v, st = sgp4_propagate_batched(plan, recs, torch.as_tensor(batch.tsince, device="cuda"),
                                      precision)
    torch.cuda.synchronize()
    r, v, st = r.double().cpu().numpy(), v.double().cpu().numpy(), st.cpu().numpy()
    for q, (el, t) in zip(batch.requests, problems):
        s0, m, T, o = int(q[0]), int(q[1]), int(q[3]), int(q[4])
        ep = (day[s0:s0 + m].astype(np.float64), frac[s0:s0 + m])
        rr, vr, sr, _ = oracle.propagate(el, t, epoch=ep)
        gs = st[o:o + m * T].reshape(m, T)
        np.testing.assert_array_equal(gs, sr)
        keep = (sr == 0) | (sr == 6)
        dr = np.linalg.norm(r[o:o + m * T].reshape(m, T, 3) - rr, axis=-1)[keep]
        rn = np.linalg.norm(rr, axis=-1)[keep]
        deep = oracle.deep_records(el, epoch=ep)["deep"] >= 1
        if deep.all():
            bar = (FP64_TOL_R_KM if precision == "fp64"
                   else DEEP_FP32_ABS_KM + FP32_STORE_REL * rn)
            assert np.all(dr <= bar), float(dr.max())
        elif precision == "fp64":
            assert np.all(dr <= FP64_TOL_R_KM), float(dr.max())


# --------------------------------------------------------------- limits, codes
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resonance_time_limit_and_code3(precision):
    """Resonant records integrate to |tsince| <= 1e7 min and give code 2 beyond; a
    low-perigee 232-min orbit whose drag drives e to its floor reaches code 3."""
    el = np.array([[1.00273 * REV, 0.001, 0.1, 1.0, 2.0, 3.0, 1e-5],     # one rev/day
                   [2.00561 * REV, 0.72, 1.107, 1.0, 4.7, 0.3, 1e-5],    # two rev/day
                   [6.2 * REV, 0.47, 0.5, 1.0, 2.0, 3.0, 1.0]])          # code 3
    day = np.array([2459000, 2459000, 2455000], dtype=np.int32)
    frac = np.array([0.3, 0.3, 0.3])
    span = np.linspace(0.0, 30.0 * 1440.0, 3001)    # code 3 lasts ~1.5 h of the 30 days
    far = np.array([-1.0e7, 1.0e7, -1.0000001e7, 1.0000001e7, 2.0e7])
    r, v, st, ist = _propagate(el, np.concatenate([span, far]), day, frac, precision)
    k = span.size
    _compare(el, span, day, frac, precision, r[:, :k], v[:, :k], st[:, :k], ist)
    # 1e7 min of resonance steps: statuses bit for bit (positions there carry the
    # rounding of 13,889 integration steps, beyond the FP64 bar)
    s = st.cpu().numpy()
    _, _, sr, _ = oracle.propagate(el, far, epoch=(day.astype(np.float64), frac))
    np.testing.assert_array_equal(s[:, k:], sr)
    assert np.all(s[:2, -3:] == 2) and np.all(s[:2, -5:-3] != 2)
    assert (s[2] == 3).any()


def test_differentiable_entry_points_leave_deep_records_out():
    """sgp4_jacobian gives deep-space records status 5 and NaN, sgp4_adjoint a zero
    gradient, sgp4_fit_step their elements unchanged with zero residual; the
    near-Earth records of the same set are unaffected."""
    import torch

    from paper_2603_27830_b300 import sgp4_adjoint, sgp4_init, sgp4_jacobian, sgp4_propagate
    from paper_2603_27830_b300 import fit as F
    el = np.array([[15.0 * REV, 0.001, 0.9, 0.2, 0.3, 0.4, 1e-4],
                   [1.00273 * REV, 0.001, 0.1, 1.0, 2.0, 3.0, 1e-5]])
    elt = torch.as_tensor(el, device="cuda")
    t = torch.linspace(0.0, 1440.0, 16, dtype=torch.float64, device="cuda")
    recs, _ = sgp4_init(elt)
    for precision in ("fp64", "fp32"):
        out = sgp4_jacobian(elt, recs, t, precision)
        st = out["status"].cpu().numpy()
        assert np.all(st[1] == 5) and np.all(st[0] == 0)
        assert torch.isnan(out["jac"][1]).all() and not torch.isnan(out["jac"][0]).any()
        r, v, _ = sgp4_propagate(recs, t, precision)
        g = sgp4_adjoint(elt, recs, t, torch.ones_like(r), None, precision)
        assert torch.all(g[1] == 0) and torch.any(g[0] != 0)
        r_obs = r.double() + 0.01
        el_out, sse = F.fit_step(elt, t, r_obs, torch.zeros(2, dtype=torch.float64,
                                                           device="cuda"), precision)
        assert torch.equal(el_out[1], elt[1]) and float(sse[1]) == 0.0
        assert float(sse[0]) > 0.0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_deep_graph_replay_and_no_alloc_entry(precision):
    """Batches holding deep-space records: a CUDA-graph replay of the batched launch
    (batched kernel + deep-space pass captured together) and the no-allocation entry
    point both equal the direct workspace launch, bit for bit."""
    import ctypes

    import torch

    from paper_2603_27830_b300 import (BatchGraph, _lib, make_batch, plan_batch, sgp4_init,
                                       sgp4_propagate_batched)
    rng = np.random.default_rng(12)
    problems = []
    for k in range(5):
        el = (W.deep_space_elements(rng, 30 + 20 * k) if k % 2 == 0
              else W.catalogue_elements(rng, 40 + 10 * k))
        problems.append((el, np.sort(rng.uniform(-720.0, 4000.0, 15 + 6 * k))))
    b = make_batch(problems)
    n = b.elements.shape[0]
    day = torch.as_tensor(rng.integers(2458000, 2462000, n).astype(np.int32), device="cuda")
    frac = torch.as_tensor(rng.uniform(0.0, 1.0, n), device="cuda")
    recs, _ = sgp4_init(torch.as_tensor(b.elements, device="cuda"), epoch_day=day,
                        epoch_frac=frac)
    ts = torch.as_tensor(b.tsince, device="cuda")
    ref = sgp4_propagate_batched(plan_batch(b.requests, 512), recs, ts, precision)
    torch.cuda.synchronize()
    assert bool((ref[2] != -1).all())   # every state written, none left marked

    g = BatchGraph(plan_batch(b.requests, 512), recs, ts, precision)
    for x in g.out:
        x.fill_(0)
    out = g.replay()
    torch.cuda.synchronize()
    for x, y in zip(out, ref[:3]):
        assert torch.equal(x.nan_to_num(7.0), y.nan_to_num(7.0))
    g.close()

    lib = _lib.load()
    nreq = len(b.requests)
    table = (_lib.Sgp4Request * nreq)()
    for k in range(nreq):
        table[k] = _lib.Sgp4Request(*[int(x) for x in b.requests[k]])
    S = ref[2].numel()
    dt = ref[0].dtype
    o = (torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
         torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
         torch.full((S,), 99, dtype=torch.int32, device="cuda"))
    stream = torch.cuda.current_stream()
    rc = lib.sgp4_propagate_batched_static(
        ctypes.cast(table, ctypes.c_void_p), nreq, 512, ctypes.byref(recs.c),
        ctypes.c_void_p(ts.data_ptr()), ts.numel(),
        _lib.SGP4_FP32 if precision == "fp32" else _lib.SGP4_FP64,
        ctypes.c_void_p(o[0].data_ptr()), ctypes.c_void_p(o[1].data_ptr()),
        ctypes.c_void_p(o[2].data_ptr()), S, ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.SGP4_OK
    torch.cuda.synchronize()
    for x, y in zip(o, ref[:3]):
        assert torch.equal(x.nan_to_num(7.0), y.nan_to_num(7.0))
