"""Host-side checks of the comparison helpers the GPU parity tests use: the oracle's
measured sensitivity (the FP64 bar on ill-conditioned states), the chunked error
statistics and the status/NaN comparison (run here on CPU tensors)."""
from __future__ import annotations

import math

import numpy as np

import oracle
from gpu_util import (COND_FACTOR, ErrorStats, assert_fp64_within_conditioning,
                      device_state_errors, oracle_sensitivity)
from paper_2603_27830_b300 import workloads as W

# A catalogue draw with B* = 8.9e-3 1/ER: over seven days its mean semi-major axis, a
# polynomial in t, passes its minimum and grows to millions of km.
BLOWN_UP = [0.07054952869664177, 0.00010506273969093095, 1.1977967187328311,
            4.843513256596061, 5.020964099899104, 5.1917508134663395, 0.008859892401055782]


def test_sensitivity_is_tiny_on_ordinary_orbits_and_large_on_blown_up_ones():
    el = np.vstack([W.config2(seed=0, n=50).elements, [BLOWN_UP]])
    t = np.linspace(0.0, 10080.0, 100)
    sr, sv = oracle_sensitivity(el, t)
    assert sr[:50].max() < 1e-8 and sv[:50].max() < 1e-11
    r, _, st, _ = oracle.propagate(el[50:], t)
    far = np.linalg.norm(r[0], axis=-1) > 1e6
    assert far.any() and (st[0][far] == 0).all()
    assert sr[50][far].max() > 1e-4           # 16 ulps of one element move r by > 0.1 m


def test_conditioning_bar_accepts_rounding_sized_errors_and_rejects_larger_ones():
    el = np.array([BLOWN_UP])
    t = np.linspace(0.0, 10080.0, 100)
    r, v, st, _ = oracle.propagate(el, t)
    keep = (st == 0) | (st == 6)
    sr, sv = oracle_sensitivity(el, t)
    k = int(np.argmax(sr[0]))
    dr = np.zeros(st.shape)
    dv = np.zeros(st.shape)
    dr[0, k] = 0.5 * COND_FACTOR * sr[0, k]
    assert assert_fp64_within_conditioning(dr, dv, el, t, keep) == 1
    dr[0, k] = 2.0 * COND_FACTOR * sr[0, k]
    try:
        assert_fp64_within_conditioning(dr, dv, el, t, keep)
    except AssertionError:
        pass
    else:
        raise AssertionError("an error above the conditioning bar passed")
    # a well-conditioned state above the absolute bar fails
    el2 = W.config2(seed=0, n=3).elements
    t2 = np.linspace(0.0, 1440.0, 10)
    dr2 = np.zeros((3, 10))
    dr2[1, 4] = 2e-6
    try:
        assert_fp64_within_conditioning(dr2, np.zeros((3, 10)), el2, t2, np.ones((3, 10), bool))
    except AssertionError:
        pass
    else:
        raise AssertionError("2e-6 km on a well-conditioned state passed")


def test_error_stats_p99_and_max():
    rng = np.random.default_rng(0)
    x = 10.0 ** rng.uniform(-12, -1, 200_000)
    s = ErrorStats()
    for part in np.array_split(x, 7):
        s.add(part, part * 1e-3)
    out = s.summary()
    assert out["n"] == x.size and out["max_dr_km"] == x.max()
    p99 = np.percentile(x, 99)
    assert p99 <= out["p99_dr_km"] <= p99 * 1.03
    assert math.isclose(out["max_dv_kms"], x.max() * 1e-3)


def test_state_comparison_on_cpu_tensors():
    import torch
    el = np.vstack([W.config1().elements[:4], [[0.06, 1.5, 1.0, 0, 0, 0, 1e-4]]])
    t = np.linspace(0.0, 1440.0, 9)
    rr, vr, sr, _ = oracle.propagate(el, t)
    r = torch.as_tensor(rr).float()
    v = torch.as_tensor(vr).float()
    st = torch.as_tensor(sr)
    dr, dv, keep = device_state_errors(r, v, st, rr, vr, sr)
    assert keep[:4].all() and not keep[4].any()
    assert dr.max() < 1e-3 and dv.max() < 1e-6 and (dr[4] == 0).all()
    st_bad = st.clone()
    st_bad[1, 3] = 6
    try:
        device_state_errors(r, v, st_bad, rr, vr, sr)
    except AssertionError as exc:
        assert "1 status mismatches" in str(exc)
    else:
        raise AssertionError("a status mismatch passed")
