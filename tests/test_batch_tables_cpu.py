"""Property tests of the request-table checks of the batched entry points (host code,
no GPU): every table that breaks a rule of the C ABI is rejected with SGP4_ERR_ARG
before any CUDA call, whatever else the table holds.  Tables the rules accept are not
passed here (they go on to upload to the device)."""
from __future__ import annotations

import ctypes

from hypothesis import given, settings, strategies as st

from paper_2603_27830_b300 import _lib

INT32_MAX = 2 ** 31 - 1
LIMIT = (2 ** 63 - 1) // 4

_value = st.one_of(st.integers(0, 50), st.integers(-3, -1), st.just(1 << 40),
                   st.just(INT32_MAX + 1), st.just(LIMIT))
_request = st.tuples(_value, _value, _value, _value, _value)


def _plan_rules_ok(rows):
    """The rules of sgp4_batch_plan_init (include/sgp4.h), restated."""
    total = 0
    spans = []
    for sat0, n, t0, T, out0 in rows:
        if min(sat0, n, t0, T, out0) < 0 or T > INT32_MAX:
            return False
        if sat0 > LIMIT - n or t0 > LIMIT - T:
            return False
        if n and T > (LIMIT // 3) // n:
            return False
        s = n * T
        if out0 > LIMIT // 3 - s:
            return False
        total += s
        if total > LIMIT:
            return False
        if s:
            spans.append((out0, out0 + s))
    spans.sort()
    return all(spans[k][0] >= spans[k - 1][1] for k in range(1, len(spans)))


def _static_rules_ok(rows, n_records, ts_len, out_len):
    """The rules of sgp4_propagate_batched_static: the plan's rules with the bounds of
    the caller's records, grid and outputs."""
    for sat0, n, t0, T, out0 in rows:
        if min(sat0, n, t0, T, out0) < 0 or T > INT32_MAX:
            return False
        if n and T > (LIMIT // 3) // n:
            return False
        s = n * T
        if sat0 > n_records - n or t0 > ts_len - T or out0 > out_len - s:
            return False
    spans = sorted((q[4], q[4] + q[1] * q[3]) for q in rows if q[1] * q[3] > 0)
    return all(spans[k][0] >= spans[k - 1][1] for k in range(1, len(spans)))


def _table(rows):
    return (_lib.Sgp4Request * max(len(rows), 1))(*[_lib.Sgp4Request(*r) for r in rows])


@settings(max_examples=400, deadline=None)
@given(st.lists(_request, min_size=1, max_size=6))
def test_plan_init_rejects_every_table_that_breaks_a_rule(rows):
    if _plan_rules_ok(rows):
        return
    lib = _lib.load()
    plan = _lib.Sgp4BatchPlan()
    nb = lib.sgp4_batch_workspace_bytes(len(rows))
    code = lib.sgp4_batch_plan_init(ctypes.cast(_table(rows), ctypes.c_void_p), len(rows), 512,
                                    0, ctypes.c_void_p(1 << 20), nb, ctypes.byref(plan), None)
    assert code == _lib.SGP4_ERR_ARG, rows


@settings(max_examples=400, deadline=None)
@given(st.lists(_request, min_size=1, max_size=6), st.integers(0, 120), st.integers(0, 120),
       st.integers(0, 3000))
def test_static_entry_rejects_every_table_that_breaks_a_rule(rows, n_records, ts_len, out_len):
    if _static_rules_ok(rows, n_records, ts_len, out_len):
        return
    lib = _lib.load()
    rec = _lib.Sgp4Records()
    assert lib.sgp4_records_bind(ctypes.c_void_p(1 << 20), lib.sgp4_records_bytes(n_records),
                                 n_records, None, ctypes.byref(rec)) == _lib.SGP4_OK
    P = ctypes.c_void_p
    code = lib.sgp4_propagate_batched_static(
        ctypes.cast(_table(rows), ctypes.c_void_p), len(rows), 512, ctypes.byref(rec),
        P(1 << 22), ts_len, _lib.SGP4_FP32, P(1 << 24), P(1 << 25), P(1 << 26), out_len, None)
    assert code == _lib.SGP4_ERR_ARG, (rows, n_records, ts_len, out_len)
