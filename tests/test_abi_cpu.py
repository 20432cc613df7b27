"""The C ABI library loads and exports every declared symbol; host-side argument
checks that return before any CUDA call (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_2603_27830_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sgp4_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declarations_match_binding_list():
    assert _declared_functions() == set(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version_and_constants():
    lib = _lib.load()
    assert lib.sgp4_version() >= 100
    c = lib.sgp4_wgs72()
    assert (c.mu_km3s2, c.radius_km, c.j2, c.j3, c.j4) == (
        398600.8, 6378.135, 0.001082616, -0.00000253881, -0.00000165597)


def test_records_bytes_and_bind_checks():
    lib = _lib.load()
    assert lib.sgp4_records_bytes(-1) == 0
    b1, b64, b65 = (lib.sgp4_records_bytes(k) for k in (1, 64, 65))
    assert b1 == b64 and b65 > b64 and b64 % 256 == 0
    rec = _lib.Sgp4Records()
    # n < 0, NULL arena, misaligned arena, too small an arena: all rejected on the host
    assert lib.sgp4_records_bind(None, 0, -1, None, ctypes.byref(rec)) == _lib.SGP4_ERR_ARG
    assert lib.sgp4_records_bind(None, 10 ** 6, 5, None, ctypes.byref(rec)) == _lib.SGP4_ERR_ARG
    assert lib.sgp4_records_bind(ctypes.c_void_p(4096 + 8), 10 ** 6, 5, None,
                                 ctypes.byref(rec)) == _lib.SGP4_ERR_ARG
    assert lib.sgp4_records_bind(ctypes.c_void_p(4096), 16, 5, None,
                                 ctypes.byref(rec)) == _lib.SGP4_ERR_OOM
    bad = _lib.Sgp4Consts(-1.0, 6378.0, 0, 0, 0)
    assert lib.sgp4_records_bind(ctypes.c_void_p(4096), 10 ** 6, 5, ctypes.byref(bad),
                                 ctypes.byref(rec)) == _lib.SGP4_ERR_ARG
    # a fake (never dereferenced) 256-aligned address binds: binding touches no memory
    assert lib.sgp4_records_bind(ctypes.c_void_p(1 << 20), lib.sgp4_records_bytes(5), 5, None,
                                 ctypes.byref(rec)) == _lib.SGP4_OK
    assert rec.n == 5 and rec.stride == 64 and rec.consts.j2 == 0.001082616


def test_propagate_rejects_bad_arguments_before_launch():
    lib = _lib.load()
    rec = _lib.Sgp4Records()
    assert lib.sgp4_records_bind(ctypes.c_void_p(1 << 20), lib.sgp4_records_bytes(5), 5, None,
                                 ctypes.byref(rec)) == _lib.SGP4_OK
    P = ctypes.c_void_p
    ok = P(1 << 24)
    args = dict(t=P(1 << 22), T=10, grid=0, prec=_lib.SGP4_FP32, r=ok, v=P(1 << 25), st=P(1 << 26))

    def call(**kw):
        a = {**args, **kw}
        return lib.sgp4_propagate(ctypes.byref(rec), a["t"], a["T"], a["grid"], a["prec"],
                                  a["r"], a["v"], a["st"], None, None)

    assert call(prec=7) == _lib.SGP4_ERR_ARG
    assert call(T=-1) == _lib.SGP4_ERR_ARG
    assert call(r=None) == _lib.SGP4_ERR_ARG
    assert call(t=None) == _lib.SGP4_ERR_ARG
    assert call(r=P((1 << 24) + 4)) == _lib.SGP4_ERR_ARG
    assert call(st=P((1 << 26) + 8)) == _lib.SGP4_ERR_ARG
    assert call(T=(1 << 62)) == _lib.SGP4_ERR_ARG
    # zero-sized work is a successful no-op
    assert call(T=0) == _lib.SGP4_OK
    # records whose stride does not match n are rejected
    bad = _lib.Sgp4Records(rec.arena, 5, 63, rec.consts)
    assert lib.sgp4_propagate(ctypes.byref(bad), args["t"], 10, 0, 1, ok, args["v"], args["st"],
                              None, None) == _lib.SGP4_ERR_ARG


def test_init_rejects_bad_arguments_before_launch():
    lib = _lib.load()
    rec = _lib.Sgp4Records()
    lib.sgp4_records_bind(ctypes.c_void_p(1 << 20), lib.sgp4_records_bytes(5), 5, None,
                          ctypes.byref(rec))
    P = ctypes.c_void_p
    assert lib.sgp4_init(None, None, None, 5, ctypes.byref(rec), P(1 << 22), None) == _lib.SGP4_ERR_ARG
    assert lib.sgp4_init(P(1 << 21), None, None, 4, ctypes.byref(rec), P(1 << 22), None) == _lib.SGP4_ERR_ARG
    assert lib.sgp4_init(P((1 << 21) + 4), None, None, 5, ctypes.byref(rec), P(1 << 22),
                         None) == _lib.SGP4_ERR_ARG


def test_python_api_refuses_cpu_tensors():
    import torch

    from paper_2603_27830_b300 import sgp4_init
    with pytest.raises(ValueError, match="CUDA"):
        sgp4_init(torch.zeros((3, 7), dtype=torch.float64))


def test_batch_plan_rejects_bad_tables_before_any_copy():
    lib = _lib.load()
    assert lib.sgp4_batch_workspace_bytes(-1) == 0
    assert lib.sgp4_batch_workspace_bytes(3) >= 256 + 3 * 40
    plan = _lib.Sgp4BatchPlan()
    ws = ctypes.c_void_p(1 << 20)
    nb = lib.sgp4_batch_workspace_bytes(2)

    def call(rows, tile=1024, grid=0, nbytes=None):
        table = (_lib.Sgp4Request * len(rows))(*[_lib.Sgp4Request(*r) for r in rows])
        return lib.sgp4_batch_plan_init(ctypes.cast(table, ctypes.c_void_p), len(rows), tile,
                                        grid, ws, nb if nbytes is None else nbytes,
                                        ctypes.byref(plan), None)

    ok = [(0, 10, 0, 5, 0), (10, 4, 5, 3, 50)]
    assert call(ok, tile=100) == _lib.SGP4_ERR_ARG          # not a multiple of 128
    assert call(ok, tile=0) == _lib.SGP4_ERR_ARG
    assert call(ok, grid=-1) == _lib.SGP4_ERR_ARG
    assert call(ok, nbytes=16) == _lib.SGP4_ERR_OOM
    assert call([(0, -1, 0, 5, 0), ok[1]]) == _lib.SGP4_ERR_ARG
    assert call([(0, 10, 0, 5, 0), (10, 4, 5, 3, 49)]) == _lib.SGP4_ERR_ARG   # outputs overlap
    assert call([(0, 1 << 40, 0, 1 << 40, 0), ok[1]]) == _lib.SGP4_ERR_ARG    # overflow
    assert lib.sgp4_batch_plan_init(None, 0, 1024, 0, None, 0, ctypes.byref(plan), None) == 0
    assert plan.n_requests == 0 and plan.total_tiles == 0


def test_static_batch_rejects_bad_tables_before_any_cuda_call():
    lib = _lib.load()
    rec = _lib.Sgp4Records()
    assert lib.sgp4_records_bind(ctypes.c_void_p(1 << 20), lib.sgp4_records_bytes(20), 20, None,
                                 ctypes.byref(rec)) == _lib.SGP4_OK
    P = ctypes.c_void_p

    def call(rows, tile=512, ts_len=100, out_len=1000, prec=_lib.SGP4_FP32):
        n = len(rows)
        table = (_lib.Sgp4Request * max(n, 1))(*[_lib.Sgp4Request(*r) for r in rows])
        return lib.sgp4_propagate_batched_static(
            ctypes.cast(table, ctypes.c_void_p), n, tile, ctypes.byref(rec), P(1 << 22), ts_len,
            prec, P(1 << 24), P(1 << 25), P(1 << 26), out_len, None)

    ok = [(0, 10, 0, 5, 0), (10, 4, 5, 3, 50)]
    assert call(ok, ts_len=-1) == _lib.SGP4_ERR_ARG
    assert call(ok, out_len=-1) == _lib.SGP4_ERR_ARG
    assert call(ok, ts_len=-(1 << 62)) == _lib.SGP4_ERR_ARG
    assert call(ok, tile=100) == _lib.SGP4_ERR_ARG
    assert call(ok, prec=9) == _lib.SGP4_ERR_ARG
    assert call([(0, 10, 0, 5, 0), (10, 4, 5, 3, 49)]) == _lib.SGP4_ERR_ARG   # outputs overlap
    assert call([(15, 10, 0, 5, 0)]) == _lib.SGP4_ERR_ARG                     # past the records
    assert call([(0, 10, 96, 5, 0)]) == _lib.SGP4_ERR_ARG                     # past tsince
    assert call([(0, 10, 0, 5, 960)]) == _lib.SGP4_ERR_ARG                    # past the outputs
    assert call([(0, 1 << 40, 0, 1 << 40, 0)]) == _lib.SGP4_ERR_ARG           # overflow
    assert call([(0, 0, 0, 0, 0)] * (_lib.STATIC_MAX_REQUESTS + 1)) == _lib.SGP4_ERR_OOM
    assert call([]) == _lib.SGP4_OK                                            # nothing to do
