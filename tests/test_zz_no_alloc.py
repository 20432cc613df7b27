"""The batched entry point for callers that cannot allocate device memory.

sgp4_propagate_batched_static takes no workspace: its scratch lives in a fixed
array inside the library.  This file is collected last on purpose.  The test calls
the entry point through the C ABI twice in a row, on two different batches, and
compares each result with the workspace-based sgp4_propagate_batched.  The second
call checks that nothing left in the shared array by the first call leaks into it.
Further cases: a table of exactly SGP4_STATIC_MAX_REQUESTS requests (every lane of
the on-device prefix sum in use, empty requests among them), and a page-locked
table that the caller overwrites as soon as the call returns, while the stream is
still busy with earlier work.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from gpu_util import FP64_TOL_R_KM, FP64_TOL_V_KMS

pytestmark = pytest.mark.gpu


def _batch(seed, n_req):
    from paper_2603_27830_b300 import make_batch
    from paper_2603_27830_b300 import workloads as W
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n_req):
        n = int(rng.integers(1, 400)) if k % 9 else 0
        T = int(rng.integers(1, 150))
        el = W.catalogue_elements(rng, max(n, 1), invalid_frac=0.02)[:n]
        probs.append((el, np.sort(rng.uniform(-720.0, 2880.0, T))))
    return make_batch(probs)


def _static_call(lib, b, recs, ts, precision, out, stream, tile=512, table_ptr=None):
    from paper_2603_27830_b300 import _lib
    n = len(b.requests)
    if table_ptr is None:
        table = (_lib.Sgp4Request * max(n, 1))()
        for k in range(n):
            table[k] = _lib.Sgp4Request(*[int(x) for x in b.requests[k]])
        table_ptr = ctypes.cast(table, ctypes.c_void_p)
    r, v, st = out
    return lib.sgp4_propagate_batched_static(
        table_ptr, n, tile, ctypes.byref(recs.c),
        ctypes.c_void_p(ts.data_ptr()), ts.numel(), _lib.SGP4_FP32 if precision == "fp32"
        else _lib.SGP4_FP64, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(v.data_ptr()),
        ctypes.c_void_p(st.data_ptr()), st.numel(), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_no_alloc_entry_matches_workspace_entry_twice(precision):
    import torch

    from paper_2603_27830_b300 import _lib, plan_batch, sgp4_init, sgp4_propagate_batched
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for seed, n_req in ((11, 40), (12, 90)):      # two calls in a row, different batches
        b = _batch(seed, n_req)
        el = torch.as_tensor(b.elements, device="cuda")
        ts = torch.as_tensor(b.tsince, device="cuda")
        recs, _ = sgp4_init(el)
        ref = sgp4_propagate_batched(plan_batch(b.requests, 1024), recs, ts, precision)
        dt = ref[0].dtype
        S = ref[2].numel()
        out = (torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
               torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
               torch.full((S,), 99, dtype=torch.int32, device="cuda"))
        assert _static_call(lib, b, recs, ts, precision, out, stream) == _lib.SGP4_OK
        torch.cuda.synchronize()
        assert torch.equal(out[2], ref[2])
        ok = (ref[2] == 0) | (ref[2] == 6)
        dr = (out[0][ok].double() - ref[0][ok].double()).norm(dim=-1)
        dv = (out[1][ok].double() - ref[1][ok].double()).norm(dim=-1)
        assert float(dr.max()) <= FP64_TOL_R_KM and float(dv.max()) <= FP64_TOL_V_KMS
        assert torch.all(torch.isnan(out[0][~ok]))


def test_no_alloc_entry_rejects_more_requests_than_its_scratch_holds():
    import torch

    from paper_2603_27830_b300 import _lib, sgp4_init
    lib = _lib.load()
    b = _batch(13, 3)
    recs, _ = sgp4_init(torch.as_tensor(b.elements, device="cuda"))
    n = _lib.STATIC_MAX_REQUESTS + 1
    table = (_lib.Sgp4Request * n)()
    code = lib.sgp4_propagate_batched_static(
        ctypes.cast(table, ctypes.c_void_p), n, 512, ctypes.byref(recs.c), None, 0,
        _lib.SGP4_FP32, None, None, None, 0, None)
    assert code == _lib.SGP4_ERR_OOM


def _compare(out, ref):
    import torch
    assert torch.equal(out[2], ref[2])
    ok = (ref[2] == 0) | (ref[2] == 6)
    dr = (out[0][ok].double() - ref[0][ok].double()).norm(dim=-1)
    dv = (out[1][ok].double() - ref[1][ok].double()).norm(dim=-1)
    if int(ok.sum()):
        assert float(dr.max()) <= FP64_TOL_R_KM and float(dv.max()) <= FP64_TOL_V_KMS
    assert torch.all(torch.isnan(out[0][~ok]))


def _fresh_out(ref):
    import torch
    S = ref[2].numel()
    dt = ref[0].dtype
    return (torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
            torch.full((S, 3), 555.0, dtype=dt, device="cuda"),
            torch.full((S,), 99, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_no_alloc_entry_at_its_request_limit(precision):
    """SGP4_STATIC_MAX_REQUESTS small requests, some with no satellites or no times:
    the one-block prefix sum then runs with every lane holding a request."""
    import torch

    from paper_2603_27830_b300 import _lib, make_batch, plan_batch, sgp4_init
    from paper_2603_27830_b300 import sgp4_propagate_batched
    from paper_2603_27830_b300 import workloads as W
    lib = _lib.load()
    rng = np.random.default_rng(21)
    probs = []
    for k in range(_lib.STATIC_MAX_REQUESTS):
        n = 0 if k % 13 == 0 else int(rng.integers(1, 12))
        T = 0 if k % 17 == 0 else int(rng.integers(1, 40))
        el = W.catalogue_elements(rng, max(n, 1), invalid_frac=0.02)[:n]
        probs.append((el, np.sort(rng.uniform(-720.0, 2880.0, T))))
    b = make_batch(probs)
    assert len(b.requests) == _lib.STATIC_MAX_REQUESTS
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    ref = sgp4_propagate_batched(plan_batch(b.requests, 128), recs, ts, precision)
    for tile in (128, 1024):
        out = _fresh_out(ref)
        assert _static_call(lib, b, recs, ts, precision, out, torch.cuda.current_stream(),
                            tile=tile) == _lib.SGP4_OK
        torch.cuda.synchronize()
        _compare(out, ref)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_no_alloc_entry_page_locked_table_reused_on_return(precision):
    """The caller rewrites its page-locked table right after the call, while the
    stream is still busy: the launch must still use the table it was given."""
    import torch

    from paper_2603_27830_b300 import _lib, plan_batch, sgp4_init, sgp4_propagate_batched
    lib = _lib.load()
    b = _batch(31, 60)
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    ref = sgp4_propagate_batched(plan_batch(b.requests, 512), recs, ts, precision)
    table = torch.as_tensor(np.asarray(b.requests, dtype=np.int64)).pin_memory()
    assert table.is_pinned() and table.shape[1] == 5
    out = _fresh_out(ref)
    torch.cuda.synchronize()
    torch.cuda._sleep(20_000_000)            # keep the stream busy (about 10 ms)
    code = _static_call(lib, b, recs, ts, precision, out, torch.cuda.current_stream(),
                        table_ptr=ctypes.c_void_p(table.data_ptr()))
    table.zero_()                            # every request now empty
    assert code == _lib.SGP4_OK
    torch.cuda.synchronize()
    _compare(out, ref)


def test_no_alloc_entry_refuses_stream_capture():
    """Under an active stream capture the entry point returns SGP4_ERR_ARG and enqueues
    nothing (its table copy reads a host array that a replay would read too late); the
    capture itself stays valid, and the same call outside it runs."""
    import torch

    from paper_2603_27830_b300 import _lib, plan_batch, sgp4_init, sgp4_propagate_batched
    lib = _lib.load()
    b = _batch(13, 30)
    el = torch.as_tensor(b.elements, device="cuda")
    ts = torch.as_tensor(b.tsince, device="cuda")
    recs, _ = sgp4_init(el)
    ref = sgp4_propagate_batched(plan_batch(b.requests, 512), recs, ts, "fp32")
    out = _fresh_out(ref)
    dummy = torch.zeros(4, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = _static_call(lib, b, recs, ts, "fp32", out, torch.cuda.current_stream())
        dummy.add_(1.0)                  # the capture holds some work of its own
    assert rc == _lib.SGP4_ERR_ARG
    g.replay()
    torch.cuda.synchronize()
    assert float(dummy.sum()) == 4.0     # the capture ended valid and replays
    assert bool((out[2] == 99).all())    # nothing of the refused call ran
    assert _static_call(lib, b, recs, ts, "fp32", out, torch.cuda.current_stream()) == _lib.SGP4_OK
    torch.cuda.synchronize()
    _compare(out, ref)
