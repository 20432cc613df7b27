"""The batched entry point for callers that cannot allocate device memory.

sgp4_propagate_batched_static takes no workspace: its scratch lives in a fixed
array inside the library.  This file is collected last on purpose.  The test calls
the entry point through the C ABI twice in a row, on two different batches, and
compares each result with the workspace-based sgp4_propagate_batched.  The second
call checks that nothing left in the shared array by the first call leaks into it.
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


def _static_call(lib, b, recs, ts, precision, out, stream):
    from paper_2603_27830_b300 import _lib
    n = len(b.requests)
    table = (_lib.Sgp4Request * max(n, 1))()
    for k in range(n):
        table[k] = _lib.Sgp4Request(*[int(x) for x in b.requests[k]])
    r, v, st = out
    return lib.sgp4_propagate_batched_static(
        ctypes.cast(table, ctypes.c_void_p), n, 512, ctypes.byref(recs.c),
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
