"""Helpers shared by the GPU tests: run the CUDA path and compare with the oracle."""
from __future__ import annotations

import numpy as np

FP64_TOL_R_KM = 1e-6
FP64_TOL_V_KMS = 1e-9


def gpu_propagate(elements, tsince, precision, fixups=False):
    import torch

    from paper_2603_27830_b300 import sgp4_init, sgp4_propagate
    el = torch.as_tensor(np.ascontiguousarray(elements, dtype=np.float64), device="cuda")
    ts = torch.as_tensor(np.ascontiguousarray(tsince, dtype=np.float64), device="cuda")
    recs, ist = sgp4_init(el)
    fx = torch.zeros(1, dtype=torch.int64, device="cuda") if fixups else None
    r, v, st = sgp4_propagate(recs, ts, precision, fixups=fx)
    torch.cuda.synchronize()
    out = (r.double().cpu().numpy(), v.double().cpu().numpy(), st.cpu().numpy(),
           ist.cpu().numpy())
    if fixups:
        return out + (int(fx.item()),)
    return out


def state_errors(r_gpu, v_gpu, r_ref, v_ref, st_ref):
    """|dr|, |dv| over states with finite reference output (codes 0 and 6)."""
    keep = (st_ref == 0) | (st_ref == 6)
    dr = np.linalg.norm(r_gpu[keep] - r_ref[keep], axis=-1)
    dv = np.linalg.norm(v_gpu[keep] - v_ref[keep], axis=-1)
    return dr, dv


def assert_status_and_nan(st_gpu, st_ref, r_gpu, v_gpu, ist_gpu=None, ist_ref=None):
    mism = np.argwhere(st_gpu != st_ref)
    assert mism.size == 0, (f"{len(mism)} status mismatches, first {mism[:5].tolist()}: "
                            f"gpu {st_gpu[tuple(mism[0])]} oracle {st_ref[tuple(mism[0])]}")
    if ist_gpu is not None:
        np.testing.assert_array_equal(ist_gpu, ist_ref)
    bad = (st_ref != 0) & (st_ref != 6)
    assert np.all(np.isnan(r_gpu[bad])) and np.all(np.isnan(v_gpu[bad]))
    good = ~bad
    assert np.all(np.isfinite(r_gpu[good])) and np.all(np.isfinite(v_gpu[good]))


def error_summary(dr, dv):
    if dr.size == 0:
        return {"n": 0}
    return {"n": int(dr.size), "max_dr_km": float(dr.max()),
            "p99_dr_km": float(np.percentile(dr, 99)), "median_dr_km": float(np.median(dr)),
            "max_dv_kms": float(dv.max()), "p99_dv_kms": float(np.percentile(dv, 99))}


def valid_codes_only(st) -> bool:
    """Every entry of a (possibly > 2^31-element) device status array is 0, 1, 2, 4 or 6."""
    import torch
    flat = st.reshape(-1)
    step = 1 << 28
    for k in range(0, flat.numel(), step):
        c = flat[k:k + step]
        ok = (c == 0) | (c == 1) | (c == 2) | (c == 4) | (c == 6)
        if not bool(torch.all(ok)):
            return False
    return True
