"""Per-state Jacobians and covariance propagation vs the oracle's forward-mode (dual
number) derivatives of its FP64 propagation."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import FP64_TOL_R_KM, assert_status_and_nan, state_errors
from paper_2603_27830_b300 import workloads as W

pytestmark = pytest.mark.gpu

# (relative, floor as a fraction of the entry's largest magnitude over the states)
TOL = {"fp64": (1e-7, 1e-9), "fp32": (5e-3, 2e-4)}


def _cases():
    rng = np.random.default_rng(41)
    near = W.config1(seed=6, n=40, t_count=50)
    cat = W.config3(seed=8, n=120, t_count=30)
    return [("near-earth", near.elements, near.tsince),
            ("catalogue-7d", cat.elements, cat.tsince),
            ("per-sat-grid", near.elements[:16],
             np.sort(rng.uniform(-500, 2000, (16, 21)), axis=1))]


def _covariances(n, rng):
    sig = np.array([1e-8, 1e-5, 1e-5, 1e-5, 1e-4, 1e-4, 1e-6])
    A = rng.normal(size=(n, 7, 7))
    R = A @ A.transpose(0, 2, 1) + 7 * np.eye(7)
    d = np.sqrt(np.einsum("nii->ni", R))
    R = R / d[:, :, None] / d[:, None, :]
    return R * sig[None, :, None] * sig[None, None, :]


def _run(el, t, prec, cov):
    import torch

    from paper_2603_27830_b300 import sgp4_init, sgp4_jacobian
    e = torch.as_tensor(el, device="cuda")
    recs, ist = sgp4_init(e)
    out = sgp4_jacobian(e, recs, torch.as_tensor(t, device="cuda"), prec,
                        cov=torch.as_tensor(cov, device="cuda"))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, ist.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(3))
def test_jacobian_and_covariance_match_the_oracle(case, prec):
    name, el, t = _cases()[case]
    rng = np.random.default_rng(case)
    cov = _covariances(len(el), rng)
    out, ist = _run(el, t, prec, cov)
    dr, dv, sj = oracle.jacobian(el, t)
    rr, vr, sr, isr = oracle.propagate(el, t)
    np.testing.assert_array_equal(sj, sr)
    r, v, st = out["r"].astype(np.float64), out["v"].astype(np.float64), out["status"]
    assert_status_and_nan(st, sr, r, v, ist, isr)
    ok = (sr == 0) | (sr == 6)
    if prec == "fp64":
        e_r, e_v = state_errors(r, v, rr, vr, sr)
        assert e_r.max() <= FP64_TOL_R_KM
    J = out["jac"].astype(np.float64)
    assert np.all(np.isnan(J[~ok])) and np.all(np.isfinite(J[ok]))
    Jref = np.concatenate([dr, dv], axis=2)                  # [n, T, 6, 7]
    rel, floor = TOL[prec]
    scale = np.abs(np.where(ok[..., None, None], Jref, 0.0)).max(axis=1, keepdims=True)
    bad = ok[..., None, None] & (np.abs(J - Jref) > rel * np.abs(Jref) + floor * scale)
    assert not bad.any(), f"{bad.sum()} Jacobian entries off ({name}, {prec})"
    # covariance: P = J C J^T against the oracle's J, relative to sqrt(P_pp P_qq)
    Pref = np.einsum("ntpk,nkl,ntql->ntpq", Jref, cov, Jref)
    iu = np.triu_indices(6)
    P = out["cov"].astype(np.float64)
    dref = np.sqrt(np.einsum("ntpp->ntp", Pref))
    norm = dref[..., iu[0]] * dref[..., iu[1]]
    err = np.abs(P - Pref[..., iu[0], iu[1]]) / np.maximum(norm, 1e-300)
    tol = 1e-6 if prec == "fp64" else 2e-2
    assert np.all(err[ok] <= tol), (name, prec, float(np.max(err[ok])))
    assert np.all(np.isnan(P[~ok]))


@pytest.mark.parametrize("T", [100, 400])
def test_jacobian_fp32_guard_band_states(T):
    """Inclinations within 1e-5 rad of 180 degrees: most FP32 states are guard-band
    states, done through the FP64 sweeps.  The i0 column is left out (and given no
    variance): d/di0 of 1 / (1 + cos i0) is not resolved by the FP32 record build's dual
    numbers this close to the pole."""
    import math
    rng = np.random.default_rng(50 + T)
    n = 16
    el = np.column_stack([rng.uniform(14.0, 15.5, n) * W.REV_PER_DAY,
                          rng.uniform(0.03, 0.08, n), np.full(n, math.pi - 1e-5),
                          rng.uniform(0, 2 * math.pi, (n, 3)), rng.uniform(1e-5, 1e-4, n)])
    t = np.linspace(0.0, 1440.0, T)
    cov = _covariances(n, rng)
    cov[:, 2, :] = 0.0
    cov[:, :, 2] = 0.0
    out, ist = _run(el, t, "fp32", cov)
    dr, dv, sj = oracle.jacobian(el, t)
    rr, vr, sr, isr = oracle.propagate(el, t)
    r, v, st = out["r"].astype(np.float64), out["v"].astype(np.float64), out["status"]
    assert_status_and_nan(st, sr, r, v, ist, isr)
    e_r, _ = state_errors(r, v, rr, vr, sr)
    assert e_r.max() <= 1.0
    ok = (sr == 0) | (sr == 6)
    cols = [0, 1, 3, 4, 5, 6]
    J = out["jac"].astype(np.float64)[..., cols]
    Jref = np.concatenate([dr, dv], axis=2)[..., cols]
    rel, floor = TOL["fp32"]
    scale = np.abs(np.where(ok[..., None, None], Jref, 0.0)).max(axis=1, keepdims=True)
    bad = ok[..., None, None] & (np.abs(J - Jref) > rel * np.abs(Jref) + floor * scale)
    assert not bad.any(), f"{bad.sum()} Jacobian entries off"
    Jfull = np.concatenate([dr, dv], axis=2)
    Pref = np.einsum("ntpk,nkl,ntql->ntpq", Jfull, cov, Jfull)
    iu = np.triu_indices(6)
    P = out["cov"].astype(np.float64)
    dref = np.sqrt(np.einsum("ntpp->ntp", Pref))
    err = np.abs(P - Pref[..., iu[0], iu[1]]) / np.maximum(dref[..., iu[0]] * dref[..., iu[1]],
                                                          1e-300)
    assert np.all(err[ok] <= 2e-2), float(np.max(err[ok]))


def test_jacobian_column_for_mean_anomaly_is_the_velocity_direction():
    """d r / d M0 at t = 0 with drag off is the velocity over the mean motion for a
    circular orbit (moving the satellite along its track), a check independent of the
    oracle's derivative machinery."""
    import math
    el = np.array([[15.1 * W.REV_PER_DAY, 1e-6, math.radians(53.0), 0.3, 0.0, 0.7, 0.0]])
    t = np.array([0.0])
    out, _ = _run(el, t, "fp64", _covariances(1, np.random.default_rng(0)))
    dr_dM = out["jac"][0, 0, :3, 5]
    v = out["v"][0, 0]
    # for a circular orbit r(M) moves along v with |dr/dM| = |r| (km per rad)
    r = out["r"][0, 0]
    cosang = dr_dM @ v / (np.linalg.norm(dr_dM) * np.linalg.norm(v))
    assert cosang == pytest.approx(1.0, abs=1e-3)
    assert np.linalg.norm(dr_dM) == pytest.approx(np.linalg.norm(r), rel=2e-3)
