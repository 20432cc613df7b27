"""Element fitting with the adjoint (batch least squares, all satellites at once).

Observations are the oracle's positions of perturbed 'truth' elements (relative
N(0, 1e-4)) plus 0.01 km Gaussian noise per component; the fit starts from the
unperturbed elements and must bring the rms position residual to the noise level.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2603_27830_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(n, T, seed=0):
    import torch
    w = W.config5(seed=seed, n=n, t_count=T)
    truth = w.meta["truth"]
    r_true, _, st, _ = oracle.propagate(truth, w.tsince)
    r_obs = r_true + w.meta["noise"](r_true.shape)
    dev = "cuda"
    return (w, torch.as_tensor(w.elements, device=dev), torch.as_tensor(w.tsince, device=dev),
            torch.as_tensor(r_obs, device=dev), truth, st)


@pytest.mark.parametrize("precision,tol_km", [("fp64", 0.025), ("fp32", 0.04)])
def test_fit_recovers_elements(precision, tol_km):
    from paper_2603_27830_b300.fit import fit_elements
    w, start, ts, r_obs, truth, st = _setup(48, 120)
    res = fit_elements(start, ts, r_obs, precision, iters=8)
    rms = np.sqrt(res.sse.cpu().numpy() / w.t_count)
    assert res.history[0] > 10 * tol_km, res.history
    assert np.median(rms) < tol_km, res.history
    assert np.percentile(rms, 90) < 2 * tol_km, res.history
    el = res.elements.cpu().numpy()
    # mean motion, inclination and node are pinned down to well below the perturbation
    for k in (0, 2, 3):
        rel = np.abs(el[:, k] - truth[:, k]) / np.abs(truth[:, k] - w.elements[:, k]).clip(1e-30)
        assert np.median(rel) < 0.05, (k, np.median(rel))


def test_fit_full_size_10000x500():
    """The fitting workload at full size (10,000 satellites x 500 times), FP64."""
    from paper_2603_27830_b300.fit import fit_elements
    w, start, ts, r_obs, truth, st = _setup(10_000, 500)
    res = fit_elements(start, ts, r_obs, "fp64", iters=6)
    rms = np.sqrt(res.sse.cpu().numpy() / w.t_count)
    print("fit history (median rms km):", res.history)
    assert np.median(rms) < 0.025 and np.percentile(rms, 99) < 0.2, res.history
