"""Adjoint kernel vs the oracle: the oracle's forward-mode (dual number) Jacobian
contracted with the same upstream gradients, and central finite differences of the
plain FP64 oracle."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2603_27830_b300 import workloads as W

pytestmark = pytest.mark.gpu

REV = W.REV_PER_DAY


def _gpu_adjoint(el, t, gr, gv, precision):
    import torch

    from paper_2603_27830_b300 import sgp4_adjoint, sgp4_init
    dt = torch.float32 if precision == "fp32" else torch.float64
    e = torch.as_tensor(el, device="cuda")
    ts = torch.as_tensor(t, device="cuda")
    recs, _ = sgp4_init(e)
    g = sgp4_adjoint(e, recs, ts, torch.as_tensor(gr, device="cuda").to(dt),
                     torch.as_tensor(gv, device="cuda").to(dt), precision)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def _oracle_vjp(el, t, gr, gv):
    dr, dv, st = oracle.jacobian(el, t)
    keep = ((st == 0) | (st == 6))[..., None, None]
    dr = np.where(keep, dr, 0.0)
    dv = np.where(keep, dv, 0.0)
    return np.einsum("ntck,ntc->nk", dr, gr) + np.einsum("ntck,ntc->nk", dv, gv)


def _compare(g, ref, rel, floor):
    scale = np.abs(ref).max(axis=0, keepdims=True)
    tol = rel * np.abs(ref) + floor * scale
    bad = np.abs(g - ref) > tol
    assert not bad.any(), (f"{bad.sum()} entries off; worst rel "
                           f"{np.max(np.abs(g - ref) / (np.abs(ref) + 1e-300))}")


def _cases():
    rng = np.random.default_rng(21)
    near = W.config1(seed=3, n=48, t_count=60)
    cat = W.config3(seed=5, n=200, t_count=40)
    return [("near-earth", near.elements, near.tsince),
            ("catalogue-7d", cat.elements, cat.tsince),
            ("per-sat-grid", near.elements[:20],
             np.sort(rng.uniform(-500, 2000, (20, 33)), axis=1))]


@pytest.mark.parametrize("case", range(3))
def test_adjoint_fp64_matches_oracle_jacobian(case):
    name, el, t = _cases()[case]
    rng = np.random.default_rng(case)
    T = t.shape[-1]
    gr = rng.normal(size=(len(el), T, 3))
    gv = rng.normal(size=(len(el), T, 3)) * 100.0
    g = _gpu_adjoint(el, t, gr, gv, "fp64")
    ref = _oracle_vjp(el, t, gr, gv)
    _compare(g, ref, 1e-7, 1e-9)


@pytest.mark.parametrize("case", range(3))
def test_adjoint_fp32_matches_oracle_jacobian(case):
    name, el, t = _cases()[case]
    rng = np.random.default_rng(10 + case)
    T = t.shape[-1]
    gr = rng.normal(size=(len(el), T, 3))
    gv = rng.normal(size=(len(el), T, 3)) * 100.0
    g = _gpu_adjoint(el, t, gr, gv, "fp32")
    ref = _oracle_vjp(el, t, gr, gv)
    _compare(g, ref, 5e-3, 2e-4)


def test_adjoint_fp32_odd_grid_and_mixed_pairs():
    """The FP32 sweep takes two consecutive times per thread: an odd time count leaves
    the last pair one state short, and a pair with one usable state and one that is not
    (here, orbits that decay within the two-day grid: codes 1 and 6 among the states) is
    swept state by state after the loop.  37 shared times, against the oracle."""
    rng = np.random.default_rng(44)
    n = 24
    el = np.column_stack([rng.uniform(15.8, 16.4, n) * REV, rng.uniform(0.0005, 0.01, n),
                          rng.uniform(0.5, 1.5, n), rng.uniform(0, 2 * math.pi, (n, 3)),
                          rng.uniform(0.002, 0.05, n)])
    t = np.linspace(0.0, 2880.0, 37)
    _, _, st, _ = oracle.propagate(el, t)
    ok = (st == 0) | (st == 6)
    assert (ok[:, 0:36:2] != ok[:, 1:37:2]).sum() >= 5     # pairs with one usable state
    assert (~ok).any() and (st == 6).any()
    gr = rng.normal(size=(n, t.size, 3))
    gv = rng.normal(size=(n, t.size, 3)) * 100.0
    g = _gpu_adjoint(el, t, gr, gv, "fp32")
    ref = _oracle_vjp(el, t, gr, gv)
    _compare(g, ref, 5e-3, 2e-4)


@pytest.mark.parametrize("T", [100, 400])
def test_adjoint_fp32_guard_band_states(T):
    """Inclinations within 1e-5 rad of 180 degrees make most FP32 states guard-band
    states, swept in FP64 after the block's loop: from its queue (T = 100) or, past the
    queue's 256 entries, by finding them again (T = 400); against the oracle.  The i0
    column is left out: its terms in d/di0 of 1 / (1 + cos i0) are not resolved by the
    FP32 record build's dual numbers this close to the pole (1 + cos i0 rounds to 0 in
    FP32), which is a property of the FP32 path, not of the sweeps tested here."""
    rng = np.random.default_rng(30 + T)
    n = 24
    el = np.column_stack([rng.uniform(14.0, 15.5, n) * REV, rng.uniform(0.03, 0.08, n),
                          np.full(n, math.pi - 1e-5), rng.uniform(0, 2 * math.pi, (n, 3)),
                          rng.uniform(1e-5, 1e-4, n)])
    t = np.linspace(0.0, 1440.0, T)
    gr = rng.normal(size=(n, T, 3))
    gv = rng.normal(size=(n, T, 3)) * 100.0
    g = _gpu_adjoint(el, t, gr, gv, "fp32")
    ref = _oracle_vjp(el, t, gr, gv)
    cols = [0, 1, 3, 4, 5, 6]
    _compare(g[:, cols], ref[:, cols], 5e-3, 2e-4)


def test_adjoint_fp64_matches_central_differences():
    """Scalar loss sum(w . r) on a few satellites: adjoint vs central differences of
    the plain oracle (no dual numbers involved)."""
    el = np.array([[15.2 * REV, 0.002, math.radians(53.0), 0.4, 1.3, 2.2, 2e-4],
                   [13.8 * REV, 0.03, math.radians(97.6), 3.4, 0.3, 5.2, 5e-5],
                   [16.1 * REV, 0.001, math.radians(30.0), 1.4, 2.3, 0.2, 1e-3]])
    t = np.linspace(0.0, 1440.0, 25)
    rng = np.random.default_rng(3)
    w = rng.normal(size=(3, 25, 3))
    g = _gpu_adjoint(el, t, w, np.zeros_like(w), "fp64")
    steps = np.array([1e-9, 1e-7, 1e-7, 1e-7, 1e-7, 1e-7, 1e-8])
    for k in range(7):
        ep, em = el.copy(), el.copy()
        ep[:, k] += steps[k]
        em[:, k] -= steps[k]
        rp, _, _, _ = oracle.propagate(ep, t)
        rm, _, _, _ = oracle.propagate(em, t)
        fd = ((rp - rm) * w).sum(axis=(1, 2)) / (2 * steps[k])
        assert np.allclose(g[:, k], fd, rtol=2e-5, atol=1e-6 * np.abs(fd).max()), (k, g[:, k], fd)


def test_autograd_function_backward_is_the_adjoint():
    import torch

    from paper_2603_27830_b300 import sgp4_differentiable
    w = W.config1(seed=4, n=16, t_count=30)
    el = torch.as_tensor(w.elements, device="cuda").requires_grad_(True)
    ts = torch.as_tensor(w.tsince, device="cuda")
    r, v, st = sgp4_differentiable(el, ts, "fp64")
    rng = np.random.default_rng(0)
    wr = torch.as_tensor(rng.normal(size=r.shape), device="cuda")
    loss = (wr * r).sum() + (v * v).sum()
    (g,) = torch.autograd.grad(loss, el)
    ref = _oracle_vjp(w.elements, w.tsince, wr.cpu().numpy(), 2 * v.detach().cpu().numpy())
    _compare(g.cpu().numpy(), ref, 1e-7, 1e-9)


def test_unusable_records_get_zero_gradient():
    el = np.array([[15.0 * REV, 1.2, 0.9, 0, 0, 0, 1e-4],
                   [-0.01, 0.01, 0.9, 0, 0, 0, 1e-4],
                   [15.0 * REV, 0.01, 0.9, 0, 0, 0, 1e-4]])
    t = np.linspace(0, 100, 5)
    g = _gpu_adjoint(el, t, np.ones((3, 5, 3)), np.ones((3, 5, 3)), "fp64")
    assert np.all(g[:2] == 0.0) and np.all(np.isfinite(g[2])) and np.any(g[2] != 0.0)
