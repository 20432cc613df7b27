"""The oracle against what the mathematics fixes (CPU only)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=[p.__name__ for p in P.ALL_PINS])
def test_pin(lib, pin):
    fails = pin(lib)
    assert not fails, "\n".join(fails[:10])


def test_threads_do_not_change_results(lib):
    rng = np.random.default_rng(1)
    el = np.column_stack([rng.uniform(11, 16, 37) * P.REV_DAY, rng.uniform(0, 0.1, 37),
                          rng.uniform(0, 3, 37), rng.uniform(0, 6, 37), rng.uniform(0, 6, 37),
                          rng.uniform(0, 6, 37), rng.uniform(1e-5, 1e-3, 37)])
    t = np.linspace(-100, 3000, 11)
    a = oracle.propagate(el, t, threads=1)
    b = oracle.propagate(el, t, threads=5)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_per_satellite_grid_matches_common_grid(lib):
    rng = np.random.default_rng(2)
    el = np.column_stack([rng.uniform(11, 16, 5) * P.REV_DAY, rng.uniform(0, 0.1, 5),
                          rng.uniform(0, 3, 5), rng.uniform(0, 6, 5), rng.uniform(0, 6, 5),
                          rng.uniform(0, 6, 5), rng.uniform(1e-5, 1e-3, 5)])
    t = np.linspace(0, 1440, 9)
    r1, v1, s1, _ = oracle.propagate(el, t)
    r2, v2, s2, _ = oracle.propagate(el, np.tile(t, (5, 1)))
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(s1, s2)


def test_dual_number_jacobian_matches_central_differences(lib):
    """Forward-mode derivatives of the oracle against central finite differences of
    the plain FP64 oracle (two independent routes through the same equations)."""
    rng = np.random.default_rng(4)
    n = 6
    el = np.column_stack([rng.uniform(13, 15.5, n) * P.REV_DAY, rng.uniform(0.001, 0.05, n),
                          rng.uniform(0.3, 2.5, n), rng.uniform(0, 6, n), rng.uniform(0, 6, n),
                          rng.uniform(0, 6, n), rng.uniform(1e-5, 5e-4, n)])
    t = np.array([0.0, 90.0, 720.0, 1440.0])
    dr, dv, st = oracle.jacobian(el, t)
    assert np.all(st == 0)
    steps = np.array([1e-9, 1e-7, 1e-7, 1e-7, 1e-7, 1e-7, 1e-9])
    for k in range(7):
        ep, em = el.copy(), el.copy()
        ep[:, k] += steps[k]
        em[:, k] -= steps[k]
        rp, vp, _, _ = oracle.propagate(ep, t)
        rm, vm, _, _ = oracle.propagate(em, t)
        fd_r = (rp - rm) / (2 * steps[k])
        fd_v = (vp - vm) / (2 * steps[k])
        scale_r = np.abs(dr[..., k]).max() + 1e-30
        scale_v = np.abs(dv[..., k]).max() + 1e-30
        assert np.abs(fd_r - dr[..., k]).max() < 1e-5 * scale_r + 1e-6, f"d r / d el[{k}]"
        assert np.abs(fd_v - dv[..., k]).max() < 1e-5 * scale_v + 1e-9, f"d v / d el[{k}]"


def test_kepler_iteration_count_is_bounded(lib):
    for U, axn, ayn in ((0.3, 0.1, 0.05), (3.0, 0.0, 0.0), (5.0, 0.7, -0.2)):
        _, it = oracle.kepler(U, axn, ayn)
        assert 1 <= it <= 10


def test_retrograde_pole_guard(lib):
    """i = 180 deg: (1 + cos i) is replaced by 1.5e-12, results stay finite."""
    el = np.array([[15.0 * P.REV_DAY, 0.001, math.pi, 0.2, 0.3, 0.4, 1e-4]])
    r, v, st, ist = oracle.propagate(el, np.linspace(0, 1440, 5))
    assert np.all(st == 0) and np.all(np.isfinite(r)) and np.all(np.isfinite(v))


def test_deep_dual_number_jacobian_matches_central_differences(lib):
    """The dual-number derivatives through the deep-space branch (lunar-solar terms,
    the resonance integration, the Lyddane form) against central differences."""
    el = np.array([[1.00273 * P.REV_DAY, 0.001, 0.1, 1.0, 2.0, 3.0, 1e-5],
                   [2.00561 * P.REV_DAY, 0.72, 1.107, 1.0, 4.7, 0.3, 1e-4],
                   [2.0056 * P.REV_DAY, 0.01, 0.96, 2.0, 1.0, 3.0, 0.0],
                   [0.5 * P.REV_DAY, 0.6, 2.6, 4.0, 5.5, 1.0, 0.0]])
    ep = (np.full(4, 2455000.0), np.full(4, 0.3))
    t = np.array([0.0, 700.0, 5000.0, -3000.0])
    dr, dv, st = oracle.jacobian(el, t, epoch=ep)
    assert np.all(st == 0)
    steps = np.array([1e-10, 1e-8, 1e-7, 1e-7, 1e-7, 1e-7, 1e-6])
    for k in range(7):
        ep_, em_ = el.copy(), el.copy()
        ep_[:, k] += steps[k]
        em_[:, k] -= steps[k]
        rp, vp, _, _ = oracle.propagate(ep_, t, epoch=ep)
        rm, vm, _, _ = oracle.propagate(em_, t, epoch=ep)
        fd_r = (rp - rm) / (2 * steps[k])
        fd_v = (vp - vm) / (2 * steps[k])
        scale_r = np.abs(dr[..., k]).max() + 1e-30
        scale_v = np.abs(dv[..., k]).max() + 1e-30
        assert np.abs(fd_r - dr[..., k]).max() < 1e-5 * scale_r + 1e-5, f"d r / d el[{k}]"
        assert np.abs(fd_v - dv[..., k]).max() < 1e-5 * scale_v + 1e-8, f"d v / d el[{k}]"


def test_deep_epoch_matters_only_for_deep_records(lib):
    """Near-Earth results do not depend on the epoch; deep-space ones do (the Sun's
    and Moon's positions, the sidereal angle)."""
    el = np.array([[15.0 * P.REV_DAY, 0.001, 0.9, 0.2, 0.3, 0.4, 1e-4],
                   [1.00273 * P.REV_DAY, 0.001, 0.1, 1.0, 2.0, 3.0, 1e-5]])
    t = np.linspace(0, 2880, 5)
    a = oracle.propagate(el, t, epoch=(np.full(2, 2455000.0), np.full(2, 0.3)))
    b = oracle.propagate(el, t, epoch=(np.full(2, 2458000.0), np.full(2, 0.7)))
    np.testing.assert_array_equal(a[0][0], b[0][0])
    assert np.abs(a[0][1] - b[0][1]).max() > 1.0
