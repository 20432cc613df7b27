"""Seeded synthetic element sets and time grids for the five benchmark workloads.

This module only draws numbers: it holds none of the propagation arithmetic, so
that the CUDA path and the CPU oracle can both be fed from it.  Elements are rows
(n0 [rad/min, Kozai], e0, i0, RAAN0, argp0, M0 [rad], B* [1/Earth radii]).

The paper measures on CelesTrak Starlink TLEs (Sec. 3.1) that are not available
here; the Starlink-shaped shell generator stands in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

REV_PER_DAY = 2.0 * math.pi / 1440.0   # rev/day -> rad/min
DEG = math.pi / 180.0
# Two-body constants used only to reject draws whose perigee is too low
# (WGS-72 mu and Earth radius); this is input screening, not propagation.
_MU_KM3S2 = 398600.8
_RE_KM = 6378.135


@dataclass
class Workload:
    name: str
    elements: np.ndarray            # [n, 7] float64
    tsince: np.ndarray              # [T] or [n, T] float64, minutes
    description: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.elements.shape[0])

    @property
    def t_count(self) -> int:
        return int(self.tsince.shape[-1])

    @property
    def states(self) -> int:
        return self.n * self.t_count


@dataclass
class Request:
    elements: np.ndarray            # [n_i, 7]
    tsince: np.ndarray              # [T_i], sorted


def _semi_major_km(n_radmin: np.ndarray) -> np.ndarray:
    n_rads = n_radmin / 60.0
    return (_MU_KM3S2 / n_rads ** 2) ** (1.0 / 3.0)


def config1(seed: int = 0, n: int = 64, t_count: int = 100) -> Workload:
    """64 near-Earth satellites x 100 times over one day (plain FP64 case)."""
    rng = np.random.default_rng(1000 + seed)
    el = np.column_stack([
        rng.uniform(11.0, 16.0, n) * REV_PER_DAY,
        rng.uniform(0.0, 0.02, n),
        rng.uniform(0.0, 100.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        np.exp(rng.uniform(math.log(1e-5), math.log(1e-3), n)),
    ])
    return Workload("near-earth-64x100", el, np.linspace(0.0, 1440.0, t_count),
                    "64 sats, n U[11,16] rev/day, e U[0,0.02], i U[0,100] deg, "
                    "B* log-U[1e-5,1e-3], tsince 0..1440 min")


STARLINK_SHELLS = ((53.0, 0.45), (53.2, 0.35), (70.0, 0.05), (97.6, 0.15))


def config2(seed: int = 0, n: int = 9341, t_count: int = 1000) -> Workload:
    """Starlink-shaped shells, 9,341 satellites x 1,000 times over one day."""
    rng = np.random.default_rng(2000 + seed)
    incs = np.array([s[0] for s in STARLINK_SHELLS])
    w = np.array([s[1] for s in STARLINK_SHELLS])
    shell = rng.choice(len(incs), size=n, p=w / w.sum())
    planes, slots = 72, 22
    plane = rng.integers(0, planes, n)
    slot = rng.integers(0, slots, n)
    raan = (plane * (360.0 / planes) + shell * 5.0 + rng.uniform(-0.5, 0.5, n)) % 360.0
    mean_anom = (slot * (360.0 / slots) + plane * (360.0 / (planes * slots))
                 + rng.uniform(-0.5, 0.5, n)) % 360.0
    # 540-570 km altitude <-> about 15.05-15.10 rev/day, jitter 1e-3 rev/day
    n_rev = rng.uniform(15.05, 15.10, n) + rng.normal(0.0, 1e-3, n)
    el = np.column_stack([
        n_rev * REV_PER_DAY,
        np.abs(rng.normal(0.0, 2e-4, n)),
        incs[shell] * DEG,
        raan * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        mean_anom * DEG,
        np.exp(rng.normal(math.log(1e-4), 0.5, n)),
    ])
    return Workload("starlink-9341x1000", el, np.linspace(0.0, 1440.0, t_count),
                    "Starlink-shaped shells i {53,53.2,70,97.6} deg, n U[15.05,15.10] rev/day "
                    "+N(0,1e-3), e |N(0,2e-4)|, RAAN/M on a 72x22 lattice + U(-0.5,0.5) deg, "
                    "B* lognormal(ln 1e-4, 0.5), tsince 0..1440 min")


def catalogue_elements(rng: np.random.Generator, n: int, invalid_frac: float = 0.01,
                       bstar_range=(1e-6, 1e-2), e_max: float = 0.2,
                       return_invalid: bool = False):
    """Near-Earth catalogue draw: period < 225 min, e U[0, e_max] with perigee above
    6,578 km, B* log-uniform; a fraction of deliberately invalid records (half with
    e0 in [1, 1.5], half with a perigee below the Earth's surface)."""
    out = np.empty((n, 7))
    filled = 0
    while filled < n:
        m = max(1024, int((n - filled) * 1.6))
        n_rev = rng.uniform(6.45, 16.5, m)
        e = rng.uniform(0.0, e_max, m)
        ok = _semi_major_km(n_rev * REV_PER_DAY) * (1.0 - e) > 6578.0
        k = min(int(ok.sum()), n - filled)
        out[filled:filled + k, 0] = n_rev[ok][:k] * REV_PER_DAY
        out[filled:filled + k, 1] = e[ok][:k]
        filled += k
    out[:, 2] = rng.uniform(0.0, 180.0, n) * DEG
    out[:, 3] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 4] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 5] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 6] = np.exp(rng.uniform(math.log(bstar_range[0]), math.log(bstar_range[1]), n))
    n_bad = int(round(invalid_frac * n))
    if n_bad:
        bad = rng.choice(n, size=n_bad, replace=False)
        half = n_bad // 2
        out[bad[:half], 1] = rng.uniform(1.0, 1.5, half)
        low = bad[half:]
        a = _semi_major_km(out[low, 0])
        out[low, 1] = 1.0 - _RE_KM * rng.uniform(0.85, 0.995, low.size) / a
    else:
        bad = np.zeros(0, dtype=np.int64)
    if return_invalid:
        return out, np.sort(bad)
    return out


def config3(seed: int = 0, n: int = 1_000_000, t_count: int = 100) -> Workload:
    """Catalogue scale: 1,000,000 satellites x 100 times over 7 days, ~1% invalid."""
    rng = np.random.default_rng(3000 + seed)
    el, bad = catalogue_elements(rng, n, return_invalid=True)
    return Workload("catalogue-1Mx100", el, np.linspace(0.0, 10080.0, t_count),
                    "n U[6.45,16.5] rev/day (period < 225 min), e U[0,0.2] with perigee > "
                    "6578 km, i U[0,180) deg, B* log-U[1e-6,1e-2], 1% invalid, "
                    "tsince 0..10080 min", meta={"invalid": bad})


def config4(seed: int = 0, n_requests: int = 256, n_range=(100, 50_000),
            t_range=(10, 5_000)) -> list[Request]:
    """256 uneven requests, each with its own sorted grid drawn U[-720, 2880] min."""
    rng = np.random.default_rng(4000 + seed)
    reqs = []
    for _ in range(n_requests):
        n_i = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        t_i = int(round(math.exp(rng.uniform(math.log(t_range[0]), math.log(t_range[1])))))
        el = catalogue_elements(rng, n_i)
        t = np.sort(rng.uniform(-720.0, 2880.0, t_i))
        reqs.append(Request(el, t))
    return reqs


def config5(seed: int = 0, n: int = 10_000, t_count: int = 500):
    """Element fitting: base elements, the perturbed 'truth' (relative N(0, 1e-4)),
    the time grid and a generator for the 0.01 km observation noise."""
    rng = np.random.default_rng(5000 + seed)
    base = np.column_stack([
        rng.uniform(12.0, 16.0, n) * REV_PER_DAY,
        rng.uniform(0.001, 0.05, n),
        rng.uniform(10.0, 170.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        rng.uniform(0.0, 360.0, n) * DEG,
        np.exp(rng.uniform(math.log(1e-5), math.log(1e-3), n)),
    ])
    truth = base * (1.0 + rng.normal(0.0, 1e-4, base.shape))
    t = np.linspace(0.0, 1440.0, t_count)
    noise_seed = 5500 + seed

    def noise(shape):
        return np.random.default_rng(noise_seed).normal(0.0, 0.01, shape)

    return Workload("fit-10000x500", base, t, "elements fit, truth = base (1 + N(0,1e-4))",
                    meta={"truth": truth, "noise": noise})


def deep_space_elements(rng: np.random.Generator, n: int):
    """Deep-space catalogue draw (periods of 225 min or more) in five classes:
    geosynchronous 35% (n U[0.99, 1.01] rev/day, e |N(0, 5e-4)|, i U[0, 15] deg),
    Molniya 15% (n U[2.0, 2.02], e U[0.6, 0.75], i N(63.4, 1) deg), navigation 20%
    (n U[1.7, 2.01], e U[0, 0.02], i U[50, 65] deg), transfer orbits 20% (n U[2.2,
    2.4], e U[0.65, 0.73], i U[0, 30] deg, perigee above 6,578 km) and others 10%
    (period U[225 min, 3 days], e U[0, 0.5], perigee above 6,578 km); node, perigee and
    mean anomaly U[0, 360) deg; B* log-U[1e-6, 1e-3]."""
    cls = rng.choice(5, size=n, p=[0.35, 0.15, 0.20, 0.20, 0.10])
    out = np.empty((n, 7))
    for c in range(5):
        k = np.nonzero(cls == c)[0]
        m = k.size
        if m == 0:
            continue
        if c == 0:
            nr, e, i = rng.uniform(0.99, 1.01, m), np.minimum(np.abs(rng.normal(0, 5e-4, m)),
                                                               0.01), rng.uniform(0, 15, m)
        elif c == 1:
            nr, e, i = rng.uniform(2.0, 2.02, m), rng.uniform(0.6, 0.75, m), rng.normal(63.4, 1, m)
        elif c == 2:
            nr, e, i = rng.uniform(1.7, 2.01, m), rng.uniform(0, 0.02, m), rng.uniform(50, 65, m)
        else:
            nr = np.empty(m)
            e = np.empty(m)
            filled = 0
            while filled < m:
                q = 2 * (m - filled) + 16
                if c == 3:
                    nq, eq = rng.uniform(2.2, 2.4, q), rng.uniform(0.65, 0.73, q)
                else:
                    nq, eq = 1440.0 / rng.uniform(225.0, 4320.0, q), rng.uniform(0.0, 0.5, q)
                ok = _semi_major_km(nq * REV_PER_DAY) * (1.0 - eq) > 6578.0
                take = min(int(ok.sum()), m - filled)
                nr[filled:filled + take] = nq[ok][:take]
                e[filled:filled + take] = eq[ok][:take]
                filled += take
            i = rng.uniform(0, 30, m) if c == 3 else rng.uniform(0, 180, m)
        out[k, 0] = nr * REV_PER_DAY
        out[k, 1] = e
        out[k, 2] = np.clip(i, 0.0, 180.0) * DEG
    out[:, 3] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 4] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 5] = rng.uniform(0.0, 360.0, n) * DEG
    out[:, 6] = np.exp(rng.uniform(math.log(1e-6), math.log(1e-3), n))
    return out


def deep_space(seed: int = 0, n: int = 10_000, t_count: int = 1000) -> Workload:
    """Deep-space catalogue: n satellites of deep_space_elements x t_count times over
    seven days, each with its own epoch (Julian day U{2458000..2461999} + U[0, 1))."""
    rng = np.random.default_rng(6000 + seed)
    el = deep_space_elements(rng, n)
    day = rng.integers(2458000, 2462000, n).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, n)
    return Workload(f"deep-space-{n}x{t_count}", el, np.linspace(0.0, 10080.0, t_count),
                    "deep-space classes (geosynchronous, Molniya, navigation, transfer, "
                    "other), own epochs, tsince 0..10080 min",
                    meta={"epoch_day": day, "epoch_frac": frac})
