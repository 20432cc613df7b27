"""SGP4 FP64 CPU oracle (near-Earth and deep-space branches) -- TEST INFRASTRUCTURE ONLY.

This package is the independent reference that the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library under ``paper_2603_27830_b300/`` never does.

It wraps ``sgp4_oracle.cpp`` (plain C++17, FP64, built with ``-ffp-contract=off`` and
no fast-math), which restates the near-Earth SGP4 theory that the paper implements
(Sec. 2.1: the Hoots & Roehrich Spacetrack Report #3 equations as revised in 2006,
WGS-72 constants).  The comments in that file list every reading of a point the
paper leaves open.

Parity status of each part (pins live in ``tests/oracle_pins.py``):
  * two-body geometry, Kepler solve, J2/J3/J4 periodics and secular rates: pinned
    (closed forms, bisection, numerical integration of the zonal force model);
  * drag: C1 and the decay polynomials D2..D4, L2..L5 pinned as the Taylor
    coefficients of the circular decay law; the e-dependence of C2 and the drag-only
    part of C4 by orbit averages of Gauss's equations; C5 and the once-per-revolution
    perigee/mean-anomaly term by harmonics of the same equations integrated along the
    orbit; the quadratic node term by the chain rule on the J2 node rate;
  * drag with zonals: the J2 terms of C2 and C4 by an integration of J2 and the
    theory's atmosphere, C3 (drag with J3) by the drift of the eccentricity vector in
    an integration with J3 x10 and drag;
  * the node rate with its second-order J2 and J4 parts: pinned by the node of a
    long numerical integration; the J4 part of the perigee rate by the orbit- and
    perigee-averaged J4 potential through Lagrange's equations;
  * the J3 long-period term of the mean longitude (xlcof, with its 1 / (a(1 - e^2))
    factor): pinned by the evolution of node + argument of latitude in an
    integration with J3 x10;
  * parity unpinned: the cos 2w part of C4's J2 term, the second-order J2 parts of
    the mean-anomaly and perigee rates and the second-order Kozai->Brouwer recovery
    (delta1, the a0 series) -- each a second-order effect that no comparison with a
    numerical integration started from the theory's first-order osculating state can
    resolve.

Deep space (periods of 225 min or more; pins in ``tests/oracle_deep_pins.py``):
  * the sidereal angle: pinned (the degrees-per-day form of the IAU 1982 expression);
  * the Sun's and Moon's secular rates and their application: pinned (the quadrupole
    tide averaged over both orbits through Lagrange's equations, the bodies' orbits
    built from rotation matrices);
  * their long-period terms: pinned for circular body orbits (the tide integrated
    along the body's orbit), directly above 0.2 rad and in the Lyddane form below it
    (first-order normal and longitude, continuity across 0.2 rad and across a
    negative inclination);
  * the resonance amplitudes: pinned (Kaula's F_lmp exactly, his G_lpq from Hansen
    coefficients within the theory's series or fits) and the resonance integration
    (an 8th-order integration of the same equations);
  * classes and code 3: pinned (period and mean-motion windows, e leaving [0, 1]);
  * parity unpinned: the first-order terms in the bodies' orbital eccentricities (the
    theory keeps only an orientation-free sin f term and the first-order true anomaly,
    which no exact reference truncates the same way) and the d2n/dt2 term of the
    resonance integrator's last partial step (~1e-4 of the resonance's effect).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgp4_oracle.cpp")
_LIB = os.path.join(_HERE, "libsgp4_oracle.so")

# WGS-72: mu (km^3/s^2), Earth radius (km), J2, J3, J4 (paper Sec. 2.1).
WGS72 = (398600.8, 6378.135, 0.001082616, -0.00000253881, -0.00000165597)

# Deep-space theory constants (Sun n, e, tide coefficient; Moon n, e, tide
# coefficient; resonance amplitude factor): the values of the theory.
DEEP_THEORY = (1.19459e-5, 0.01675, 2.9864797e-6, 1.5835218e-4, 0.05490, 4.7968065e-7, 1.0)

DEEP_FIELDS = (
    "gsto", "edot", "idot", "mdot_ls", "argpdot_ls", "raandot_ls",
    "sun_e2", "sun_e3", "sun_i2", "sun_i3", "sun_l2", "sun_l3", "sun_l4",
    "sun_gh2", "sun_gh3", "sun_gh4", "sun_h2", "sun_h3", "sun_M0",
    "moon_e2", "moon_e3", "moon_i2", "moon_i3", "moon_l2", "moon_l3", "moon_l4",
    "moon_gh2", "moon_gh3", "moon_gh4", "moon_h2", "moon_h3", "moon_M0",
    "del1", "del2", "del3",
    "d2201", "d2211", "d3210", "d3222", "d4410", "d4422", "d5220", "d5232", "d5421", "d5433",
    "lambda0", "xfact", "irez",
)

RECORD_FIELDS = (
    "n0pp", "a0pp", "cosi", "sini", "x3thm1", "x1mth2", "x7thm1", "beta0",
    "s", "xi", "eta", "C1", "C3", "C4", "C5", "D2", "D3", "D4",
    "Mdot", "argpdot", "raandot", "raan_cf", "argp_cf", "m_cf",
    "L2", "L3", "L4", "L5", "xlcof", "aycof", "delM0", "sinM0",
    "e0", "i0", "bstar", "xke",
)

_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle shared library with g++ (plain FP64, no FMA contraction)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", out + ".tmp", src]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build of it."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    lib.oracle_propagate.argtypes = [P, P, P, P, I64, P, I64, ctypes.c_int, P, P, P, P,
                                     ctypes.c_int]
    lib.oracle_records.argtypes = [P, P, P, P, I64, P, P, P]
    lib.oracle_deep_records.argtypes = [P, P, P, P, I64, P, P]
    lib.oracle_mean.argtypes = [P, P, P, P, I64, P, I64, P]
    lib.oracle_deep_periodics.argtypes = [P, P, P, P, I64, P, I64, P]
    lib.oracle_kepler.argtypes = [D, D, D, P]
    lib.oracle_kepler.restype = D
    lib.oracle_gmst.argtypes = [D, D]
    lib.oracle_gmst.restype = D
    lib.oracle_jacobian.argtypes = [P, P, P, P, I64, P, I64, ctypes.c_int, P, P, P, ctypes.c_int]
    lib.oracle_nrec.restype = ctypes.c_int
    lib.oracle_ndeep.restype = ctypes.c_int
    assert lib.oracle_nrec() == len(RECORD_FIELDS)
    assert lib.oracle_ndeep() == len(DEEP_FIELDS)
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(elements, tsince, consts):
    el = np.ascontiguousarray(elements, dtype=np.float64)
    if el.ndim != 2 or el.shape[1] != 7:
        raise ValueError("elements must be [n, 7]")
    t = np.ascontiguousarray(tsince, dtype=np.float64)
    c = np.ascontiguousarray(consts, dtype=np.float64)
    assert c.shape == (5,)
    return el, t, c


def _epoch(epoch, n):
    """(day [n], frac [n]) Julian-date epochs -> a contiguous [n, 2] array, or None."""
    if epoch is None:
        return None
    day, frac = epoch
    ep = np.empty((n, 2))
    ep[:, 0] = np.broadcast_to(np.asarray(day, dtype=np.float64), (n,))
    ep[:, 1] = np.broadcast_to(np.asarray(frac, dtype=np.float64), (n,))
    return ep


def _deep(deep):
    if deep is None:
        return None
    d = np.ascontiguousarray(deep, dtype=np.float64)
    assert d.shape == (7,)
    return d


def _optr(a):
    return None if a is None else _ptr(a)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def propagate(elements, tsince, consts=WGS72, threads: int | None = None, lib=None,
              epoch=None, deep=None):
    """r [n,T,3] km, v [n,T,3] km/s, status [n,T] int32, init_status [n] int32.

    ``tsince`` is [T] (one grid for all satellites) or [n, T] (a grid per satellite).
    ``epoch`` = (day, frac): each record's epoch as a split Julian date (scalars or
    [n]; None: epoch 0), which the deep-space terms depend on.  ``deep`` overrides the
    deep-space constants (``DEEP_THEORY`` layout).  States with codes 1, 2, 3, 4 (and
    records with unusable elements) are NaN.
    """
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n = el.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    per_sat = 1 if t.ndim == 2 else 0
    T = t.shape[-1]
    if per_sat and t.shape[0] != n:
        raise ValueError("per-satellite grid must be [n, T]")
    r = np.empty((n, T, 3))
    v = np.empty((n, T, 3))
    st = np.empty((n, T), dtype=np.int32)
    ist = np.empty((n,), dtype=np.int32)
    lib.oracle_propagate(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(t), T, per_sat,
                         _ptr(r), _ptr(v), _ptr(st), _ptr(ist), int(threads or default_threads()))
    return r, v, st, ist


def records(elements, consts=WGS72, lib=None, epoch=None, deep=None):
    """Per-satellite constants: dict name -> [n] array, plus 'isimp' and 'init_status'."""
    lib = lib or load()
    el, _, c = _prep(elements, np.zeros(1), consts)
    n = el.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    out = np.empty((n, len(RECORD_FIELDS)))
    isimp = np.empty((n,), dtype=np.int32)
    ist = np.empty((n,), dtype=np.int32)
    lib.oracle_records(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(out), _ptr(isimp),
                       _ptr(ist))
    d = {name: out[:, k].copy() for k, name in enumerate(RECORD_FIELDS)}
    d["isimp"] = isimp
    d["init_status"] = ist
    return d


def deep_records(elements, consts=WGS72, lib=None, epoch=None, deep=None):
    """Deep-space constants: dict name -> [n] array (NaN for near-Earth records), plus
    'deep' = -1 (unusable), 0 (near-Earth) or 1 + irez (deep space; irez 0 none,
    1 one revolution per day, 2 two)."""
    lib = lib or load()
    el, _, c = _prep(elements, np.zeros(1), consts)
    n = el.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    out = np.empty((n, len(DEEP_FIELDS)))
    flag = np.empty((n,), dtype=np.int32)
    lib.oracle_deep_records(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(out), _ptr(flag))
    d = {name: out[:, k].copy() for k, name in enumerate(DEEP_FIELDS)}
    d["deep"] = flag
    return d


def mean_elements(elements, tsince, consts=WGS72, lib=None, epoch=None, deep=None):
    """[n, T, 8]: a (ER), e, n (rad/min), RAAN, argp, M (reduced), code, i after the
    secular step (deep space: with the lunar-solar secular rates and the resonance)."""
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n, T = el.shape[0], t.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    out = np.empty((n, T, 8))
    lib.oracle_mean(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(t), T, _ptr(out))
    return out


def deep_periodics(elements, tsince, consts=WGS72, lib=None, epoch=None, deep=None):
    """[n, T, 6]: e, i, RAAN, argp, M after the lunar-solar periodic terms, and the
    code (0, 3; -1 for a near-Earth record; the secular code where that failed)."""
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n, T = el.shape[0], t.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    out = np.empty((n, T, 6))
    lib.oracle_deep_periodics(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(t), T, _ptr(out))
    return out


def kepler(U: float, axn: float, ayn: float, lib=None):
    """Root psi of psi - a_xN sin psi + a_yN cos psi = U, and the Newton step count."""
    lib = lib or load()
    it = ctypes.c_int32(0)
    psi = lib.oracle_kepler(float(U), float(axn), float(ayn), ctypes.byref(it))
    return psi, it.value


def gmst(day: float, frac: float, lib=None) -> float:
    """Greenwich mean sidereal angle (rad) at the Julian date day + frac."""
    lib = lib or load()
    return lib.oracle_gmst(float(day), float(frac))


def jacobian(elements, tsince, consts=WGS72, threads: int | None = None, lib=None,
             epoch=None, deep=None):
    """Forward-mode (dual-number) d(r, v)/d(n0, e0, i0, RAAN0, argp0, M0, B*).

    Returns dr, dv [n, T, 3, 7] and status [n, T].
    """
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n = el.shape[0]
    ep, dc = _epoch(epoch, n), _deep(deep)
    per_sat = 1 if t.ndim == 2 else 0
    T = t.shape[-1]
    dr = np.empty((n, T, 3, 7))
    dv = np.empty((n, T, 3, 7))
    st = np.empty((n, T), dtype=np.int32)
    lib.oracle_jacobian(_ptr(c), _optr(dc), _ptr(el), _optr(ep), n, _ptr(t), T, per_sat,
                        _ptr(dr), _ptr(dv), _ptr(st), int(threads or default_threads()))
    return dr, dv, st
