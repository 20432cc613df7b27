"""SGP4 near-Earth FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

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
    lib.oracle_propagate.argtypes = [P, P, I64, P, I64, ctypes.c_int, P, P, P, P, ctypes.c_int]
    lib.oracle_records.argtypes = [P, P, I64, P, P, P]
    lib.oracle_mean.argtypes = [P, P, I64, P, I64, P]
    lib.oracle_kepler.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
    lib.oracle_kepler.restype = ctypes.c_double
    lib.oracle_jacobian.argtypes = [P, P, I64, P, I64, ctypes.c_int, P, P, P, ctypes.c_int]
    lib.oracle_nrec.restype = ctypes.c_int
    assert lib.oracle_nrec() == len(RECORD_FIELDS)
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


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def propagate(elements, tsince, consts=WGS72, threads: int | None = None, lib=None):
    """r [n,T,3] km, v [n,T,3] km/s, status [n,T] int32, init_status [n] int32.

    ``tsince`` is [T] (one grid for all satellites) or [n, T] (a grid per satellite).
    States with codes 1, 2, 4 (and records with unusable elements) are NaN.
    """
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n = el.shape[0]
    per_sat = 1 if t.ndim == 2 else 0
    T = t.shape[-1]
    if per_sat and t.shape[0] != n:
        raise ValueError("per-satellite grid must be [n, T]")
    r = np.empty((n, T, 3))
    v = np.empty((n, T, 3))
    st = np.empty((n, T), dtype=np.int32)
    ist = np.empty((n,), dtype=np.int32)
    lib.oracle_propagate(_ptr(c), _ptr(el), n, _ptr(t), T, per_sat, _ptr(r), _ptr(v), _ptr(st),
                         _ptr(ist), int(threads or default_threads()))
    return r, v, st, ist


def records(elements, consts=WGS72, lib=None):
    """Per-satellite constants: dict name -> [n] array, plus 'isimp' and 'init_status'."""
    lib = lib or load()
    el, _, c = _prep(elements, np.zeros(1), consts)
    n = el.shape[0]
    out = np.empty((n, len(RECORD_FIELDS)))
    isimp = np.empty((n,), dtype=np.int32)
    ist = np.empty((n,), dtype=np.int32)
    lib.oracle_records(_ptr(c), _ptr(el), n, _ptr(out), _ptr(isimp), _ptr(ist))
    d = {name: out[:, k].copy() for k, name in enumerate(RECORD_FIELDS)}
    d["isimp"] = isimp
    d["init_status"] = ist
    return d


def mean_elements(elements, tsince, consts=WGS72, lib=None):
    """[n, T, 7]: a (ER), e, n (rad/min), RAAN, argp, M (reduced), code after the secular step."""
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n, T = el.shape[0], t.shape[0]
    out = np.empty((n, T, 7))
    lib.oracle_mean(_ptr(c), _ptr(el), n, _ptr(t), T, _ptr(out))
    return out


def kepler(U: float, axn: float, ayn: float, lib=None):
    """Root psi of psi - a_xN sin psi + a_yN cos psi = U, and the Newton step count."""
    lib = lib or load()
    it = ctypes.c_int32(0)
    psi = lib.oracle_kepler(float(U), float(axn), float(ayn), ctypes.byref(it))
    return psi, it.value


def jacobian(elements, tsince, consts=WGS72, threads: int | None = None, lib=None):
    """Forward-mode (dual-number) d(r, v)/d(n0, e0, i0, RAAN0, argp0, M0, B*).

    Returns dr, dv [n, T, 3, 7] and status [n, T].
    """
    lib = lib or load()
    el, t, c = _prep(elements, tsince, consts)
    n = el.shape[0]
    per_sat = 1 if t.ndim == 2 else 0
    T = t.shape[-1]
    dr = np.empty((n, T, 3, 7))
    dv = np.empty((n, T, 3, 7))
    st = np.empty((n, T), dtype=np.int32)
    lib.oracle_jacobian(_ptr(c), _ptr(el), n, _ptr(t), T, per_sat, _ptr(dr), _ptr(dv), _ptr(st),
                        int(threads or default_threads()))
    return dr, dv, st
