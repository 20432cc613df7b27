"""Two-line element sets: parse TLE text into the elements and split epochs that
`sgp4_init` takes, and write (synthetic) catalogues back out.  Thin wrappers of the
library's host functions `sgp4_tle_parse`, `sgp4_tle_parse_text`, `sgp4_tle_format`.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib


@dataclass
class TleSet:
    elements: np.ndarray      # [n, 7]: n0 rad/min, e0, i0, RAAN0, argp0, M0 rad, B* 1/ER
    epoch_day: np.ndarray     # [n] int32, Julian day
    epoch_frac: np.ndarray    # [n] float64, fraction of the Julian day in [0, 1)
    satnum: np.ndarray        # [n] int32 catalogue numbers
    rejected: int = 0         # malformed sets skipped by parse_text


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def parse(line1: str, line2: str) -> TleSet:
    """One set; raises Sgp4Error on a malformed set or a checksum mismatch."""
    lib = _lib.load()
    el = np.zeros(7)
    day = np.zeros(1, dtype=np.int32)
    frac = np.zeros(1)
    num = np.zeros(1, dtype=np.int32)
    _lib.check("sgp4_tle_parse", lib.sgp4_tle_parse(line1.encode(), line2.encode(), _p(el),
                                                     _p(day), _p(frac), _p(num)))
    return TleSet(el[None], day, frac, num)


def parse_text(text: str) -> TleSet:
    """Every valid two- or three-line set of a text, in order."""
    lib = _lib.load()
    raw = text.encode()
    rej = ctypes.c_int64(0)
    cap = max(1, raw.count(b"\n") // 2 + 1)
    while True:
        el = np.zeros((cap, 7))
        day = np.zeros(cap, dtype=np.int32)
        frac = np.zeros(cap)
        num = np.zeros(cap, dtype=np.int32)
        n = lib.sgp4_tle_parse_text(raw, len(raw), cap, _p(el), _p(day), _p(frac), _p(num),
                                    ctypes.byref(rej))
        if n < 0:
            raise _lib.Sgp4Error("sgp4_tle_parse_text", _lib.SGP4_ERR_ARG)
        if n <= cap:
            return TleSet(el[:n], day[:n], frac[:n], num[:n], int(rej.value))
        cap = n


def format_sets(elements, epoch_day, epoch_frac, satnum=None) -> list[tuple[str, str]]:
    """Lines of the sets for [n, 7] elements and split epochs (format resolution)."""
    lib = _lib.load()
    el = np.ascontiguousarray(elements, dtype=np.float64).reshape(-1, 7)
    n = el.shape[0]
    day = np.broadcast_to(np.asarray(epoch_day, dtype=np.int64), (n,))
    frac = np.broadcast_to(np.asarray(epoch_frac, dtype=np.float64), (n,))
    nums = np.arange(1, n + 1) if satnum is None else np.asarray(satnum)
    out = []
    l1 = ctypes.create_string_buffer(70)
    l2 = ctypes.create_string_buffer(70)
    for k in range(n):
        row = np.ascontiguousarray(el[k])
        _lib.check("sgp4_tle_format", lib.sgp4_tle_format(_p(row), int(day[k]), float(frac[k]),
                                                          int(nums[k]), l1, l2))
        out.append((l1.value.decode(), l2.value.decode()))
    return out


def write_catalogue(path: str, elements, epoch_day, epoch_frac, names=None) -> int:
    """Write a three-line-set catalogue file; returns the number of sets."""
    sets = format_sets(elements, epoch_day, epoch_frac)
    with open(path, "w") as f:
        for k, (a, b) in enumerate(sets):
            f.write(f"{names[k] if names is not None else f'SAT-{k + 1:05d}'}\n{a}\n{b}\n")
    return len(sets)
