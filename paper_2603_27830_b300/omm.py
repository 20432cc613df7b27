"""CCSDS Orbit Mean-Elements Messages (OMM): parse KVN or XML messages with SGP4 mean
elements into the elements and split epochs that `sgp4_init` takes, and write KVN
messages for (synthetic) catalogues.  Thin wrappers of the library's host functions
`sgp4_omm_parse_text` and `sgp4_omm_format`.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .tle import TleSet, _p


def parse_text(text: str) -> TleSet:
    """Every valid message of a KVN or XML text, in order (satnum -1 where the message
    has no NORAD_CAT_ID; `rejected` counts the messages skipped)."""
    lib = _lib.load()
    raw = text.encode()
    rej = ctypes.c_int64(0)
    cap = max(1, raw.count(b"MEAN_MOTION"))
    while True:
        el = np.zeros((cap, 7))
        day = np.zeros(cap, dtype=np.int32)
        frac = np.zeros(cap)
        num = np.zeros(cap, dtype=np.int32)
        n = lib.sgp4_omm_parse_text(raw, len(raw), cap, _p(el), _p(day), _p(frac), _p(num),
                                    ctypes.byref(rej))
        if n < 0:
            raise _lib.Sgp4Error("sgp4_omm_parse_text", _lib.SGP4_ERR_ARG)
        if n <= cap:
            return TleSet(el[:n], day[:n], frac[:n], num[:n], int(rej.value))
        cap = n


def format_messages(elements, epoch_day, epoch_frac, satnum=None, names=None) -> list[str]:
    """KVN messages for [n, 7] elements and split epochs."""
    lib = _lib.load()
    el = np.ascontiguousarray(elements, dtype=np.float64).reshape(-1, 7)
    n = el.shape[0]
    day = np.broadcast_to(np.asarray(epoch_day, dtype=np.int64), (n,))
    frac = np.broadcast_to(np.asarray(epoch_frac, dtype=np.float64), (n,))
    nums = np.arange(1, n + 1) if satnum is None else np.asarray(satnum)
    buf = ctypes.create_string_buffer(1024)
    out = []
    for k in range(n):
        row = np.ascontiguousarray(el[k])
        name = (names[k] if names is not None else f"SAT-{int(nums[k]):05d}").encode()
        _lib.check("sgp4_omm_format", lib.sgp4_omm_format(_p(row), int(day[k]), float(frac[k]),
                                                          int(nums[k]), name, buf, len(buf)))
        out.append(buf.value.decode())
    return out


def write_catalogue(path: str, elements, epoch_day, epoch_frac, satnum=None,
                    names=None) -> int:
    """Write the messages of a catalogue to one KVN file; returns the number written."""
    msgs = format_messages(elements, epoch_day, epoch_frac, satnum, names)
    with open(path, "w") as f:
        f.write("".join(msgs))
    return len(msgs)
