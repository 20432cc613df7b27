"""PyTorch-facing wrappers of the C ABI: device memory and streams come from torch,
every step of the computation runs in the CUDA kernels of ``libsgp4_b300.so``.

Typical use::

    recs, init_status = sgp4_init(elements_cuda_f64)          # [n, 7]
    r, v, status = sgp4_propagate(recs, tsince_cuda_f64, "fp32")

There is no CPU path: inputs must be CUDA tensors.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib

PRECISIONS = {"fp64": _lib.SGP4_FP64, "fp32": _lib.SGP4_FP32}
WGS72 = (398600.8, 6378.135, 0.001082616, -0.00000253881, -0.00000165597)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream: torch.cuda.Stream | None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(name: str, t: torch.Tensor, dtype: torch.dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class Records:
    """Device records of n satellites: a caller-owned arena plus the ABI struct."""
    arena: torch.Tensor
    c: _lib.Sgp4Records

    @property
    def n(self) -> int:
        return int(self.c.n)


def consts_struct(consts=None) -> _lib.Sgp4Consts:
    c = WGS72 if consts is None else tuple(consts)
    return _lib.Sgp4Consts(*[float(x) for x in c])


def alloc_records(n: int, device=None, consts=None) -> Records:
    lib = _lib.load()
    nbytes = int(lib.sgp4_records_bytes(int(n)))
    arena = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")
    rec = _lib.Sgp4Records()
    cs = consts_struct(consts)
    _lib.check("sgp4_records_bind",
               lib.sgp4_records_bind(_ptr(arena), nbytes, int(n), ctypes.byref(cs),
                                     ctypes.byref(rec)))
    return Records(arena, rec)


def sgp4_init(elements: torch.Tensor, consts=None, epoch_day: torch.Tensor | None = None,
              epoch_frac: torch.Tensor | None = None, records: Records | None = None,
              init_status: torch.Tensor | None = None, stream=None):
    """Build device records from [n, 7] FP64 mean elements.  Returns (records, init_status)."""
    _require_cuda("elements", elements, torch.float64)
    if elements.dim() != 2 or elements.shape[1] != 7:
        raise ValueError("elements must be [n, 7]")
    n = elements.shape[0]
    if epoch_day is not None:
        _require_cuda("epoch_day", epoch_day, torch.int32)
    if epoch_frac is not None:
        _require_cuda("epoch_frac", epoch_frac, torch.float64)
    recs = records if records is not None else alloc_records(n, elements.device, consts)
    if init_status is None:
        init_status = torch.empty(n, dtype=torch.int32, device=elements.device)
    lib = _lib.load()
    _lib.check("sgp4_init", lib.sgp4_init(_ptr(elements), _ptr(epoch_day), _ptr(epoch_frac), n,
                                          ctypes.byref(recs.c), _ptr(init_status),
                                          _stream_handle(stream)))
    return recs, init_status


def sgp4_propagate(records: Records, tsince: torch.Tensor, precision: str = "fp32",
                   out: tuple | None = None, fixups: torch.Tensor | None = None, stream=None):
    """r, v [n, T, 3] (km, km/s, TEME) and status [n, T] for a [T] or [n, T] grid."""
    _require_cuda("tsince", tsince, torch.float64)
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    n = records.n
    per_sat = tsince.dim() == 2
    if per_sat and tsince.shape[0] != n:
        raise ValueError("a per-satellite grid must be [n, T]")
    if tsince.dim() not in (1, 2):
        raise ValueError("tsince must be [T] or [n, T]")
    T = tsince.shape[-1]
    dt = torch.float32 if precision == "fp32" else torch.float64
    dev = tsince.device
    if out is None:
        r = torch.empty((n, T, 3), dtype=dt, device=dev)
        v = torch.empty((n, T, 3), dtype=dt, device=dev)
        st = torch.empty((n, T), dtype=torch.int32, device=dev)
    else:
        r, v, st = out
    if fixups is not None:
        _require_cuda("fixups", fixups, torch.int64)
    lib = _lib.load()
    _lib.check("sgp4_propagate",
               lib.sgp4_propagate(ctypes.byref(records.c), _ptr(tsince), T, 1 if per_sat else 0,
                                  PRECISIONS[precision], _ptr(r), _ptr(v), _ptr(st),
                                  _ptr(fixups), _stream_handle(stream)))
    return r, v, st


def propagate_host(elements, tsince, precision: str = "fp32", device="cuda"):
    """End-to-end call on host arrays: copy in, init, propagate, copy out (numpy out)."""
    import numpy as np
    el = torch.from_numpy(np.ascontiguousarray(elements, dtype=np.float64)).pin_memory()
    ts = torch.from_numpy(np.ascontiguousarray(tsince, dtype=np.float64)).pin_memory()
    el_d = el.to(device, non_blocking=True)
    ts_d = ts.to(device, non_blocking=True)
    recs, ist = sgp4_init(el_d)
    r, v, st = sgp4_propagate(recs, ts_d, precision)
    return r.cpu().numpy(), v.cpu().numpy(), st.cpu().numpy(), ist.cpu().numpy()
