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

import numpy as np
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


def sgp4_propagate_jd(records: Records, jd_day: torch.Tensor, jd_frac: torch.Tensor,
                      precision: str = "fp32", out: tuple | None = None,
                      fixups: torch.Tensor | None = None, stream=None):
    """r, v [n, T, 3] and status [n, T] at absolute times given as Julian dates split
    into int32 days jd_day [T] and fractions jd_frac [T]; each record propagates from
    the split epoch it was built with (sgp4_init's epoch_day, epoch_frac)."""
    _require_cuda("jd_day", jd_day, torch.int32)
    _require_cuda("jd_frac", jd_frac, torch.float64)
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    if jd_day.dim() != 1 or jd_frac.shape != jd_day.shape:
        raise ValueError("jd_day and jd_frac must both be [T]")
    n = records.n
    T = jd_day.shape[0]
    dt = torch.float32 if precision == "fp32" else torch.float64
    dev = jd_day.device
    if out is None:
        r = torch.empty((n, T, 3), dtype=dt, device=dev)
        v = torch.empty((n, T, 3), dtype=dt, device=dev)
        st = torch.empty((n, T), dtype=torch.int32, device=dev)
    else:
        r, v, st = out
    if fixups is not None:
        _require_cuda("fixups", fixups, torch.int64)
    lib = _lib.load()
    _lib.check("sgp4_propagate_jd",
               lib.sgp4_propagate_jd(ctypes.byref(records.c), _ptr(jd_day), _ptr(jd_frac), T,
                                     PRECISIONS[precision], _ptr(r), _ptr(v), _ptr(st),
                                     _ptr(fixups), _stream_handle(stream)))
    return r, v, st


def sgp4_jacobian(elements: torch.Tensor, records: Records, tsince: torch.Tensor,
                  precision: str = "fp64", cov: torch.Tensor | None = None,
                  want_state: bool = True, want_jac: bool = True, stream=None) -> dict:
    """Per-state Jacobians J = d(r, v)/d(elements) [n, T, 6, 7] and, given an element
    covariance cov [n, 7, 7], the state covariance J cov J^T as its upper triangle
    [n, T, 21] (row by row).  Returns a dict with 'status' and those of 'r', 'v', 'jac',
    'cov' that were asked for."""
    _require_cuda("elements", elements, torch.float64)
    _require_cuda("tsince", tsince, torch.float64)
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    n = records.n
    per_sat = tsince.dim() == 2
    T = tsince.shape[-1]
    dt = torch.float32 if precision == "fp32" else torch.float64
    dev = tsince.device
    out = {"status": torch.empty((n, T), dtype=torch.int32, device=dev)}
    if want_state:
        out["r"] = torch.empty((n, T, 3), dtype=dt, device=dev)
        out["v"] = torch.empty((n, T, 3), dtype=dt, device=dev)
    if want_jac:
        out["jac"] = torch.empty((n, T, 6, 7), dtype=dt, device=dev)
    if cov is not None:
        _require_cuda("cov", cov, torch.float64)
        if tuple(cov.shape) != (n, 7, 7):
            raise ValueError("cov must be [n, 7, 7]")
        out["cov"] = torch.empty((n, T, 21), dtype=dt, device=dev)
    lib = _lib.load()
    ws_bytes = int(lib.sgp4_jacobian_workspace_bytes(n))
    ws = torch.empty(max(ws_bytes // 8, 1), dtype=torch.float64, device=dev)
    _lib.check("sgp4_jacobian",
               lib.sgp4_jacobian(_ptr(elements), ctypes.byref(records.c), _ptr(tsince), T,
                                 1 if per_sat else 0, PRECISIONS[precision], _ptr(out.get("r")),
                                 _ptr(out.get("v")), _ptr(out["status"]), _ptr(out.get("jac")),
                                 _ptr(cov), _ptr(out.get("cov")), _ptr(ws), ws_bytes,
                                 _stream_handle(stream)))
    return out


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


# ------------------------------------------------------------------------ batching
@dataclass
class BatchPlan:
    """A prepared batch of requests: device workspace plus the ABI plan struct."""
    workspace: torch.Tensor
    c: _lib.Sgp4BatchPlan
    requests: np.ndarray          # [n_req, 5] int64: sat_offset, n, t_offset, t_count, out_offset

    @property
    def total_states(self) -> int:
        return int(self.c.total_states)


@dataclass
class Batch:
    """Concatenated inputs of many requests (see ``make_batch``)."""
    elements: np.ndarray          # [sum n_i, 7]
    tsince: np.ndarray            # [sum T_i]
    requests: np.ndarray          # [n_req, 5] int64, outputs contiguous in request order


def make_batch(problems) -> Batch:
    """Concatenate (elements [n_i, 7], tsince [T_i]) pairs into one record set, one
    grid array and a request table whose outputs follow each other."""
    els, ts, rows = [], [], []
    sat = tof = out = 0
    for el, t in problems:
        el = np.asarray(el, dtype=np.float64).reshape(-1, 7)
        t = np.asarray(t, dtype=np.float64).reshape(-1)
        rows.append((sat, el.shape[0], tof, t.shape[0], out))
        els.append(el)
        ts.append(t)
        sat += el.shape[0]
        tof += t.shape[0]
        out += el.shape[0] * t.shape[0]
    return Batch(np.concatenate(els) if els else np.zeros((0, 7)),
                 np.concatenate(ts) if ts else np.zeros(0),
                 np.asarray(rows, dtype=np.int64).reshape(-1, 5))


def plan_batch(requests, tile_states: int = 1024, grid_blocks: int = 0, device=None,
               stream=None) -> BatchPlan:
    """Validate a request table ([n_req, 5] int64) and place it in a device workspace."""
    req = np.ascontiguousarray(np.asarray(requests, dtype=np.int64).reshape(-1, 5))
    n = req.shape[0]
    lib = _lib.load()
    nbytes = int(lib.sgp4_batch_workspace_bytes(n))
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")
    plan = _lib.Sgp4BatchPlan()
    table = (_lib.Sgp4Request * max(n, 1))()
    for k in range(n):
        table[k] = _lib.Sgp4Request(*[int(x) for x in req[k]])
    _lib.check("sgp4_batch_plan_init",
               lib.sgp4_batch_plan_init(ctypes.cast(table, ctypes.c_void_p), n, int(tile_states),
                                        int(grid_blocks), _ptr(ws), nbytes, ctypes.byref(plan),
                                        _stream_handle(stream)))
    return BatchPlan(ws, plan, req)


def _batch_out(plan: BatchPlan, precision: str, device, out):
    if out is not None:
        return out
    dt = torch.float32 if precision == "fp32" else torch.float64
    S = int(plan.c.out_needed)
    return (torch.empty((S, 3), dtype=dt, device=device),
            torch.empty((S, 3), dtype=dt, device=device),
            torch.empty((S,), dtype=torch.int32, device=device))


def sgp4_propagate_batched(plan: BatchPlan, records: Records, tsince: torch.Tensor,
                           precision: str = "fp32", out: tuple | None = None,
                           fixups: torch.Tensor | None = None, stream=None):
    """All requests of a plan in one persistent launch.  Returns r, v [S, 3] and
    status [S] over the concatenated output states (request k at its out_offset)."""
    _require_cuda("tsince", tsince, torch.float64)
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    r, v, st = _batch_out(plan, precision, tsince.device, out)
    if fixups is not None:
        _require_cuda("fixups", fixups, torch.int64)
    lib = _lib.load()
    _lib.check("sgp4_propagate_batched",
               lib.sgp4_propagate_batched(ctypes.byref(plan.c), ctypes.byref(records.c),
                                          _ptr(tsince), tsince.numel(), PRECISIONS[precision],
                                          _ptr(r), _ptr(v), _ptr(st), st.numel(), _ptr(fixups),
                                          _stream_handle(stream)))
    return r, v, st


class BatchGraph:
    """The batched launch captured once in a CUDA graph; ``replay()`` re-runs it on
    the same buffers (stream-ordered)."""

    def __init__(self, plan: BatchPlan, records: Records, tsince: torch.Tensor,
                 precision: str = "fp32", out: tuple | None = None, stream=None):
        _require_cuda("tsince", tsince, torch.float64)
        self.plan, self.records, self.tsince = plan, records, tsince
        self.out = _batch_out(plan, precision, tsince.device, out)
        self._capture_stream = torch.cuda.Stream(device=tsince.device)
        self._capture_stream.wait_stream(torch.cuda.current_stream(tsince.device))
        r, v, st = self.out
        handle = ctypes.c_void_p()
        lib = _lib.load()
        _lib.check("sgp4_batch_graph_create",
                   lib.sgp4_batch_graph_create(ctypes.byref(plan.c), ctypes.byref(records.c),
                                               _ptr(tsince), tsince.numel(),
                                               PRECISIONS[precision], _ptr(r), _ptr(v), _ptr(st),
                                               st.numel(), None,
                                               _stream_handle(self._capture_stream),
                                               ctypes.byref(handle)))
        self.handle = handle
        self._stream = stream

    def replay(self, stream=None):
        lib = _lib.load()
        _lib.check("sgp4_batch_graph_launch",
                   lib.sgp4_batch_graph_launch(self.handle, _stream_handle(stream or self._stream)))
        return self.out

    def close(self):
        if self.handle:
            _lib.load().sgp4_batch_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------- adjoint
def sgp4_adjoint(elements: torch.Tensor, records: Records, tsince: torch.Tensor,
                 grad_r: torch.Tensor | None, grad_v: torch.Tensor | None,
                 precision: str = "fp64", out: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """d(sum g_r . r + g_v . v)/d(elements) [n, 7] through init and propagation."""
    _require_cuda("elements", elements, torch.float64)
    _require_cuda("tsince", tsince, torch.float64)
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    n = records.n
    if elements.shape != (n, 7):
        raise ValueError("elements must be [n, 7] and match the records")
    per_sat = tsince.dim() == 2
    T = tsince.shape[-1]
    dt = torch.float32 if precision == "fp32" else torch.float64
    for name, g in (("grad_r", grad_r), ("grad_v", grad_v)):
        if g is not None:
            _require_cuda(name, g, dt)
            if g.shape != (n, T, 3):
                raise ValueError(f"{name} must be [n, T, 3]")
    lib = _lib.load()
    if workspace is None:
        workspace = torch.empty(max(int(lib.sgp4_adjoint_workspace_bytes(n)), 8),
                                dtype=torch.uint8, device=elements.device)
    if out is None:
        out = torch.empty((n, 7), dtype=torch.float64, device=elements.device)
    _lib.check("sgp4_adjoint",
               lib.sgp4_adjoint(_ptr(elements), ctypes.byref(records.c), _ptr(tsince), T,
                                1 if per_sat else 0, PRECISIONS[precision], _ptr(grad_r),
                                _ptr(grad_v), _ptr(out), _ptr(workspace), workspace.numel(),
                                _stream_handle(stream)))
    return out


class SGP4Function(torch.autograd.Function):
    """(r, v) = SGP4(elements, tsince) with a hand-written adjoint for backward.

    elements [n, 7] float64 CUDA (n0 rad/min, e0, i0, RAAN0, argp0, M0, B*); tsince
    [T] or [n, T] float64.  r, v are [n, T, 3] in the precision's dtype; states with
    status 1, 2, 4 are NaN and get no gradient.
    """

    @staticmethod
    def forward(ctx, elements, tsince, precision="fp64"):
        recs, _ = sgp4_init(elements.detach().contiguous())
        r, v, st = sgp4_propagate(recs, tsince, precision)
        ctx.save_for_backward(elements, tsince)
        ctx.records = recs
        ctx.precision = precision
        ctx.mark_non_differentiable(st)
        return r, v, st

    @staticmethod
    def backward(ctx, grad_r, grad_v, _grad_st):
        elements, tsince = ctx.saved_tensors
        dt = torch.float32 if ctx.precision == "fp32" else torch.float64
        gr = None if grad_r is None else grad_r.to(dt).nan_to_num(0.0).contiguous()
        gv = None if grad_v is None else grad_v.to(dt).nan_to_num(0.0).contiguous()
        g = sgp4_adjoint(elements.detach().contiguous(), ctx.records, tsince, gr, gv,
                         ctx.precision)
        return g, None, None


def sgp4_differentiable(elements: torch.Tensor, tsince: torch.Tensor, precision: str = "fp64"):
    """Differentiable propagation: returns (r, v, status); backward runs the adjoint."""
    return SGP4Function.apply(elements, tsince, precision)
