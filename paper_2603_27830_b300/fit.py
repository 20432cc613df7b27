"""Fit mean elements to observed positions (batch least squares, all satellites in
parallel): Levenberg-Marquardt on top of ``sgp4_fit_step``, whose Jacobians come
from the hand-written adjoint sweep (paper Sec. 5: gradient-based orbit
determination with a differentiable SGP4).

Each satellite keeps its own damping: a step is kept when it lowers that
satellite's sum of squared residuals, otherwise it is undone and the damping grows.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from . import _lib
from .api import PRECISIONS, _ptr, _require_cuda, _stream_handle, sgp4_init


def fit_step(elements: torch.Tensor, tsince: torch.Tensor, r_obs: torch.Tensor,
             lam: torch.Tensor, precision: str = "fp64", stream=None):
    """One damped Gauss-Newton step: returns (proposed elements, sse at `elements`)."""
    _require_cuda("elements", elements, torch.float64)
    _require_cuda("tsince", tsince, torch.float64)
    _require_cuda("r_obs", r_obs, torch.float64)
    _require_cuda("lambda", lam, torch.float64)
    recs, _ = sgp4_init(elements, stream=stream)
    n = elements.shape[0]
    out = torch.empty_like(elements)
    sse = torch.empty(n, dtype=torch.float64, device=elements.device)
    lib = _lib.load()
    ws_bytes = int(lib.sgp4_fit_workspace_bytes(n))
    ws = torch.empty(max(ws_bytes // 8, 1), dtype=torch.float64, device=elements.device)
    _lib.check("sgp4_fit_step",
               lib.sgp4_fit_step(_ptr(elements), ctypes.byref(recs.c), _ptr(tsince),
                                 tsince.shape[-1], 1 if tsince.dim() == 2 else 0,
                                 PRECISIONS[precision], _ptr(r_obs), _ptr(lam), _ptr(out),
                                 _ptr(sse), _ptr(ws), ws_bytes, _stream_handle(stream)))
    return out, sse


@dataclass
class FitResult:
    elements: torch.Tensor
    sse: torch.Tensor                  # [n] km^2 at the final elements
    history: list = field(default_factory=list)   # per iteration: median rms |res| (km)


def fit_elements(start: torch.Tensor, tsince: torch.Tensor, r_obs: torch.Tensor,
                 precision: str = "fp64", iters: int = 10, lam0: float = 1e-3) -> FitResult:
    """Levenberg-Marquardt from `start` ([n, 7]) to the observations r_obs ([n, T, 3])."""
    el = start.clone()
    n = el.shape[0]
    T = tsince.shape[-1]
    lam = torch.full((n,), lam0, dtype=torch.float64, device=el.device)
    prop, sse = fit_step(el, tsince, r_obs, lam, precision)
    hist = [float(torch.sqrt(sse / T).median())]
    for _ in range(iters):
        prop2, sse_new = fit_step(prop, tsince, r_obs, lam, precision)
        better = sse_new < sse
        el = torch.where(better[:, None], prop, el)
        sse = torch.where(better, sse_new, sse)
        lam = torch.where(better, lam * 0.3, lam * 10.0).clamp(1e-9, 1e9)
        # next proposal: from the kept point (recomputed where the step was undone)
        if bool(better.all()):
            prop = prop2
        else:
            redo, _ = fit_step(el, tsince, r_obs, lam, precision)
            prop = torch.where(better[:, None], prop2, redo)
        hist.append(float(torch.sqrt(sse / T).median()))
    return FitResult(el, sse, hist)
