"""B300-native SGP4 near-Earth propagation.

The C ABI is declared in include/sgp4.h and implemented by the CUDA kernels under
csrc/, built in-tree into libsgp4_b300.so.  The Python layer (api.py) only
marshals torch tensors to that ABI; there is no CPU fallback.
"""
from .api import (Batch, BatchGraph, BatchPlan, Records, alloc_records,  # noqa: F401
                  SGP4Function, make_batch, plan_batch, propagate_host, sgp4_adjoint,
                  sgp4_differentiable, sgp4_init, sgp4_propagate, sgp4_propagate_batched,
                  sgp4_propagate_jd, sgp4_jacobian)

__all__ = ["Batch", "BatchGraph", "BatchPlan", "Records", "alloc_records", "make_batch",
           "plan_batch", "propagate_host", "sgp4_init", "sgp4_propagate", "sgp4_propagate_jd",
           "sgp4_propagate_batched", "SGP4Function", "sgp4_adjoint", "sgp4_differentiable",
           "sgp4_jacobian"]
