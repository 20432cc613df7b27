"""B300-native SGP4 near-Earth propagation.

The C ABI is declared in include/sgp4.h and implemented by the CUDA kernels under
csrc/, built in-tree into libsgp4_b300.so.  The Python layer (api.py) only
marshals torch tensors to that ABI; there is no CPU fallback.
"""
from .api import (Records, alloc_records, propagate_host, sgp4_init,  # noqa: F401
                  sgp4_propagate)

__all__ = ["Records", "alloc_records", "propagate_host", "sgp4_init", "sgp4_propagate"]
