"""GB300-native Randomized Tensor Global GMRES (RTG-GMRES).

The compute path is librtg (hand-written sm_103a CUDA behind a C ABI,
include/rtg.h); this package holds its sources, its build step and a thin
Python binding (`api`).  Importing the package does not load the library;
`api.Handle()` does, and fails loudly if it has not been built.
"""
from . import _lib
from .api import (Factor, Handle, Krylov, SolveResult, banded, dense, empty, identity,
                  to_device, colmajor_strides)

__all__ = ["Handle", "Krylov", "Factor", "SolveResult", "banded", "dense", "identity", "empty",
           "to_device", "colmajor_strides", "build"]


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
