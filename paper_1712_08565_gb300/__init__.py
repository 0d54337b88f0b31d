"""GB300 (sm_103a) matrix-free weighted-quadrature isogeometric k-method.

The compute lives in libmfwq.so (CUDA, C ABI in include/mfwq.h); this package
holds the in-tree build, the ctypes binding and the seeded input generators.
"""
from .mfwq import Batch, MfwqError, Operator, SolveInfo, kernel_launches, lib, solve_fn, tables_1d  # noqa: F401

__all__ = ["Batch", "Operator", "MfwqError", "SolveInfo", "kernel_launches", "lib", "solve_fn", "tables_1d"]
