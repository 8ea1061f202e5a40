"""Segment-parallel Riccati recursion (Laine & Tomlin, arXiv 1809.06360) on GB300.

The solver is the C-ABI library liblqr.so (include/lqr.h) built from csrc/ for
sm_103a; `lqr` is its thin ctypes binding. Importing this package does not load
the library; the first call does, and fails loudly if it has not been built.
"""
from .lqr import Solver, LqrError, load, library_path  # noqa: F401

__all__ = ["Solver", "LqrError", "load", "library_path"]
