"""GB300-native direct FFT pressure solver (Brown, arXiv 2010.14132, Section 2.1).

Forward real 2-D FFT over the periodic x/y plane at every level, an independent
tridiagonal solve per (kx, ky) column, inverse FFT -- in hand-written sm_103a
CUDA kernels behind the C ABI of include/poisson.h.

    from paper_2010_14132_gb300.solver import Plan, poisson_solve, Batch

Importing the package loads nothing native; the library is loaded on first use.
"""
import importlib

__all__ = ["Plan", "Batch", "PoissonSolve", "poisson_solve"]


def __getattr__(name):
    if name in __all__:
        return getattr(importlib.import_module(__name__ + ".solver"), name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
