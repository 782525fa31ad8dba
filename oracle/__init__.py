"""FP64 CPU oracle for the direct FFT pressure solve.

Test infrastructure only: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference arm of ``bench.py``; never by the product
path.  See ``poisson_oracle`` for the definitions and their sources.
"""
from .poisson_oracle import *  # noqa: F401,F403
from .poisson_oracle import __all__  # noqa: F401
