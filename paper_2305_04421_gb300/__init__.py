"""GB300 (sm_103a) solver for the heat-equation-constrained KKT system with the two-level
time-domain-decomposition Schur-complement preconditioner of arXiv 2305.04421.

The compute path is the CUDA library ``libkkt.so`` behind the C ABI of ``include/kkt.h``;
``kkt`` is its ctypes binding and ``build`` compiles it. Importing this package does not
load the library; the first call into ``kkt`` does, and raises if it is not built.
"""

__all__ = ["kkt", "build"]
