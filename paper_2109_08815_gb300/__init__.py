"""Multiple-shooting SVGD over a differentiable planar articulated-body simulator.

GB300 (sm_103a) CUDA kernels behind a C-ABI shared library; this package is
the thin Python binding (``api``) plus the seeded synthetic workloads
(``workloads``).  Importing the package loads nothing; the CUDA library is
loaded on first use by ``api`` and raises if it is missing.
"""
__all__ = ["api", "workloads"]
