"""GB300-native short-range P3M gravity (CONCEPT 1.0, arXiv:2112.01508, Section 2.1.3).

The compute path is the CUDA library ``libp3m_sr.so`` (C ABI in
``include/p3m_sr.h``), built by ``buildlib.build()``.  This package holds its
ctypes binding (``_native``), a torch-facing wrapper (``ShortRange``) and the
differentiable force / leapfrog built on the library's forward and adjoint
kernels (``autograd``).
"""
from .buildlib import build  # noqa: F401
from .shortrange import ShortRange, Stats  # noqa: F401

__all__ = ["build", "ShortRange", "Stats"]
