"""GB300-native P3M gravity of CONCEPT 1.0 (arXiv:2112.01508, Section 2.1.3).

The compute path is two CUDA libraries built by ``buildlib.build()``:
``libp3m_sr.so`` (short-range particle-particle force over tiles and subtiles,
rungs, kick, drift, adjoint; C ABI in ``include/p3m_sr.h``) and
``libp3m_pm.so`` (long-range particle-mesh force; ``include/p3m_pm.h``).  This
package holds their ctypes binding (``_native``), torch-facing wrappers
(``ShortRange``, ``LongRange``), the differentiable force / leapfrog built on the
forward and adjoint kernels (``autograd``), the rung-based leapfrog
(``integrate``), the timed subtile refinement (``refine``) and the slab
decomposition over ranks with its halo exchange (``slabs``).
"""
from .buildlib import build  # noqa: F401
from .longrange import LongRange, PMStats  # noqa: F401
from .shortrange import ShortRange, Stats  # noqa: F401

__all__ = ["build", "ShortRange", "Stats", "LongRange", "PMStats"]
