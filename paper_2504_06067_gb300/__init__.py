"""GB300-native NSGA-III environmental selection engine.

The compute path is the CUDA library ``libnsga3.so`` (hand-written sm_103a
kernels behind the C ABI declared in ``include/nsga3.h``).  The submodule
``native`` is a thin ctypes binding with the same entry-point names; it
raises on import if the library has not been built.  ``workloads`` draws the
seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads"]
