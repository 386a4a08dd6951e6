"""GB300 (sm_103a) library for the DFPT screening hot path: chi0bar = v^1/2 chi0 v^1/2 applied by
Sternheimer solves, and its projective eigendecomposition (PDEP).

The compute lives in libwdf.so (CUDA kernels behind the C ABI of include/wdf.h); ``wdf`` is the
ctypes binding and ``build`` compiles the library in-tree.
"""

from .wdf import Context, NotConverged, Stats, WdfError, load  # noqa: F401

__all__ = ["Context", "NotConverged", "Stats", "WdfError", "load"]
