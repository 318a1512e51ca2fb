"""GB300-native space-time isogeometric solver for the monodomain equation
with the Rogers-McCulloch ionic model (Spline Upwind stabilization).

The compute path is libst.so (include/st.h): CUDA kernels for sm_103a behind
a C ABI.  This package holds the in-tree build script and a thin ctypes
binding; it has no CPU fallback.
"""

from ._lib import (Solver, footprint, load, make_desc, StError, wupdate_static,  # noqa: F401
                   ST_FP64, ST_MIXED, ST_PICARD, ST_NEWTON, EXPORTS,
                   ST_ERR_CAPACITY, ST_ERR_NAN, ST_ERR_NOT_CONVERGED, ST_WUPDATE_STATIC_CAPACITY)
