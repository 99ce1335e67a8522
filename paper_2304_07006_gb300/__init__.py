"""GB300-native grid-quadrature build of the xTC corrections (arXiv 2304.07006).

The compute path lives in the CUDA library ``libxtc.so`` (C ABI in ``include/xtc.h``);
``paper_2304_07006_gb300.xtc`` is its ctypes binding.
"""
from .xtc import Context, XtcError, load, unpack_pairs, pair_index, PRECISIONS  # noqa: F401
