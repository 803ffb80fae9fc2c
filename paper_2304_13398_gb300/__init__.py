"""GB300-native timing-aware 4-value gate-level re-simulation (arXiv 2304.13398).

The compute path is libgls.so (hand-written CUDA for sm_103a behind the C-ABI
in include/gls.h); this package holds its build script and a thin ctypes
binding with the same names.
"""
from .gls import (CELLS, Context, GlsError, RunStats, check_netlist, check_stimulus, load_library,  # noqa: F401
                  unpack)
