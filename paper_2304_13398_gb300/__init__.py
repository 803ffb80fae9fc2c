"""GB300-native timing-aware 4-value gate-level re-simulation (arXiv 2304.13398).

The compute path is libgls.so (hand-written CUDA for sm_103a behind the C-ABI
in include/gls.h); this package holds its build script and a thin ctypes
binding with the same names.
"""
from .gls import (CELLS, Context, GlsError, RunStats, cell_table, check_netlist, check_stimulus,  # noqa: F401
                  load_library, unpack)
