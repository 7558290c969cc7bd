"""GB300-native cell-graph construction (sign vectors, cells, Hamming-1 edges).

The compute path is the CUDA library ``libcellgraph.so`` (sources in ``csrc/``,
C-ABI in ``include/cellgraph.h``); ``cellgraph`` is its ctypes binding. Importing
this package loads nothing; the library is loaded on first use and a missing or
unloadable library raises instead of falling back to any CPU code.
"""

__all__ = ["inputs", "cellgraph"]
