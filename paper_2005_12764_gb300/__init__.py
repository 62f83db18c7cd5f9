"""GB300-native two-component colour-gradient lattice Boltzmann step (D3Q19).

The compute path lives in the CUDA library ``liblbm.so`` (sources in ``csrc/``,
C-ABI in ``include/lbm.h``); :mod:`paper_2005_12764_gb300.lbm` is its thin ctypes
binding. Importing this package does not load the library; nothing here falls back
to CPU arithmetic.
"""
__all__ = ["lbm", "inputs"]
