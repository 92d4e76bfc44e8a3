"""GB300-native half-range finite-difference lattice Boltzmann solver.

The compute path is the CUDA library ``liblbm.so`` (sources in ``csrc/``,
C-ABI declared in ``include/lbm.h``); ``lbm`` is its thin ctypes binding.
Importing this package loads nothing; the first call into ``lbm`` loads the
library and raises if it has not been built.
"""
