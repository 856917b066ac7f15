"""GB300-native CF4 spin-half / spin-one integrator (arXiv 2204.05586 method).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/spinsim.h``); :mod:`.spinsim` is its ctypes binding and
:mod:`.workloads` draws seeded synthetic requests.
"""
from . import workloads  # noqa: F401
