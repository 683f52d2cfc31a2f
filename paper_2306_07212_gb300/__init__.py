"""GB300-native polyhedral-complex extraction from ReLU networks by edge subdivision.

The compute path is the CUDA library ``libpc.so`` (C ABI in ``include/pc.h``);
this package holds its thin ctypes binding, the build script and the seeded
workload generators.
"""
from .binding import Extractor, PcError, load_library  # noqa: F401
from . import workloads  # noqa: F401
