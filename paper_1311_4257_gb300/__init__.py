"""GB300-native directional fast multipole matvec (arXiv:1311.4257).

The compute path is the CUDA library libdfmm.so (C ABI in include/dfmm.h);
this package holds its sources (csrc/), the build script and a thin ctypes
binding (dfmm.py).
"""
from .dfmm import Batch, Plan, DfmmError, Graph, Server, apply_batched, representation, lib  # noqa: F401
