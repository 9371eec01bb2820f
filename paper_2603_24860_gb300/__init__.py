"""GB300-native symmetry-reduced Bethe-Salpeter block builder.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/bse.h``); :mod:`paper_2603_24860_gb300.bse` is its ctypes binding.
"""
from . import bse  # noqa: F401
