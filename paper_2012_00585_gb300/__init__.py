"""GB300-native finite-element sparse-matrix assembly (arXiv 2012.00585).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/feasm.h``); ``feasm`` is its ctypes binding.
"""

from . import feasm  # noqa: F401
