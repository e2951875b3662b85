"""GB300-native NURSD / SRSD operator for NLOS imaging (arXiv 2501.05244).

The compute lives in the CUDA library ``libnursd`` (``csrc/``, C ABI in
``include/nursd.h``); :mod:`paper_2501_05244_gb300.nursd` is its ctypes
binding.  Importing the package does not load the library; the first plan
does, and fails loudly if it has not been built.
"""
from .build import build  # noqa: F401
from .nursd import (EXPORTS, LIB_PATH, NursdError, Plan, load_library,  # noqa: F401
                    phasor_frequencies, status_string, subsample, upsample)
