"""GB300-native Toeplitz-structured spatio-angular MMSE tomographic reconstructor.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI declared
in ``include/tomo.h``); ``tomo`` is its thin ctypes binding.  ``workloads``
holds the seeded synthetic inputs.  Importing the package loads nothing.
"""
