"""GB300-native Cartesian FMM operators for the 1/r kernel (arXiv:1811.06332).

The compute path is the CUDA library ``libfmm_gb300.so`` (C-ABI declared in
``include/fmm_gb300.h``); ``paper_1811_06332_gb300.fmm`` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library
on first use and raises if it is missing.
"""
