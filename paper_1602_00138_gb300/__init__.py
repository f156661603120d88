"""GB300-native inner-outer recycled Krylov solves for DOT reduced-order models.

The compute path is the CUDA library librcg (C ABI in include/rcg.h); the
Python module `rcg` is its ctypes binding.  Importing this package does not
load the library; `from paper_1602_00138_gb300 import rcg` does.
"""
