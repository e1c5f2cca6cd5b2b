"""GB300-native HDD likelihood library (arXiv 1708.02207).

The C ABI (include/hdd.h, libhdd.so built by ``build.build()``) holds the whole
likelihood path in hand-written CUDA for sm_103a; ``hdd`` is its thin ctypes
binding.  Importing this package loads nothing; ``hdd.load_library()`` does.
"""
__all__ = ["build", "hdd"]
