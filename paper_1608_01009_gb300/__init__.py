"""GB300-native particle-in-cell hot path (arXiv:1608.01009's PIC cycle).

The compute runs in the CUDA library ``libpicgb.so`` (C ABI in include/pic.h);
``paper_1608_01009_gb300.pic`` is the thin ctypes binding over it.  Importing
this package loads nothing; the binding loads the library on first use and
raises if it has not been built.
"""
__all__ = ["pic", "workloads"]
