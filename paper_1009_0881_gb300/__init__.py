"""GB300-native multilevel NMF (Gillis & Glineur, arXiv:1009.0881).

The compute path is the C-ABI shared library built from ``csrc/`` (see
``include/nmf.h``); ``native`` is a thin ctypes binding with the same entry
point names.  Importing this package does not load the library; the first call
through ``native`` does, and raises if it is missing.
"""
__all__ = ["native", "synth"]
