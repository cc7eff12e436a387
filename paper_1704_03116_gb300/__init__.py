"""GB300-native DOPE ADMM hot path (Dolz, Ben Ayed, Desrosiers, arXiv 1704.03116).

The compute path is the CUDA shared library ``libdope.so`` built from
``csrc/`` (C-ABI declared in ``include/dope.h``); ``dope.py`` is the thin
ctypes binding with the same names.  Importing this package loads nothing;
``paper_1704_03116_gb300.dope`` loads the library and fails loudly if it is
missing.  ``inputs`` draws seeded synthetic instances.
"""
__all__ = ["inputs", "dope"]
