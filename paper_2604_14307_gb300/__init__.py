"""GB300-native MPCD with rigid-body discrete-particle colloids (arXiv 2604.14307).

The time step runs as hand-written sm_103a CUDA kernels behind the C ABI of
``include/mpcd.h`` (library ``libmpcd.so``); :mod:`.binding` is the thin ctypes
layer over it and :mod:`.inputs` builds seeded synthetic systems.  Importing
this package loads nothing: the CUDA library is loaded on first use and a
missing or unloadable library raises instead of falling back to anything else.
"""
__all__ = ["inputs", "binding"]
