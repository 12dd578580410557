"""GB300 (sm_103a) implementation of the A-DOT path-conservative scheme for the
1D de Saint Venant-Exner system (arXiv 1912.04791).

The compute path is the C-ABI library ``libadot.so`` (hand-written CUDA,
declared in ``include/adot.h``); :mod:`.adot` is its thin ctypes binding and
:mod:`.workloads` builds seeded synthetic inputs. Importing this package loads
nothing; the library is loaded on first use of :mod:`.adot` and raises if it is
missing (there is no CPU fallback).
"""
__all__ = ["adot", "workloads", "build"]
