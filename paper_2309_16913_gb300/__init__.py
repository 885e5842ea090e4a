"""GB300 (sm_103a) R-tree range select and spatial join.

The compute path is the CUDA library ``librtree.so`` built from ``csrc/``;
:mod:`paper_2309_16913_gb300.rtree` is a thin ctypes binding over its C ABI
(``include/rtree.h``).  :mod:`paper_2309_16913_gb300.datagen` draws the seeded
synthetic inputs.  Importing this package loads nothing; the library is loaded
on first use and a missing library is an error, never a fallback.
"""
__all__ = ["datagen", "rtree"]
