"""GB300-native short-range Lennard-Jones MD hot path (tinyMD, arXiv 2009.07400).

The compute path is hand-written CUDA for sm_103a behind a C ABI
(``include/md.h``); :mod:`paper_2009_07400_gb300.md` is a thin ctypes binding
over it.  Importing this package loads nothing: the shared library is loaded
on first use and the binding raises if it is missing.
"""
__all__ = ["md", "inputs"]
