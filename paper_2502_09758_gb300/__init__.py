"""GB300-native (sm_103a) hot path of ADP-beta solved by MAID (arXiv 2502.09758).

The compute lives in ``libadp.so`` (hand-written CUDA behind a C ABI declared in
``include/adp.h``); :mod:`paper_2502_09758_gb300.adp` is the thin ctypes binding
with the same names.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["adp", "synth"]
