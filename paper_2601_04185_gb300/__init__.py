"""ImLoc localization hot path (lift + LO-RANSAC PnP) for GB300 (sm_103a).

The compute lives in ``libimloc.so`` (hand-written CUDA kernels behind a C ABI,
declared in ``include/imloc.h``); :mod:`paper_2601_04185_gb300.imloc` is the thin
ctypes binding and :mod:`paper_2601_04185_gb300.synth` makes seeded inputs.
"""
__all__ = ["imloc", "synth"]
