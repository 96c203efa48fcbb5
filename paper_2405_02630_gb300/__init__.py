"""GB300-native quantum-kernel estimation for QSVMs (after arXiv 2405.02630).

The compute lives in ``libqsvm.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/qsvm.h``).  ``paper_2405_02630_gb300.qsvm`` is a thin ctypes
binding with the same names; importing this package does not load CUDA.
"""
__all__ = ["inputs", "qsvm"]
