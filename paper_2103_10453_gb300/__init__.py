"""GB300-native (sm_103a) hot path of MPMA for partial Latin square extension
(Goudet & Hao, arXiv 2103.10453).  The compute lives in hand-written CUDA kernels
behind the C ABI declared in ``include/plse.h``; ``plse`` is the thin ctypes
binding to that library.  Importing this package loads nothing; the CUDA library
is opened on first use by ``paper_2103_10453_gb300.plse``.
"""
