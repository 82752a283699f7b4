"""gtb: B300-native hdiff / vadv stencils (GT4Py paper, arXiv 2311.08322, Sec. 3.1).

The compute path is ``libgtb.so`` (hand-written CUDA for sm_103a behind a C ABI,
declared in ``include/gtb.h``); ``gtb`` is its thin ctypes binding.  Importing
this package does not load the library; the first call into ``gtb`` does, and
raises if the library is missing.
"""
