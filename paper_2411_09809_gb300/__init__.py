"""gr: exact graph-layout readability metrics on one GB300 (arXiv 2411.09809).

The metrics run in the CUDA library ``libgr.so`` (hand-written sm_103a kernels
behind a C ABI declared in ``include/gr.h``); :mod:`.gr` is its thin ctypes
binding and :mod:`.synth` draws seeded synthetic layouts.  Importing this package
loads nothing; the library is loaded on first use and the binding raises if it
is missing -- there is no CPU fallback.
"""
