"""B300 (sm_103a) FX-correlator X-engine.

The engine itself is the C-ABI library ``libxengine.so`` (include/xengine.h)
built from ``csrc/``; :mod:`paper_1708_00720_b300.xengine` is its thin Python
binding.  Importing this package does not load the library; importing
``paper_1708_00720_b300.xengine`` does, and raises if it cannot.
"""
__all__ = ["xengine", "build"]
