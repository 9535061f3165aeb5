"""GB300 (sm_103a) finite-element numerical integration for first-order elements.

The compute path is the CUDA library ``libfe.so`` built from ``csrc/`` (C ABI in
``include/fe.h``); ``api`` is its thin Python binding and ``meshgen`` the seeded
synthetic workloads. Importing this package loads nothing; the library is loaded
on first use by ``api`` and raises if it has not been built.
"""
__all__ = ["api", "meshgen"]
