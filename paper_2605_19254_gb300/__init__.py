"""GB300-native exact integer matrix product in the Residue Number System.

The compute lives in ``libsmf.so`` (CUDA kernels for sm_103a behind a C ABI,
declared in ``include/smf.h``); ``smf`` is the thin ctypes binding.  Importing
this package does not load the library; ``smf.lib()`` does, and fails loudly
when it has not been built.
"""
