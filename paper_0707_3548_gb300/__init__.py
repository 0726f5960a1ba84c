"""GB300-native tiled Householder QR and least squares.

The compute path is the CUDA library ``libtqr.so`` (hand-written sm_103a
kernels behind a C ABI, declared in ``include/tqr.h``); ``paper_0707_3548_gb300.tqr``
is its thin ctypes binding.  ``inputs`` holds the seeded synthetic input
generators.  Importing the package does not load the library; the binding
loads it on first use and raises if it is missing.
"""
