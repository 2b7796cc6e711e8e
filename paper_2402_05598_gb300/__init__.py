"""GB300-native FCG-NO: flexible conjugate gradients preconditioned by a Fourier neural
operator (Rudikov et al., arXiv 2402.05598), as a C-ABI CUDA library for sm_103a.

Submodules
- ``inputs``: seeded synthetic problems and weight blobs (no method arithmetic).
- ``fcgno``: ctypes binding of ``include/fcgno.h`` (loads ``libfcgno.so``; raises if absent).
- ``build``: compiles the CUDA sources in-tree.

Importing the package itself does not load the CUDA library.
"""
__version__ = "0.1.0"
