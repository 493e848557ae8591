"""GB300-native randomized XR-preconditioned CholeskyQR (rLU-/rQR-CholeskyQR).

The factorisation runs in the CUDA kernels of ``librxr.so`` (built by
``paper_2111_11148_gb300.build``) behind the C ABI declared in
``include/rxr.h``; ``paper_2111_11148_gb300.rxr`` is its thin Python binding.
Nothing is loaded at import time.
"""
__all__ = ["rxr", "inputs", "build"]
