"""GB300-native SIP-DG Stokes solver library (arXiv 1607.03777 hot path).

The compute path is the CUDA library ``libsipstokes.so`` behind the C ABI
of ``include/sipstokes.h``; ``api`` is its thin Python binding and
``synth`` the seeded synthetic-input generators.
"""
__all__ = ["api", "synth", "build"]
