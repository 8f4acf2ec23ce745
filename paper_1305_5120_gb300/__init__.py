"""GB300-native Chebyshev filtered subspace iteration for sequences of dense Hermitian
generalized eigenproblems (Berljafa & Di Napoli, arXiv:1305.5120).

The compute lives in the C-ABI library ``libchfsi.so`` (include/chfsi.h); ``chfsi`` is its
thin Python binding (argument marshalling only).  ``synth`` builds seeded inputs.
"""
__all__ = ["chfsi", "synth", "build"]
