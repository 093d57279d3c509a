"""GB300-native retarded scalar/vector potentials for multi-domain TDDFT.

The compute path is a CUDA library (``csrc/``, sm_103a) behind the C-ABI in
``include/rp.h``; ``rp`` is its thin Python binding.  Importing the package
does not load the library: ``rp.load()`` does, and fails loudly if it is
missing.
"""
__all__ = ["synth", "rp"]
