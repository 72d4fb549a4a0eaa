"""GB300-native batched NDGSBP decoding of LDPC codes.

Importing the package is cheap: ``inputs`` (seeded problem generators) has no native
dependency, and the CUDA library binding ``ndgsbp`` is loaded only when it is imported.
"""
__all__ = ["inputs", "ndgsbp"]
