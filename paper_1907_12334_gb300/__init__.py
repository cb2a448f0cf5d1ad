"""GB300-native MSG-MIMC hot path (arXiv:1907.12334): C-ABI CUDA library + thin binding.

Importing the package loads nothing; ``paper_1907_12334_gb300.msg`` loads the
CUDA library (and fails loudly if it is missing).
"""
