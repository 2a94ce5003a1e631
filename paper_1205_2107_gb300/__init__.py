"""GB300-native MRRR eigensolver for real symmetric tridiagonal matrices (FP64).

The compute path is the CUDA shared library built from ``csrc/``; this package
only marshals arguments to its C ABI (``include/mrrr.h``).
"""
