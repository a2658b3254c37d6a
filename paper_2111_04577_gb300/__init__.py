"""GB300-native dual-resolution phase-field solver (arXiv 2111.04577).

The compute path is the CUDA library under ``csrc/`` behind a C ABI
(``include/dualpf.h``); ``binding`` marshals arguments to it with ctypes.
"""
