"""GB300-native PSATD Maxwell push (arXiv:1812.07357's local / hybrid FFT
solver, batched on one GPU).

The compute path is libpsatd.so (CUDA, sm_103a) behind the C ABI of
include/psatd.h; ``_abi`` binds it with ctypes and ``solver.Plan`` adds
numpy/torch packing helpers.  ``inputs`` holds the seeded synthetic
workloads.  Importing the package does not load the library; the first call
that needs it raises if it is missing.
"""
__all__ = ["inputs", "build", "_abi", "solver"]
