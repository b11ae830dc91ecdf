"""GB300-native pixel-level CKKS with cached encryption (arXiv 2409.03568, "iCHEETAH").

Submodules:
  ichee   -- ctypes binding of the C-ABI library libichee.so (CUDA kernels for sm_103a)
  inputs  -- seeded synthetic images and operation arguments (no cryptographic arithmetic)
  metrics -- MSE / PSNR (Sec. 4.3.2)
  build   -- compiles libichee.so in-tree with nvcc

Importing the package loads nothing; `from paper_2409_03568_gb300 import ichee` loads the
CUDA library and fails loudly if it has not been built.
"""
