"""CPU oracle for pixel-level CKKS with cached encryption (arXiv 2409.03568).

TEST INFRASTRUCTURE: the checker, never the product. Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference legs may import it. It shares no code with the CUDA
library under paper_2409_03568_gb300/.
"""
from .ckks import Oracle, Params, mse, psnr, llround, ID_POOL_BASE, ID_RADIX_BASE  # noqa: F401
