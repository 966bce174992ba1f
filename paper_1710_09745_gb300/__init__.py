"""GB300-native block-CGrQ solver for the even-odd improved-staggered normal
operator (arXiv:1710.09745).

The compute path is libblockcg.so (hand-written CUDA for sm_103a behind the
C ABI of include/blockcg.h).  This package only marshals arguments: it holds
device memory and streams through PyTorch and calls the library.  There is no
CPU fallback; without the built library every call raises.
"""
from .binding import BlockCG, BlockCGBatch, BlockCGError, load_library, PREC  # noqa: F401

__all__ = ["BlockCG", "BlockCGBatch", "BlockCGError", "load_library", "PREC"]
