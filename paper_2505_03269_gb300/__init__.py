"""GB300 (sm_103a) tensor-core beamformer: Y = W X as a batched complex GEMM.

The compute path is the CUDA library ``libtcbf.so`` (C ABI in
``include/tcbf.h``); ``binding`` is its ctypes shim and ``api`` a small
torch-facing convenience layer on top of it.  Nothing here computes on the
CPU: without the built library or a GPU every call raises.
"""
from .binding import (FLAG_AUTO_LAYOUT, FLAG_FP8_BLOCK_SCALES, FLAG_FP8_FOUR_PRODUCTS, FLAG_FP8_HI_ONLY,  # noqa: F401
                      FLAG_INTERLEAVED_X,
                      FLAG_STACKED_X,
                      MODE_1BIT, MODE_FP8SPLIT, MODE_FP16, MODE_TF32, SRC_CF16, SRC_CF32, Plan, TcbfError,
                      load, status_string)

__all__ = ["Plan", "TcbfError", "load", "status_string", "MODE_FP16", "MODE_FP8SPLIT",
           "MODE_1BIT", "MODE_TF32", "SRC_CF16", "SRC_CF32", "FLAG_STACKED_X", "FLAG_FP8_HI_ONLY",
           "FLAG_FP8_FOUR_PRODUCTS", "FLAG_INTERLEAVED_X", "FLAG_FP8_BLOCK_SCALES",
           "FLAG_AUTO_LAYOUT"]
