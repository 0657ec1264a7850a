"""GB300-native viewport-dependent wavelet video decoder.

The decoder (libwv.so, CUDA for sm_103a) sits behind the C ABI declared in
include/wv.h; ``wv`` is its Python binding.  It implements the hot path of
Groth et al., "Wavelet-Based Fast Decoding of 360 deg Videos": viewport
footprint, coefficient gather and dequantisation, inverse inter-frame Haar,
fused multi-level inverse wavelet transform, reprojection and colour.
"""
from . import wv  # noqa: F401
from .wv import Stream, decode_batch, encode, query  # noqa: F401

__all__ = ["wv", "Stream", "decode_batch", "encode", "query"]
