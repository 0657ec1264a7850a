// codes.cuh -- device helpers shared by the tile decoders (ifwt.cu, strip.cu):
// the CDF 9/7 lifting constants, int16 code unpacking and the subband index
// of a symmetrically extended interleaved line.
#pragma once

#include "wv_impl.h"

namespace wv {

// CDF 9/7 lifting factorisation (Daubechies & Sweldens 1998; JPEG2000 Part 1
// irreversible wavelet): analysis lifts with alpha, beta, gamma, delta and
// scales the low band by 1/K and the high band by K.
constexpr float kAlpha = -1.586134342059924f;
constexpr float kBeta = -0.052980118572961f;
constexpr float kGamma = 0.882911075530934f;
constexpr float kDelta = 0.443506852043971f;
constexpr double kK = 1.230174104914001;

__device__ __forceinline__ int lo16(uint32_t w) { return (int)(int16_t)(w & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t w) { return (int)(int16_t)(w >> 16); }

// Both int16 halves of a word as floats, exactly and without a conversion
// instruction: each half, biased to unsigned (v + 2^15), becomes the low
// mantissa bits of 2^23, and 2^23 + 2^15 is subtracted.
__device__ __forceinline__ void halves_to_float(uint32_t w, float &lo, float &hi) {
    const uint32_t x = w ^ 0x80008000u;
    lo = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7610)) - 8421376.0f;
    hi = __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7632)) - 8421376.0f;
}

// reflect_idx with a branch for the common case of an index inside [0, n).
__device__ __forceinline__ int refl(int i, int n) {
    return (unsigned)i < (unsigned)n ? i : reflect_idx(i, n);
}

// Index of coefficient k of a subband of n coefficients after whole-sample
// symmetric extension of the interleaved line (low band: even positions,
// high band: odd positions).
__device__ __forceinline__ int refl_sub(int k, int n, int high) {
    return reflect_idx(2 * k + high, 2 * n) >> 1;
}

}  // namespace wv
