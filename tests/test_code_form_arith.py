"""The arithmetic the tile decoder relies on for 9/7 dead-zone codes held
on the device as t = 2q + sign(q), checked exhaustively over int16 on the
CPU (float32 emulated with numpy):

* t * step / 2 is the dead-zone midpoint reconstruction sign(q)(|q| + 1/2)
  step (0 for q = 0);
* for |q| <= 8191 the pair L +- H of two such codes fits a 16-bit lane;
* a 16-bit value, biased by 2^15 and placed in the low mantissa bits of 2^23,
  minus 2^23 + 2^15 gives that value exactly as a float32."""
import numpy as np


def test_midpoint_reconstruction_identity():
    q = np.arange(-32768, 32768, dtype=np.int64)
    t = 2 * q + np.sign(q)
    step = 4.0
    np.testing.assert_array_equal(t * step / 2, np.sign(q) * (np.abs(q) + 0.5) * step)


def test_band_pair_fits_16_bits():
    q = np.arange(-8191, 8192, dtype=np.int64)
    t = 2 * q + np.sign(q)
    assert t.max() + t.max() <= 32767 and t.min() + t.min() >= -32768
    assert t.max() - t.min() <= 32767


def test_mantissa_placement_is_exact():
    v = np.arange(-32768, 32768, dtype=np.int32)
    bits = (0x4B000000 | ((v.astype(np.uint32) ^ 0x8000) & 0xFFFF)).astype(np.uint32)
    f = bits.view(np.float32) - np.float32(8421376.0)
    assert f.dtype == np.float32
    np.testing.assert_array_equal(f, v.astype(np.float32))
