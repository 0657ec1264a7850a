"""Pins of the oracle's wavelet transforms (CPU only).

Each test checks the oracle against something other than itself: published
filter taps, a hand-worked example, a library matrix inverse, closed forms of
constant and alternating signals, and perfect reconstruction."""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _taps():
    h = {"h0": {}, "h1": {}}
    with open(os.path.join(GOLD, "cdf97_analysis_taps.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, off, val = line.split()
            h[name][int(off)] = float(val)
    return h


def _sym_filter(taps: dict) -> dict:
    out = {}
    for k, v in taps.items():
        out[k] = v
        out[-k] = v
    return out


def _reflect(i, n):
    period = 2 * (n - 1)
    i = i % period
    return period - i if i >= n else i


def test_97_analysis_matches_published_taps_interior():
    """Impulse responses of the oracle's lifting analysis are the published
    CDF 9/7 analysis filters (JPEG2000 normalisation)."""
    h = _taps()
    h0, h1 = _sym_filter(h["h0"]), _sym_filter(h["h1"])
    n = 64
    for i0 in (30, 31):
        e = np.zeros(n)
        e[i0] = 1.0
        c = O.fwd1d(e, O.WAVELET_97)
        s, d = c[:n // 2], c[n // 2:]
        for k in range(8, 24):
            # s[k] = sum_i h0[2k - i] x[i],  d[k] = sum_i h1[2k + 1 - i] x[i]
            assert abs(s[k] - h0.get(2 * k - i0, 0.0)) < 1e-10
            assert abs(d[k] - h1.get(2 * k + 1 - i0, 0.0)) < 1e-10


def test_97_lifting_equals_convolution_with_symmetric_extension():
    """The whole analysis (boundaries included) equals the filter bank built
    from the published taps with whole-sample symmetric extension."""
    h = _taps()
    h0, h1 = _sym_filter(h["h0"]), _sym_filter(h["h1"])
    rng = np.random.default_rng(7)
    for n in (8, 10, 16, 32):
        x = rng.normal(0, 50, n)
        c = O.fwd1d(x, O.WAVELET_97)
        s_ref = [sum(h0[m] * x[_reflect(2 * k - m, n)] for m in h0) for k in range(n // 2)]
        d_ref = [sum(h1[m] * x[_reflect(2 * k + 1 - m, n)] for m in h1) for k in range(n // 2)]
        np.testing.assert_allclose(c[:n // 2], s_ref, atol=1e-9)
        np.testing.assert_allclose(c[n // 2:], d_ref, atol=1e-9)


def test_97_synthesis_is_matrix_inverse_of_analysis():
    """Synthesis matrix (from impulses) equals numpy.linalg.inv of the
    analysis matrix assembled from the published taps."""
    h = _taps()
    h0, h1 = _sym_filter(h["h0"]), _sym_filter(h["h1"])
    for n in (8, 16, 24):
        A = np.zeros((n, n))
        for k in range(n // 2):
            for m, v in h0.items():
                A[k, _reflect(2 * k - m, n)] += v
            for m, v in h1.items():
                A[n // 2 + k, _reflect(2 * k + 1 - m, n)] += v
        S = np.stack([O.inv1d(np.eye(n)[j], O.WAVELET_97) for j in range(n)], axis=1)
        np.testing.assert_allclose(S, np.linalg.inv(A), atol=1e-9)


def test_53_hand_worked_example():
    rows = {}
    with open(os.path.join(GOLD, "legall53_worked_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *vals = line.split()
            rows[k] = np.array([int(v) for v in vals])
    np.testing.assert_array_equal(O.fwd1d(rows["x"], O.WAVELET_53), rows["sd"])
    np.testing.assert_array_equal(O.inv1d(rows["sd"], O.WAVELET_53), rows["x"])


def test_53_equals_linear_legall_filters_without_rounding():
    """On inputs that are multiples of 8 the integer lifting does no rounding
    and equals the LeGall 5/3 filter bank: low (-1 2 6 2 -1)/8, high
    (-1 2 -1)/2 (JPEG2000 Part 1 reversible filter)."""
    rng = np.random.default_rng(3)
    lo = {0: 6 / 8, 1: 2 / 8, -1: 2 / 8, 2: -1 / 8, -2: -1 / 8}
    hi = {0: 1.0, 1: -0.5, -1: -0.5}
    for n in (6, 8, 16, 30):
        x = 8 * rng.integers(-16, 16, n)
        c = O.fwd1d(x, O.WAVELET_53)
        s_ref = [sum(v * x[_reflect(2 * k - m, n)] for m, v in lo.items()) for k in range(n // 2)]
        d_ref = [sum(v * x[_reflect(2 * k + 1 - m, n)] for m, v in hi.items()) for k in range(n // 2)]
        np.testing.assert_array_equal(c[:n // 2], s_ref)
        np.testing.assert_array_equal(c[n // 2:], d_ref)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 14, 64])
def test_1d_perfect_reconstruction(n):
    rng = np.random.default_rng(n)
    x = rng.integers(-300, 300, n)
    np.testing.assert_array_equal(O.inv1d(O.fwd1d(x, O.WAVELET_53), O.WAVELET_53), x)
    xf = rng.normal(0, 100, n)
    np.testing.assert_allclose(O.inv1d(O.fwd1d(xf, O.WAVELET_97), O.WAVELET_97), xf, atol=1e-10)


@pytest.mark.parametrize("size,levels", [(8, 1), (16, 3), (32, 2), (64, 5), (48, 4), (128, 6)])
def test_2d_perfect_reconstruction(size, levels):
    rng = np.random.default_rng(size * 10 + levels)
    h, w = size, size * 2 if size <= 32 else size
    x = rng.integers(-128, 128, (h, w))
    c = O.fwd2d(x, levels, O.WAVELET_53)
    np.testing.assert_array_equal(O.inv2d(c, levels, O.WAVELET_53), x)
    xf = rng.normal(0, 60, (h, w))
    cf = O.fwd2d(xf, levels, O.WAVELET_97)
    assert np.abs(O.inv2d(cf, levels, O.WAVELET_97) - xf).max() < 1e-10


@pytest.mark.parametrize("wavelet", [O.WAVELET_53, O.WAVELET_97])
def test_2d_constant_goes_to_LL_with_unit_gain(wavelet):
    """Low-pass DC gain 1 per axis and level: a constant frame leaves the
    constant in LL_L and zeros in every detail subband."""
    levels = 3
    x = np.full((32, 64), 37)
    c = O.fwd2d(x, levels, wavelet)
    ll = c[:32 >> levels, :64 >> levels]
    assert np.allclose(ll, 37, atol=1e-12)
    c2 = c.astype(float).copy()
    c2[:32 >> levels, :64 >> levels] = 0
    assert np.abs(c2).max() < 1e-12


def test_2d_subband_orientation():
    """A signal alternating along x only lands in HL_1 (top-right quadrant:
    horizontal high-pass, vertical low-pass) with gain 2 (Nyquist gain of
    the 9/7 high-pass); one alternating along y lands in LH_1."""
    h, w = 16, 16
    xs = np.tile((-1.0) ** np.arange(w), (h, 1)) * 10
    c = O.fwd2d(xs, 1, O.WAVELET_97)
    assert np.allclose(c[:8, 8:], c[0, 8], atol=1e-9) and abs(abs(c[0, 8]) - 20) < 1e-9
    c[:8, 8:] = 0
    assert np.abs(c).max() < 1e-9
    c = O.fwd2d(xs.T.copy(), 1, O.WAVELET_97)
    assert abs(abs(c[8, 0]) - 20) < 1e-9
    c[8:, :8] = 0
    assert np.abs(c).max() < 1e-9


def test_default_levels_and_mask_resolution_from_paper():
    """Sec. 3.1: l_max = log2(N/32) - 2 gives the 6 levels the paper found
    best for 8k, and the 256x256 mask for an 8k frame is a 32-pixel cell."""
    import math
    assert int(math.log2(8192 / 32)) - 2 == 6
    assert 8192 // O.CELL == 256
