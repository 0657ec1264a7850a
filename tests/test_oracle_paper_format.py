"""Pins of the paper-faithful format in the oracle (Sec. 3.3, 3.4, 3.6): the
mapping factor and Eq. 3 in closed form, the byte quantiser's extremes and
error bound, records and BlockEnd pointers against a per-coefficient loop,
identical frames leaving the inter-frame detail packages empty, and the
decode error on the equator rows."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import paper_format as PF
import synth


def test_mapping_factor_closed_form():
    H = PF.mapping_factor(8)
    assert H[0] == 1.0
    assert H[4] == pytest.approx(0.0, abs=1e-15)          # the equator row
    np.testing.assert_allclose(H, 1 - np.sin(math.pi * np.arange(8) / 8))


def test_threshold_map_follows_eq3():
    T = PF.threshold_map(64, 32, 3, 0.4)
    # LL_3 (8 x 4): l = l_max, the level term is 0 and H applies to details only
    np.testing.assert_array_equal(T[:4, :8], 0.0)
    # HL_3 (8 x 4): alpha ((3 - 3) / 3)^2 + H = H
    np.testing.assert_allclose(T[:4, 8:16], np.repeat(PF.mapping_factor(4)[:, None], 8, 1))
    # HH_1 (32 x 16): alpha ((3 - 1) / 3)^2 + H
    np.testing.assert_allclose(T[16:, 32:], 0.4 * (2 / 3) ** 2 + np.repeat(PF.mapping_factor(16)[:, None], 32, 1))
    # HL_2: alpha (1/3)^2 + H
    np.testing.assert_allclose(T[:8, 16:32], 0.4 / 9 + np.repeat(PF.mapping_factor(8)[:, None], 16, 1))


def test_temporal_threshold_map_closed_form():
    k = 2
    # the low band (j = 0): level term alpha_t ((k - k) / k)^2 = 0 everywhere
    np.testing.assert_array_equal(PF.temporal_threshold_map(64, 32, 3, 0.3, 0, k), 0.0)
    # a detail frame of temporal level j = 1: alpha_t ((2 - 1) / 2)^2, plus H on
    # the spatial detail bands, none on the approximation area
    T = PF.temporal_threshold_map(64, 32, 3, 0.3, 1, k)
    np.testing.assert_allclose(T[:4, :8], 0.3 / 4)
    np.testing.assert_allclose(T[16:, 32:], 0.3 / 4 + np.repeat(PF.mapping_factor(16)[:, None], 32, 1))


def test_constant_frames_survive_at_every_row():
    """A constant frame has energy in the approximation band only; with H on
    the detail bands only, it decodes to itself at every row, the poles
    included (H = 1 there would otherwise zero it)."""
    frames = [(np.full((64, 64), 200, np.uint8), np.full((32, 32), 90, np.uint8),
               np.full((32, 32), 160, np.uint8))] * 4
    pp = PF.PaperParams(64, 64, 3, 1, 3, 4, 2, alpha=0.25, alpha_t=0.005)
    st = PF.PaperStream(PF.encode(frames, pp))
    for f in range(4):
        for pl, v in enumerate((200, 90, 160)):
            x, u8 = st.decode_plane(f, pl)
            # the extremes are stored as float32: a rounding of ~1e-7 relative remains
            assert np.abs(x - v).max() < 1e-3, (f, pl, np.abs(x - v).max())


def test_byte_quantiser_extremes_and_error():
    rng = np.random.default_rng(0)
    c = rng.normal(0, 0.2, (16, 16))
    keep = np.abs(c) > 0.1
    approx = PF.approx_mask(16, 16, 2)
    codes, ext = PF.quantize_bytes(np.where(keep, c, 0), keep, approx)
    for cls, (lo, hi) in zip((approx, ~approx), ext):
        sel = keep & cls
        assert lo == c[sel].min() and hi == c[sel].max()
        assert codes[sel].min() == 0 and codes[sel].max() == 255
    d = PF.dequantize_bytes(codes, keep, approx, ext)
    assert np.all(d[~keep] == 0)
    for cls, (lo, hi) in zip((approx, ~approx), ext):
        sel = keep & cls
        assert np.abs(d[sel] - c[sel]).max() <= (hi - lo) / 510 + 1e-12


def _loop_reference(frame, pp):
    """Coefficients one frame of a set of one (tlevels 0) must decode to, by a
    plain loop over coefficients: Eq. 3 per coefficient, byte quantisation."""
    p = pp.codec()
    x = (frame.astype(np.float64) - 128) / 255
    c = O.fwd2d(x, pp.levels, O.WAVELET_97)
    h, w = c.shape
    keep = np.zeros_like(c, bool)
    for (name, lev, x0, y0, sw, sh) in O.subbands(w, h, pp.levels):
        l = pp.levels if name == "LL" else lev
        for yy in range(sh):
            # H(y) on the detail bands; the approximation band keeps the level term
            H = 0.0 if name == "LL" else 1 - math.sin(math.pi * yy / sh)
            T = pp.alpha * ((pp.levels - l) / pp.levels) ** 2 + H
            for xx in range(sw):
                keep[y0 + yy, x0 + xx] = abs(c[y0 + yy, x0 + xx]) > T
    approx = np.zeros_like(keep)
    approx[:h >> pp.levels, :w >> pp.levels] = True
    out = np.zeros_like(c)
    for cls in (approx, ~approx):
        sel = keep & cls
        if np.any(sel):
            lo, hi = c[sel].min(), c[sel].max()
            q = np.floor((c[sel] - lo) / (hi - lo) * 255 + 0.5)
            out[sel] = lo + q / 255 * (hi - lo)
    return out


def test_records_decode_to_the_loop_reference():
    fr = synth.gradient_rects_frame(64, seed=3)
    pp = PF.PaperParams(64, 64, 1, 0, 3, 1, 0, alpha=0.02, alpha_t=0.0)
    st = PF.PaperStream(PF.encode([(fr,)], pp))
    np.testing.assert_allclose(st.coef_plane(0, 0), _loop_reference(fr, pp), rtol=0, atol=1e-6)
    ext, ends, recs = st.frame_package(0)
    assert np.all(np.diff(ends.astype(np.int64)) >= 0) and int(ends[-1]) == len(recs)
    assert np.all((recs & 0xFFFF) < 32 * 32) and np.all((recs >> 16) < 256)


def test_identical_frames_leave_detail_packages_empty():
    fr = synth.gradient_rects_frame(64, seed=4)
    pp = PF.PaperParams(64, 64, 1, 0, 3, 4, 2, alpha=0.01, alpha_t=0.005)
    st = PF.PaperStream(PF.encode([(fr,)] * 4, pp))
    counts = [len(st.frame_package(t)[2]) for t in range(4)]
    assert counts[0] > 0 and counts[1:] == [0, 0, 0]
    for f in range(4):
        np.testing.assert_array_equal(st.decode_plane(f, 0)[1], st.decode_plane(0, 0)[1])


def test_equator_rows_decode_close_to_the_source():
    """With small constants the only loss near the equator is the byte
    quantiser (H ~ 0 there): the middle rows stay within a few levels."""
    frames = synth.equirect_gop(128, 4, seed=5, n_discs=4)
    pp = PF.PaperParams(128, 128, 3, 1, 3, 4, 2, alpha=0.0, alpha_t=0.0)
    st = PF.PaperStream(PF.encode(frames, pp))
    for f in (0, 3):
        x, u8 = st.decode_plane(f, 0)
        mid = slice(56, 72)
        err = np.abs(x[mid] - frames[f][0][mid].astype(np.float64))
        assert err.mean() < 2.0, err.mean()
        # near the poles H ~ 1 zeroes the details: the top rows are much smoother
        assert np.abs(x[:4] - frames[f][0][:4]).mean() > err.mean()
