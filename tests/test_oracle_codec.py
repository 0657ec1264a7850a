"""Pins of the oracle's inter-frame Haar, quantiser, stream format and
dependency cone (CPU only)."""
import os
import struct

import numpy as np
import pytest

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_haar_float_worked_example():
    """Sec. 3.2: one frame of a set is L plus log2(n) details times -1 or +1.
    x = 1 5 2 10 (n = 4) by hand: L1 = 3 6, H1 = 2 4, L2 = 4.5, H2 = 1.5."""
    x = [np.array(v, float) for v in (1.0, 5.0, 2.0, 10.0)]
    bands = O.haar_forward(x, 2, integer=False)
    assert [float(b) for b in bands] == [4.5, 1.5, 2.0, 4.0]
    # frame 2: +H2 (second half), -H1[1] (first of its pair) -> 4.5 + 1.5 - 4
    for f in range(4):
        need = O.haar_needed_slots(2, f)
        got = O.haar_inverse([bands[s] for (s, _, _) in need], 2, f, integer=False)
        assert float(got) == float(x[f])
    assert [s for (s, _, _) in O.haar_needed_slots(2, 2)] == [0, 1, 3]


def test_haar_integer_s_transform():
    """S-transform: H = b - a, L = a + floor(H/2) = floor((a+b)/2); the
    inverse is exact."""
    rng = np.random.default_rng(0)
    for k in (1, 2, 3):
        n = 1 << k
        fr = [rng.integers(-500, 500, (5, 7)) for _ in range(n)]
        bands = O.haar_forward(fr, k, integer=True)
        if k == 1:
            np.testing.assert_array_equal(bands[0], np.floor_divide(fr[0] + fr[1], 2))
            np.testing.assert_array_equal(bands[1], fr[1] - fr[0])
        for f in range(n):
            need = O.haar_needed_slots(k, f)
            got = O.haar_inverse([bands[s] for (s, _, _) in need], k, f, integer=True)
            np.testing.assert_array_equal(got, fr[f])


def test_dequantizer_closed_form():
    q = np.array([-3, -1, 0, 1, 2])
    np.testing.assert_allclose(O.dequantize(q, 4.0, False), [-14, -6, 0, 6, 10])
    np.testing.assert_array_equal(O.dequantize(q, 1, True), q)
    np.testing.assert_array_equal(O.dequantize(q, 3, True), [-10, -4, 0, 4, 7])


def test_quantizer_error_bound():
    rng = np.random.default_rng(1)
    c = rng.normal(0, 30, 10000)
    for step in (0.5, 4.0, 7.25):
        q = O.quantize(c, step, False)
        r = O.dequantize(q, step, False)
        big = np.abs(c) >= step
        assert np.all(np.abs(c - r)[big] <= step / 2 + 1e-12)
        assert np.all(q[~big] == 0) and np.all(r[~big] == 0)


def test_lossless_round_trip_53():
    """5/3 at step 1 reproduces the frames bit for bit, gray and YCbCr, with
    and without inter-frame sets."""
    img = synth.gradient_rects_frame(128, seed=1)
    p = O.Params(128, 128, 1, 0, 3, O.WAVELET_53, 1, 0, 32, 1.0)
    st = O.Stream(O.encode([(img,)], p))
    np.testing.assert_array_equal(O.decode_plane(st, 0, 0)[1], img)
    fr = synth.equirect_gop(128, 4, seed=4, n_discs=5)
    for k in (1, 2):
        p = O.Params(128, 128, 3, 1, 3, O.WAVELET_53, 4, k, 32, 1.0)
        st = O.Stream(O.encode(fr, p))
        for f in range(4):
            for pl in range(3):
                np.testing.assert_array_equal(O.decode_plane(st, f, pl)[1], fr[f][pl])


def test_lossy_97_error_within_quantiser_bound():
    """9/7 with a small step: every sample is within the synthesis gain times
    the dead-zone bound (step per coefficient, two temporal bands)."""
    fr = synth.equirect_gop(64, 2, seed=6, n_discs=3)
    p = O.Params(64, 64, 3, 1, 3, O.WAVELET_97, 2, 1, 16, 0.01)
    st = O.Stream(O.encode(fr, p))
    for f in range(2):
        for pl in range(3):
            x, u8 = O.decode_plane(st, f, pl)
            assert np.abs(x - fr[f][pl]).max() < 0.25
            assert np.abs(u8.astype(int) - fr[f][pl]).max() <= 1


def test_all_zero_blocks_are_omitted():
    """A constant frame has only its LL block(s) stored (Sec. 3.4 loads only
    blocks that hold coefficients)."""
    img = np.full((64, 64), 200, np.uint8)
    p = O.Params(64, 64, 1, 0, 2, O.WAVELET_97, 1, 0, 16, 1.0)
    st = O.Stream(O.encode([(img,)], p))
    present = [O.block_list(p)[b][1] for b in np.nonzero(st.table[0] >= 0)[0]]
    assert present == ["LL"] * 1
    np.testing.assert_array_equal(O.decode_plane(st, 0, 0)[1], img)


def test_block_order_level_wise_from_lowest_frequency():
    p = O.Params(64, 64, 1, 0, 2, O.WAVELET_97, 1, 0, 16, 1.0)
    names = [(b[1], b[2]) for b in O.block_list(p)]
    order = []
    for nm in names:
        if not order or order[-1] != nm:
            order.append(nm)
    assert order == [("LL", 2), ("HL", 2), ("LH", 2), ("HH", 2), ("HL", 1), ("LH", 1), ("HH", 1)]
    assert len(names) == 1 + 3 + 12


def test_stream_header_rejects_corruption():
    img = synth.gradient_rects_frame(32, seed=2)
    p = O.Params(32, 32, 1, 0, 2, O.WAVELET_53, 1, 0, 16, 1.0)
    b = bytearray(O.encode([(img,)], p))
    with pytest.raises(ValueError):
        O.Stream(bytes(b[:40]))
    bad = bytearray(b)
    bad[0:4] = b"XXXX"
    with pytest.raises(ValueError):
        O.Stream(bytes(bad))
    bad = bytearray(b)
    toff = struct.unpack_from("<Q", b, 72)[0]
    struct.pack_into("<i", bad, toff, 99)
    with pytest.raises(ValueError):
        O.Stream(bytes(bad))


@pytest.mark.parametrize("wavelet,levels", [(O.WAVELET_53, 2), (O.WAVELET_97, 2), (O.WAVELET_97, 3)])
def test_cone_contains_every_influencing_coefficient(wavelet, levels):
    """Brute force: perturb each coefficient of a small plane, run the full
    iFWT, and record which coefficients change any pixel of a region; all of
    them must lie in the oracle's cone of that region (Sec. 3.1 masked iFWT)."""
    n = 32
    rng = np.random.default_rng(11 + wavelet + levels)
    base = rng.integers(-50, 50, (n, n)) if wavelet == O.WAVELET_53 else rng.normal(0, 20, (n, n))
    ref = O.inv2d(base, levels, wavelet)
    for region in [(5, 9, 11, 14), (0, 4, 28, 32), (30, 32, 0, 3)]:
        r0, r1, c0, c1 = region
        R = np.zeros((n, n), bool)
        R[r0:r1, c0:c1] = True
        need = O.cone(R, levels, wavelet)
        full = np.zeros((n, n), bool)
        for (name, lev, x0, y0, sw, sh) in O.subbands(n, n, levels):
            full[y0:y0 + sh, x0:x0 + sw] = need[(name, lev)]
        influencing = np.zeros((n, n), bool)
        for y in range(n):
            for x in range(n):
                pert = base.copy()
                pert[y, x] += 64
                out = O.inv2d(pert, levels, wavelet)
                influencing[y, x] = np.any(np.abs(out - ref)[R] > 1e-9)
        assert not np.any(influencing & ~full)
        # the cone is tight up to the halo: most of it really influences R
        assert influencing.sum() >= 0.6 * full.sum()


@pytest.mark.parametrize("wavelet", [O.WAVELET_53, O.WAVELET_97])
def test_decoding_only_the_cone_reproduces_the_region(wavelet):
    """Zeroing every coefficient outside the cone leaves the masked region of
    the reconstruction unchanged (bit-exact for 5/3)."""
    n, levels = 64, 3
    rng = np.random.default_rng(5)
    c = rng.integers(-40, 40, (n, n)) if wavelet == O.WAVELET_53 else rng.normal(0, 20, (n, n))
    R = synth.random_cell_mask(8, 8, seed=9, density=0.2)
    Rp = O.cell_mask_to_pixels(R, n, n)
    need = O.cone(Rp, levels, wavelet)
    full = np.zeros((n, n), bool)
    for (name, lev, x0, y0, sw, sh) in O.subbands(n, n, levels):
        full[y0:y0 + sh, x0:x0 + sw] = need[(name, lev)]
    a = O.inv2d(c, levels, wavelet)
    b = O.inv2d(np.where(full, c, 0), levels, wavelet)
    if wavelet == O.WAVELET_53:
        np.testing.assert_array_equal(a[Rp], b[Rp])
    else:
        assert np.abs(a - b)[Rp].max() < 1e-9


def test_table1_mean_is_the_abstract_193fps():
    rows = []
    with open(os.path.join(GOLD, "table1_display_fps.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(v) for v in line.split()[1:]])
    hq = np.array(rows)[:, 4]
    assert abs(hq.mean() - 192.74) < 0.01 and round(hq.mean()) == 193
