"""Pins of the oracle's projection, footprint, bilinear resampling and colour
conversion (CPU only)."""
import math

import numpy as np
import pytest

import oracle as O


def test_projection_centre_and_yaw_pitch_shifts():
    """A 3x3 viewport's centre pixel looks along the view axis: yaw 0, pitch
    0 hits the frame centre; yaw pi/2 moves it a quarter of the width east;
    pitch pi/4 moves it a quarter of the height north (Sec. 3.6 mapping)."""
    W, H = 1024, 512
    u, v = O.project(3, 3, 0.0, 0.0, math.radians(90), W, H)
    assert abs(u[1, 1] - (W / 2 - 0.5)) < 1e-9 and abs(v[1, 1] - (H / 2 - 0.5)) < 1e-9
    u2, _ = O.project(3, 3, math.pi / 2, 0.0, math.radians(90), W, H)
    assert abs(u2[1, 1] - (u[1, 1] + W / 4)) < 1e-9
    _, v3 = O.project(3, 3, 0.0, math.pi / 4, math.radians(90), W, H)
    assert abs(v3[1, 1] - (H / 4 - 0.5)) < 1e-9


def test_projection_corner_closed_form():
    """At yaw = pitch = 0 the ray of normalised image point (x, y) has
    longitude atan(x) and latitude atan(y / sqrt(1 + x^2))."""
    W, H = 4096, 2048
    n, fov = 8, math.radians(100)
    u, v = O.project(n, n, 0.0, 0.0, fov, W, H)
    t = math.tan(fov / 2)
    for (i, j) in [(0, 0), (7, 0), (3, 6), (7, 7)]:
        x = (2 * (i + 0.5) / n - 1) * t
        y = (1 - 2 * (j + 0.5) / n) * t
        lon = math.atan(x)
        lat = math.atan(y / math.sqrt(1 + x * x))
        assert abs(u[j, i] - ((lon / (2 * math.pi) + 0.5) * W - 0.5)) < 1e-9
        assert abs(v[j, i] - ((0.5 - lat / math.pi) * H - 0.5)) < 1e-9


def test_bilinear_special_cases():
    img = np.array([[10, 20, 30, 40], [50, 60, 70, 80]], np.uint8)
    # integer position: exact sample
    assert O.bilinear(img, np.array([2.0]), np.array([1.0]))[0] == 70
    # halfway between 10 and 20 -> 15
    assert O.bilinear(img, np.array([0.5]), np.array([0.0]))[0] == 15
    # longitude wraps: halfway between the last and first column -> 25
    assert O.bilinear(img, np.array([3.5]), np.array([0.0]))[0] == 25
    # latitude clamps above the top row
    assert O.bilinear(img, np.array([1.0]), np.array([-0.4]))[0] == 20
    # centre of the four pixels 10 20 50 60 -> 35
    assert O.bilinear(img, np.array([0.5]), np.array([0.5]))[0] == 35
    # quantisation to 1/256 with carry: 0.999 rounds up to the next pixel
    assert O.bilinear(img, np.array([0.999]), np.array([0.0]))[0] == 20
    const = np.full((8, 8), 77, np.uint8)
    rng = np.random.default_rng(0)
    assert np.all(O.bilinear(const, rng.uniform(-3, 11, 100), rng.uniform(-3, 11, 100)) == 77)


def test_colour_neutral_and_bt709_closed_form():
    """Y = Cb = Cr = 128 is mid grey; everywhere else the integer conversion
    is within one level of the published BT.709 inverse matrix
    (R = Y + 1.5748 Cr', G = Y - 0.1873 Cb' - 0.4681 Cr', B = Y + 1.8556 Cb')."""
    assert list(O.ycbcr_to_rgba(128, 128, 128)) == [128, 128, 128, 255]
    assert list(O.ycbcr_to_rgba(255, 128, 128)) == [255, 255, 255, 255]
    rng = np.random.default_rng(2)
    Y, Cb, Cr = (rng.integers(0, 256, 5000) for _ in range(3))
    got = O.ycbcr_to_rgba(Y, Cb, Cr).astype(float)
    cb, cr = Cb - 128.0, Cr - 128.0
    ref = np.stack([Y + 1.5748 * cr, Y - 0.1873 * cb - 0.4681 * cr, Y + 1.8556 * cb], -1)
    ref = np.clip(ref, 0, 255)
    assert np.abs(got[:, :3] - ref).max() <= 1.0


def test_footprint_contains_taps_and_pole():
    """The mask contains the cell of every tap, the dilated mask contains the
    core, and a viewport looking at the north pole needs the whole top row
    of cells (all longitudes meet there)."""
    p = O.Params(2048, 1024, 3, 1, 3, O.WAVELET_97, 1, 0, 256, 4.0)
    core, dil = O.footprint(p, 64, 64, 0.3, 0.2, math.radians(90))
    assert np.all(dil[core])
    u, v = O.project(64, 64, 0.3, 0.2, math.radians(90), 2048, 1024)
    xa, xb, ya, yb, _, _ = O.taps(u, v, 2048, 1024)
    assert np.all(core[ya // O.CELL, xa // O.CELL]) and np.all(core[yb // O.CELL, xb // O.CELL])
    core, _ = O.footprint(p, 512, 512, 0.0, math.pi / 2, math.radians(100))
    assert core[0].all() and core[1].all()
    frac = core.mean()
    assert 0.05 < frac < 0.6


def test_footprint_shifts_with_yaw():
    """Turning by a quarter turn moves the mask by a quarter of the columns
    (up to one cell at boundaries where fp64 rounding differs)."""
    p = O.Params(4096, 2048, 1, 0, 3, O.WAVELET_97, 1, 0, 256, 4.0)
    a, da = O.footprint(p, 48, 48, 0.1, 0.1, math.radians(80))
    b, db = O.footprint(p, 48, 48, 0.1 + math.pi / 2, 0.1, math.radians(80))
    q = a.shape[1] // 4
    assert np.all(np.roll(da, q, axis=1)[b]) and np.all(db[np.roll(a, q, axis=1)])


def test_viewport_of_coordinate_frame_reproduces_mapping():
    """A frame whose pixel values encode their own column reproduces the
    projected column (to the bilinear precision)."""
    W, H = 256, 128
    col = (np.arange(W) // 2).astype(np.uint8)          # value = x // 2
    img = np.tile(col, (H, 1))
    p = O.Params(W, H, 1, 0, 1, O.WAVELET_53, 1, 0, 64, 1.0)
    u, v = O.project(16, 16, 0.0, 0.0, math.radians(60), W, H)
    rgba = O.resample([img], p, u, v)
    assert np.abs(rgba[..., 0].astype(float) - u / 2).max() <= 1.0


def test_candidates_include_exact_result():
    rng = np.random.default_rng(4)
    planes = [rng.integers(0, 256, (64, 128)).astype(np.uint8),
              rng.integers(0, 256, (32, 64)).astype(np.uint8),
              rng.integers(0, 256, (32, 64)).astype(np.uint8)]
    p = O.Params(128, 64, 3, 1, 1, O.WAVELET_97, 1, 0, 32, 1.0)
    u, v = O.project(20, 20, 1.0, -0.3, 1.2, 128, 64)
    exact = O.resample(planes, p, u, v)
    cand = O.viewport_candidates(planes, p, u, v, 1e-3)
    assert np.all(np.any(np.all(cand == exact[..., None, :], axis=-1), axis=-1))


def test_stereo_eye_resamples_its_half_only():
    """Eye 1 of a top/bottom stereo frame [A; B] reprojects B exactly as a mono
    frame B; eye 0 reprojects A; taps never cross into the other half."""
    rng = np.random.default_rng(12)
    p_mono = O.Params(128, 64, 3, 1, 2, O.WAVELET_97, 1, 0, 32, 1.0)
    p_st = O.Params(128, 128, 3, 1, 2, O.WAVELET_97, 1, 0, 32, 1.0, 1)
    A = [rng.integers(0, 256, (64, 128), dtype=np.uint8)] + [rng.integers(0, 256, (32, 64), dtype=np.uint8)] * 2
    B = [rng.integers(0, 256, (64, 128), dtype=np.uint8)] + [rng.integers(0, 256, (32, 64), dtype=np.uint8)] * 2
    st = [np.vstack([a, b]) for a, b in zip(A, B)]
    for yaw, pitch, fov in [(0.3, 1.2, 1.5), (-2.0, -1.4, 1.2), (1.0, 0.0, 2.0)]:
        for eye, mono in ((0, A), (1, B)):
            r0, nr = O.eye_rows(p_st, eye)
            u, v = O.project(40, 30, yaw, pitch, fov, 128, nr, r0)
            um, vm = O.project(40, 30, yaw, pitch, fov, 128, 64)
            np.testing.assert_allclose(v - r0, vm, rtol=0, atol=1e-9)
            np.testing.assert_array_equal(O.resample(st, p_st, u, v, eye), O.resample(mono, p_mono, um, vm))
    with pytest.raises(ValueError):
        O.eye_rows(p_mono, 1)
