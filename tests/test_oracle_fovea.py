"""Pins of the oracle's foveated decoding (Sec. 3.7): the distance in closed
form, the cell -> coefficient mapping against block replication, the two
extreme radii against the plain decode and against a decode whose detail
subbands are zeroed by slicing, and locality (pixels whose synthesis support
lies inside the kept region equal the plain decode)."""
import math

import numpy as np
import pytest

import oracle as O
import helpers as H


def test_distance_closed_form_on_the_equator_rows():
    """yaw = pitch = 0, gaze at the view centre: a cell centre at longitude
    lam and latitude phi (|lam| < pi/2) is seen at theta_x = lam and
    theta_y = atan(tan(phi) / cos(lam))."""
    p = O.Params(1024, 512)
    d = O.fovea_distance(p, 0.0, 0.0, 0.0, 0.0)
    rows, cols = d.shape
    for r in (rows // 2 - 1, rows // 2, 3):
        phi = math.pi * (0.5 - (r + 0.5) * 32 / 512)
        for c in range(cols):
            lam = 2 * math.pi * ((c + 0.5) * 32 / 1024 - 0.5)
            if abs(lam) >= math.pi / 2:
                assert math.isinf(d[r, c])
                continue
            ty = math.atan(math.tan(phi) / math.cos(lam))
            assert d[r, c] == pytest.approx(max(abs(lam), abs(ty)), abs=1e-12)


def test_distance_follows_gaze_and_yaw():
    """Turning the head by yaw moves the distance field by yaw in longitude
    (whole cells); the gaze offset shifts theta_x."""
    p = O.Params(1024, 512)
    step = 2 * math.pi * 32 / 1024          # one cell of longitude
    d0 = O.fovea_distance(p, 0.0, 0.0, 0.0, 0.0)
    d5 = O.fovea_distance(p, 5 * step, 0.0, 0.0, 0.0)
    np.testing.assert_allclose(np.roll(d0, 5, axis=1), d5, rtol=0, atol=1e-12)
    # gaze 0.2 rad right and 0.1 rad up: theta_x - 0.2 and theta_y - 0.1
    dg = O.fovea_distance(p, 0.0, 0.0, 0.2, 0.1)
    r = d0.shape[0] // 2
    phi = math.pi * (0.5 - (r + 0.5) * 32 / 512)
    for c in range(d0.shape[1]):
        lam = 2 * math.pi * ((c + 0.5) * 32 / 1024 - 0.5)
        if abs(lam) < math.pi / 2:
            ty = math.atan(math.tan(phi) / math.cos(lam))
            assert dg[r, c] == pytest.approx(max(abs(lam - 0.2), abs(ty - 0.1)), abs=1e-12)


def test_coef_mask_replicates_cells():
    """A level-l coefficient of a plane subsampled by s covers s 2^l luma
    pixels per side: the coefficient mask of each kept level is the cell mask
    replicated 32 / (s 2^l) times per axis (level 3 and LL: all ones)."""
    p = O.Params(256, 128, 3, 1, 4, O.WAVELET_97)
    rng = np.random.default_rng(7)
    keep = {1: rng.random((4, 8)) < 0.5, 2: rng.random((4, 8)) < 0.5}
    for pl in range(3):
        s = 2 if pl else 1
        w, h = O.plane_dims(p, pl)
        m = O.fovea_coef_mask(p, pl, keep)
        for (name, lev, x0, y0, sw, sh) in O.subbands(w, h, p.levels):
            sub = m[y0:y0 + sh, x0:x0 + sw]
            if name == "LL" or lev > 2:
                assert sub.all()
                continue
            rep = 32 // (s << lev)
            np.testing.assert_array_equal(sub, np.kron(keep[lev], np.ones((rep, rep), bool)))


def test_infinite_radii_equal_plain_decode():
    _, p, _, st = H.case("yuv97")
    keep = O.fovea_keep(p, 0.3, 0.1, 0.0, 0.0, math.inf, math.inf)
    for pl in range(3):
        np.testing.assert_array_equal(O.decode_plane(st, 1, pl, keep)[0], O.decode_plane(st, 1, pl)[0])


@pytest.mark.parametrize("name", ["yuv97", "yuv53"])
def test_zero_radii_drop_levels_1_and_2(name):
    """Negative radii keep nothing: the decode equals the inverse transform
    of the rebuilt coefficients with the level-1 and level-2 detail subbands
    cleared by slicing the Mallat plane."""
    _, p, _, st = H.case(name)
    keep = O.fovea_keep(p, 0.0, 0.0, 0.0, 0.0, -1.0, -1.0)
    for pl in range(3):
        w, h = O.plane_dims(p, pl)
        c = O.decode_coefs(st, 2, pl).copy()
        c[:, w >> 2:] = 0            # HL_2, HL_1 and the right half of HH
        c[h >> 2:, :] = 0            # LH_2, LH_1, HH
        want = O.inv2d(c, p.levels, p.wavelet) + 128
        np.testing.assert_allclose(O.decode_plane(st, 2, pl, keep)[0], want, rtol=0, atol=1e-9)


def test_pixels_far_inside_the_kept_region_are_unchanged():
    """Locality: a pixel whose cell and its eight neighbours keep the level-1
    and level-2 details equals the plain decode (a two-level 9/7 synthesis
    reads level-1/2 coefficients within 24 pixels of the output), while
    pixels outside the level-2 region change."""
    _, p, _, st = H.case("gray97_L6")
    keep = O.fovea_keep(p, 0.0, 0.0, 0.0, 0.0, 1.2, 1.6)
    x_f = O.decode_plane(st, 0, 0, keep)[0]
    x_p = O.decode_plane(st, 0, 0)[0]
    k = keep[1].copy()
    for dy in (-1, 0, 1):                              # erode by one cell
        for dx in (-1, 0, 1):
            k &= np.roll(np.roll(keep[1], dy, 0), dx, 1)
    inside = O.cell_mask_to_pixels(k, p.width, p.height)
    assert inside.sum() > 1000
    np.testing.assert_allclose(x_f[inside], x_p[inside], rtol=0, atol=1e-9)
    assert np.abs(x_f - x_p)[~O.cell_mask_to_pixels(keep[2], p.width, p.height)].max() > 0.5


def test_foveation_loads_less():
    """Fewer kept cells, fewer coefficient bytes (Sec. 3.7: less data)."""
    _, p, _, st = H.case("yuv97")
    core, _ = O.footprint(p, 128, 128, 0.2, 0.1, math.radians(100))
    full = O.cone_bytes(st, 0, core)
    kw = O.fovea_keep(p, 0.2, 0.1, 0.0, 0.0, 0.6, 1.0)
    kn = O.fovea_keep(p, 0.2, 0.1, 0.0, 0.0, 0.2, 0.4)
    assert full > O.cone_bytes(st, 0, core, kw) > O.cone_bytes(st, 0, core, kn) > 0
    assert O.cone_bytes(st, 0, core, O.fovea_keep(p, 0.2, 0.1, 0, 0, math.inf, math.inf)) == full
