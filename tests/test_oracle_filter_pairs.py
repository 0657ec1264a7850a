"""Pins of the post-filter training-pair recipe (oracle/filter_pairs.py):
a 540 x 540, 110-degree viewport of a 2048-wide crop samples the crop as a
2160 x 2160, 110-degree viewport samples an 8192-wide frame (the ratio of
viewport pixel to frame pixel holds at every viewport position); crops are
32-aligned and inside the frame and keep the 4:2:0 chroma siting."""
import math

import numpy as np

import oracle as O
import oracle.filter_pairs as F


def test_viewport_sampling_matches_the_benchmark_geometry():
    fov = math.radians(F.FOV_DEG)
    us, vs = O.project(F.VIEW, F.VIEW, 0.4, 0.2, fov, F.CROP, F.CROP)
    ub, vb = O.project(2160, 2160, 0.4, 0.2, fov, F.FRAME, F.FRAME)
    # the same viewing directions: viewport pixel i of the small view and
    # pixel 4 i + 3/2 of the large one (pixel centres), frame positions
    # scaled by 4 (u, v are in frame pixels with centres at integers)
    i = np.array([0, 100, 269, 400, 539])
    for j in (0, 270, 539):
        small = (us[j, i] + 0.5) * 4 - 0.5
        big_u = np.interp(4 * i + 1.5, np.arange(2160), ub[4 * j + 1])
        big_u2 = np.interp(4 * i + 1.5, np.arange(2160), ub[4 * j + 2])
        np.testing.assert_allclose(small, 0.5 * (big_u + big_u2), atol=0.05)


def test_crop_origins_are_aligned_and_inside():
    for seed in (11, 12, 99):
        for x0, y0 in F.crop_origins(6, seed):
            assert x0 % 32 == 0 and y0 % 32 == 0
            assert 0 <= x0 <= F.FRAME - F.CROP and 0 <= y0 <= F.FRAME - F.CROP


def test_crop_of_a_group_keeps_the_chroma_siting():
    rng = np.random.default_rng(3)
    frames = [(rng.integers(0, 256, (F.FRAME // 64, F.FRAME // 64), dtype=np.uint8),
               rng.integers(0, 256, (F.FRAME // 128, F.FRAME // 128), dtype=np.uint8),
               rng.integers(0, 256, (F.FRAME // 128, F.FRAME // 128), dtype=np.uint8))]
    crop, frame_size = F.CROP, F.FRAME
    try:
        F.CROP, F.FRAME = 32, F.FRAME // 64
        (y, cb, cr), = F.crop_gop(frames, 64, 32)
        assert y.shape == (32, 32) and cb.shape == (16, 16) and cr.shape == (16, 16)
        np.testing.assert_array_equal(y, frames[0][0][32:64, 64:96])
        np.testing.assert_array_equal(cb, frames[0][1][16:32, 32:48])
    finally:
        F.CROP, F.FRAME = crop, frame_size
