"""Edge cases of the GPU path against the oracle: one wavelet level (the
single fused pass), a stream whose detail blocks are all omitted, 1-pixel
and one-row viewports, rays through the poles, a field of view close to
180 degrees, empty and single-request batches."""
import math

import numpy as np
import pytest

import oracle as O
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream(name):
    from paper_2208_10859_gb300 import wv
    return wv.Stream(H.case(name)[2])


def _viewport(s, frame, yaw, pitch, fov, w, h):
    out = torch.zeros((h, w, 4), dtype=torch.uint8, device="cuda")
    s.decode_viewport(frame, yaw, pitch, fov, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["l1_53", "l1_97"])
def test_one_level_streams(name):
    _, p, _, st = H.case(name)
    s = _stream(name)
    for f in range(p.num_frames):
        ref = H.oracle_planes(name, f)
        for pl in range(p.planes):
            w, h = O.plane_dims(p, pl)
            out = torch.empty((h, w), dtype=torch.uint8, device="cuda")
            s.decode_full(f, pl, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            if p.wavelet == O.WAVELET_53:
                np.testing.assert_array_equal(got, ref[pl][1])
            else:
                diff = got != ref[pl][1]
                assert not np.any(diff & ~H.near_half(ref[pl][0]))
        for yaw, pitch, fov in [(0.5, 0.2, 1.7), (-2.9, -0.6, 1.2)]:
            bad, exc = H.viewport_mismatches(ref, p, _viewport(s, f, yaw, pitch, fov, 48, 40), yaw, pitch, fov)
            assert bad == 0 and exc <= 0.01 * 48 * 40
    assert s.sync_status() == 0


def test_all_detail_blocks_omitted():
    frames, p, data, st = H.case("flat97")
    assert int((st.table >= 0).sum()) == 1   # the low band's LL block; details and the Haar band are zero
    s = _stream("flat97")
    out = torch.empty((p.height, p.width), dtype=torch.uint8, device="cuda")
    s.decode_full(1, 0, out)
    torch.cuda.synchronize()
    ref = H.oracle_planes("flat97", 1)[0][1]
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    level = int(ref[0, 0])                       # the dead-zone reconstruction of the constant
    assert np.all(ref == level) and abs(level - 77) <= 2
    vp = _viewport(s, 0, 1.0, 0.3, 1.5, 33, 17)
    assert np.all(vp[..., :3] == level) and np.all(vp[..., 3] == 255)


@pytest.mark.parametrize("size", [(1, 1), (1, 57), (64, 1)])
def test_tiny_viewports(size):
    w, h = size
    _, p, _, _ = H.case("yuv97")
    s = _stream("yuv97")
    for yaw, pitch, fov in [(0.3, 0.1, 1.9), (3.0, -1.0, 0.4)]:
        ref = H.oracle_planes("yuv97", 2)
        bad, exc = H.viewport_mismatches(ref, p, _viewport(s, 2, yaw, pitch, fov, w, h), yaw, pitch, fov)
        assert bad == 0 and exc <= max(1, 0.01 * w * h)


@pytest.mark.parametrize("pitch", [math.pi / 2, -math.pi / 2])
def test_views_straight_up_and_down(pitch):
    """The centre ray hits the pole, where longitude is undefined: every
    pixel still matches an oracle candidate or is counted as excused."""
    _, p, _, _ = H.case("yuv53")
    s = _stream("yuv53")
    ref = H.oracle_planes("yuv53", 1)
    bad, exc = H.viewport_mismatches(ref, p, _viewport(s, 1, 0.7, pitch, 1.6, 64, 64), 0.7, pitch, 1.6)
    assert bad == 0 and exc <= 0.02 * 64 * 64


def test_field_of_view_near_180_degrees():
    _, p, _, _ = H.case("ragged97")
    s = _stream("ragged97")
    ref = H.oracle_planes("ragged97", 0)
    fov = 3.1
    bad, exc = H.viewport_mismatches(ref, p, _viewport(s, 0, -0.4, 0.2, fov, 96, 96), -0.4, 0.2, fov)
    assert bad == 0 and exc <= 0.01 * 96 * 96


def test_empty_and_single_request_batches():
    from paper_2208_10859_gb300 import wv
    s = _stream("yuv97")
    wv.decode_batch([])
    out = torch.zeros((40, 52, 4), dtype=torch.uint8, device="cuda")
    wv.decode_batch([wv.ViewRequest(s, 1, 0.2, 0.1, 1.5, out)])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), _viewport(s, 1, 0.2, 0.1, 1.5, 52, 40))
    assert s.sync_status() == 0
