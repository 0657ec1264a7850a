"""GPU parity of top/bottom stereo streams (Sec. 3.6 reading: each eye an
equirect of half the frame height, eye 0 on top): per-eye viewports against
the oracle, both eyes through the batch engine and the server, the encoder's
stereo header, and rejected eyes."""
import math

import numpy as np
import pytest

import oracle as O
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POSES = [(0.0, 0.0, math.radians(100)), (2.9, 0.4, math.radians(90)),
         (-1.0, 1.3, math.radians(110)), (0.5, -1.45, math.radians(80))]


def _stream(name="stereo97"):
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case(name)
    return wv.Stream(data)


def _viewport(s, frame, yaw, pitch, fov, w, h, eye):
    out = torch.zeros((h, w, 4), dtype=torch.uint8, device="cuda")
    s.decode_viewport(frame, yaw, pitch, fov, out, eye=eye)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_stream_reports_stereo():
    _, p, _, _ = H.case("stereo97")
    assert p.stereo == 1
    assert _stream().desc["stereo"] == 1


@pytest.mark.parametrize("eye", [0, 1])
def test_eye_viewports_match_oracle_candidates(eye):
    """Each eye's viewport equals the oracle's reprojection of that eye's
    half (taps clamped to its rows) at a position within the float32 bound."""
    _, p, _, _ = H.case("stereo97")
    s = _stream()
    for k, (yaw, pitch, fov) in enumerate(POSES):
        frame = k % p.num_frames
        ref = H.oracle_planes("stereo97", frame)
        got = _viewport(s, frame, yaw, pitch, fov, 72, 56, eye)
        bad, exc = H.viewport_mismatches(ref, p, got, yaw, pitch, fov, eye)
        assert bad == 0, (eye, k, bad)
        assert exc <= 0.01 * got.shape[0] * got.shape[1]
    assert s.sync_status() == 0


def test_eyes_differ_and_stay_in_their_half():
    """The two eyes of one pose see different content (the halves differ),
    and each eye's viewport is unchanged when decoded on a fresh stream
    after the other eye (no rows of the other half leak in)."""
    s = _stream()
    a0 = _viewport(s, 0, 0.3, 0.1, 1.6, 64, 48, 0)
    a1 = _viewport(s, 0, 0.3, 0.1, 1.6, 64, 48, 1)
    assert np.any(a0 != a1)
    s2 = _stream()
    b1 = _viewport(s2, 0, 0.3, 0.1, 1.6, 64, 48, 1)
    b0 = _viewport(s2, 0, 0.3, 0.1, 1.6, 64, 48, 0)
    np.testing.assert_array_equal(a0, b0)
    np.testing.assert_array_equal(a1, b1)


def test_batch_both_eyes_equal_single_decodes():
    """Both eyes of several poses in one batch (they share the frame's decode
    target) equal one-at-a-time decodes."""
    from paper_2208_10859_gb300 import wv
    s = _stream()
    reqs, refs = [], []
    for k, (yaw, pitch, fov) in enumerate(POSES):
        for eye in (0, 1):
            out = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
            reqs.append(wv.ViewRequest(s, k % 2, yaw, pitch, fov, out, eye=eye))
            refs.append(_viewport(_stream(), k % 2, yaw, pitch, fov, 56, 40, eye))
    b = wv.Batch()
    b.decode(reqs)
    assert b.sync_status() == 0
    for r, ref in zip(reqs, refs):
        np.testing.assert_array_equal(r.out.cpu().numpy(), ref)
    assert b.stats()["surfaces"] == 2     # one per frame, shared by both eyes
    b.close()


def test_server_eye_requests():
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case("stereo97")
    srv = wv.Server(slots=2, max_batch=8)
    sid = srv.add_stream(data)
    outs, tickets = [], []
    for eye in (0, 1):
        out = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
        outs.append(out)
        tickets.append(srv.submit(sid, 1, 0.7, -0.2, 1.5, out, eye=eye))
    for t in tickets:
        srv.wait(t, 10000.0)
    torch.cuda.synchronize()
    for eye, out in enumerate(outs):
        np.testing.assert_array_equal(out.cpu().numpy(), _viewport(_stream(), 1, 0.7, -0.2, 1.5, 56, 40, eye))
    srv.close()


def test_invalid_eyes_rejected():
    from paper_2208_10859_gb300 import wv
    s = _stream()
    out = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    for eye in (-1, 2):
        with pytest.raises(wv.WVError):
            s.decode_viewport(0, 0.0, 0.0, 1.0, out, eye=eye)
        with pytest.raises(wv.WVError):
            wv.Batch().decode([wv.ViewRequest(s, 0, 0.0, 0.0, 1.0, out, eye=eye)])
    mono = _stream("yuv97")
    with pytest.raises(wv.WVError):
        mono.decode_viewport(0, 0.0, 0.0, 1.0, out, eye=1)


def test_gpu_encoder_writes_the_stereo_flag():
    from paper_2208_10859_gb300 import wv
    frames, p, data, st = H.case("stereo97")
    dev = [tuple(torch.from_numpy(np.ascontiguousarray(pl)).cuda() for pl in f) for f in frames]
    desc = dict(width=p.width, height=p.height, planes=p.planes, chroma_420=p.chroma_420,
                levels=p.levels, wavelet=p.wavelet, num_frames=p.num_frames, tlevels=p.tlevels,
                block=p.block, quant=0, step=p.step, stereo=1)
    g = wv.encode(dev, desc)
    assert O.Stream(g).p.stereo == 1
    assert wv.Stream(g).desc["stereo"] == 1
    # a height that is not a multiple of 64 cannot be split into two eyes
    # (rejected by the size query, before any frame is read)
    with pytest.raises(wv.WVError):
        wv.encode(dev, dict(desc, height=p.height - 32))
