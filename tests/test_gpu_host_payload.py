"""Host-resident coefficient store (WV_OPEN_HOST_PAYLOAD): the tile decoder
reads the coefficient blocks from pinned, device-mapped host memory.  Every
output equals the output of the same stream opened with its store in device
memory, for both code forms, the paper-faithful format and batches."""
import math

import numpy as np
import pytest

import oracle as O
import synth
import helpers as H
from oracle import paper_format as PF

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POSES = [(0.0, 0.0, math.radians(100)), (2.9, 0.4, math.radians(90)), (-1.2, 1.2, math.radians(110))]


def _both(data):
    from paper_2208_10859_gb300 import wv
    return wv.Stream(data), wv.Stream(data, host_payload=True)


def test_query_excludes_the_payload():
    from paper_2208_10859_gb300 import wv
    _, p, data, st = H.case("yuv97")
    _, dev = wv.query(data)
    _, host = wv.query(data, wv.WV_OPEN_HOST_PAYLOAD)
    payload = st.payload.size * 2
    assert dev - host >= payload
    with pytest.raises(wv.WVError):
        wv.query(data, 2)


@pytest.mark.parametrize("name", ["yuv97", "yuv53", "wideq97", "stereo97"])
def test_host_store_decodes_like_device_store(name):
    _, p, data, _ = H.case(name)
    dev, host = _both(data)
    for k, (yaw, pitch, fov) in enumerate(POSES):
        outs = []
        for s in (dev, host):
            o = torch.zeros((48, 64, 4), dtype=torch.uint8, device="cuda")
            s.decode_viewport(k % p.num_frames, yaw, pitch, fov, o)
            outs.append(o)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[0].cpu().numpy(), outs[1].cpu().numpy())
    for pl in range(p.planes):
        w, h = O.plane_dims(p, pl)
        a = torch.empty((h, w), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        dev.decode_full(1, pl, a, as_float=True)
        host.decode_full(1, pl, b, as_float=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert dev.sync_status() == 0 and host.sync_status() == 0


def test_host_store_paper_format():
    fr = synth.equirect_gop(64, 4, seed=5, n_discs=3)
    pp = PF.PaperParams(64, 64, 3, 1, 3, 4, 2, alpha=0.02, alpha_t=0.005)
    dev, host = _both(PF.encode(fr, pp))
    for f in range(4):
        a = torch.empty((64, 64), dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        dev.decode_full(f, 0, a)
        host.decode_full(f, 0, b)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_host_store_in_a_batch():
    from paper_2208_10859_gb300 import wv
    _, p, data, _ = H.case("yuv97")
    dev, host = _both(data)
    reqs, refs = [], []
    for k, (yaw, pitch, fov) in enumerate(POSES):
        o = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
        reqs.append(wv.ViewRequest(host, k % p.num_frames, yaw, pitch, fov, o, fovea=(k == 1),
                                   gaze_x=0.1, gaze_y=0.0, r1=0.3, r2=0.6))
        r = torch.zeros_like(o)
        refs.append(r)
    b = wv.Batch()
    b.decode(reqs)
    b2 = wv.Batch()
    b2.decode([wv.ViewRequest(dev, r.frame, r.yaw, r.pitch, r.fov, ref, r.fovea, r.gaze_x, r.gaze_y, r.r1, r.r2)
               for r, ref in zip(reqs, refs)])
    torch.cuda.synchronize()
    assert b.sync_status() == 0 and b2.sync_status() == 0
    for r, ref in zip(reqs, refs):
        np.testing.assert_array_equal(r.out.cpu().numpy(), ref.cpu().numpy())
    b.close()
    b2.close()
