"""GPU encoder against the oracle encoder: identical streams for the integer
5/3 path; for 9/7 (float32 on the GPU, fp64 in the oracle) every quantised
coefficient equal except where the fp64 value sits within 1e-3 of a
quantiser decision boundary, and there by at most one step."""
import numpy as np
import pytest

import oracle as O
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu_encode(frames, p):
    from paper_2208_10859_gb300 import wv
    dev = [tuple(torch.from_numpy(np.ascontiguousarray(pl)).cuda() for pl in f) for f in frames]
    desc = dict(width=p.width, height=p.height, planes=p.planes, chroma_420=p.chroma_420,
                levels=p.levels, wavelet=p.wavelet, num_frames=p.num_frames, tlevels=p.tlevels,
                block=p.block, quant=0, step=p.step)
    return wv.encode(dev, desc)


@pytest.mark.parametrize("name", ["cfg1", "yuv53", "ragged53"])
def test_53_stream_bytes_identical(name):
    frames, p, data, _ = H.case(name)
    assert _gpu_encode(frames, p) == data


@pytest.mark.parametrize("name", ["yuv97", "ragged97"])
def test_97_quantised_coefficients_agree_off_boundaries(name):
    frames, p, data, st = H.case(name)
    gst = O.Stream(_gpu_encode(frames, p))
    integer = False
    n = 1 << p.tlevels
    for s in range(p.num_frames // n):
        for pl in range(p.planes):
            coefs = [O.fwd2d(np.asarray(frames[s * n + j][pl], np.float64) - 128.0, p.levels, p.wavelet)
                     for j in range(n)]
            bands = O.haar_forward(coefs, p.tlevels, integer) if p.tlevels else coefs
            for j in range(n):
                t = s * n + j
                a = st.coef_plane(t, pl)
                b = gst.coef_plane(t, pl)
                r = np.abs(bands[j]) / p.step
                boundary = np.abs(r - np.rint(r)) < 1e-3
                diff = a != b
                assert not np.any(diff & ~boundary), (t, pl, int((diff & ~boundary).sum()))
                assert np.all(np.abs(a - b) <= 1)
