"""GPU parity: full-plane decode through the C ABI against the oracle.

Bit-exact for the integer 5/3 path and for 8-bit samples (9/7 samples within
2e-3 of a rounding boundary excepted, where float32 and fp64 may round apart);
9/7 float samples within 1e-4 of the 8-bit full scale of the fp64 oracle."""
import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream(name):
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case(name)
    return wv.Stream(data)


def _decode(s, frame, plane, as_float):
    w, h = s.desc["width"], s.desc["height"]
    if plane > 0 and s.desc["chroma_420"]:
        w, h = w // 2, h // 2
    out = torch.empty((h, w), dtype=torch.float32 if as_float else torch.uint8, device="cuda")
    s.decode_full(frame, plane, out, as_float=as_float)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_lossless_512_53_is_bit_exact():
    """512x512 grey, 3-level LeGall 5/3, step 1: the GPU inverse returns the
    input frame byte for byte."""
    frames, p, _, _ = H.case("cfg1")
    s = _stream("cfg1")
    got = _decode(s, 0, 0, False)
    np.testing.assert_array_equal(got, frames[0][0])
    np.testing.assert_array_equal(got, H.oracle_planes("cfg1", 0)[0][1])
    assert s.sync_status() == 0


@pytest.mark.parametrize("name", ["yuv53", "ragged53"])
def test_53_streams_bit_exact(name):
    """Integer path with inter-frame sets (one and two Haar levels), chroma,
    ragged tiles and a lossy integer step: equal to the oracle everywhere."""
    frames, p, _, _ = H.case(name)
    s = _stream(name)
    for f in range(p.num_frames):
        for pl in range(p.planes):
            ref_x, ref_u8 = H.oracle_planes(name, f)[pl]
            np.testing.assert_array_equal(_decode(s, f, pl, False), ref_u8)
            np.testing.assert_array_equal(_decode(s, f, pl, True), ref_x.astype(np.float32))
            if p.step == 1:
                np.testing.assert_array_equal(ref_u8, frames[f][pl])
    assert s.sync_status() == 0


@pytest.mark.parametrize("name", ["yuv97", "ragged97", "gray97_L6"])
def test_97_streams_within_tolerance(name):
    """CDF 9/7 in float32 against the fp64 oracle: |x - x64| <= 1e-4 * 255
    on every sample and within the tight regression bound in levels; 8-bit
    results equal away from rounding boundaries."""
    _, p, _, _ = H.case(name)
    s = _stream(name)
    worst = 0.0
    for f in range(p.num_frames):
        for pl in range(p.planes):
            ref_x, ref_u8 = H.oracle_planes(name, f)[pl]
            got = _decode(s, f, pl, True).astype(np.float64)
            err = np.abs(got - ref_x)
            worst = max(worst, float(err.max()))
            assert err.max() <= H.tol_97_levels(), (f, pl, err.max())
            assert err.max() <= H.reg_97_levels(), (f, pl, err.max())
            got8 = _decode(s, f, pl, False)
            diff = got8 != ref_u8
            assert not np.any(diff & ~H.near_half(ref_x)), (f, pl, int(diff.sum()))
            assert np.all(np.abs(got8.astype(int) - ref_u8)[diff] <= 1)
    print(f"{name}: max |float32 - fp64| = {worst:.3e} levels ({worst / 255:.3e} of full scale)")
    assert s.sync_status() == 0


def test_decode_full_into_internal_planes_and_bad_args():
    from paper_2208_10859_gb300 import wv
    s = _stream("yuv97")
    s.decode_full(0, 0)               # into the stream's own plane
    with pytest.raises(wv.WVError) as e:
        s.decode_full(99, 0)
    assert e.value.code == -1
    with pytest.raises(wv.WVError):
        s.decode_full(0, 3)
    assert s.sync_status() == 0


@pytest.mark.parametrize("name", ["yuv53", "yuv97", "gray97_L6", "ragged97"])
def test_coarse_fine_split_equals_fused(name):
    """The two-pass organisation (coarse levels into LL_2 planes, then levels
    2..1) and the single fused pass give the same planes: bit-exact for 5/3,
    within the 9/7 float tolerance otherwise."""
    _, p, _, _ = H.case(name)
    s = _stream(name)
    for f in (0, p.num_frames - 1):
        for pl in range(p.planes):
            s.set_decode_mode(0)
            a = _decode(s, f, pl, True)
            s.set_decode_mode(1)
            b = _decode(s, f, pl, True)
            if p.wavelet == 0:
                np.testing.assert_array_equal(a, b)
            else:
                assert np.abs(a.astype(np.float64) - b).max() <= H.tol_97_levels()
            # 8-bit samples: the strip fine pass (mode 0; float output always
            # takes the square tiles) equals the square-tile fine pass
            # (mode 2) exactly -- the same lifting arithmetic per sample
            s.set_decode_mode(0)
            u_strip = _decode(s, f, pl, False)
            s.set_decode_mode(2)
            u_square = _decode(s, f, pl, False)
            np.testing.assert_array_equal(u_strip, u_square)
    s.set_decode_mode(1)
    assert s.launches_per_viewport() == 4
    s.set_decode_mode(0)
    assert s.launches_per_viewport() == (5 if p.levels >= 3 else 4)
    assert s.sync_status() == 0
