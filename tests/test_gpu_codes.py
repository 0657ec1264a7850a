"""Both device forms of 9/7 dead-zone codes: streams whose codes stay
within |q| <= 8191 are held as 2q + sign(q) after opening, others keep q.
The second form (a fine quantiser step) decodes within the 9/7 tolerance of
the oracle, and batches over both forms equal single decodes."""
import math

import numpy as np
import pytest

import oracle as O
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stream(name):
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case(name)
    return wv.Stream(data)


def test_case_codes_exceed_the_transcode_bound():
    _, _, _, st = H.case("wideq97")
    assert int(np.abs(st.payload).max()) > 8191
    _, _, _, st = H.case("yuv97")
    assert int(np.abs(st.payload).max()) <= 8191


def test_untranscoded_codes_decode_within_tolerance():
    _, p, _, _ = H.case("wideq97")
    s = _stream("wideq97")
    for f in range(p.num_frames):
        for pl in range(p.planes):
            ref_x, ref_u8 = H.oracle_planes("wideq97", f)[pl]
            w, h = O.plane_dims(p, pl)
            out = torch.empty((h, w), dtype=torch.float32, device="cuda")
            s.decode_full(f, pl, out, as_float=True)
            torch.cuda.synchronize()
            err = np.abs(out.cpu().numpy().astype(np.float64) - ref_x)
            assert err.max() <= H.tol_97_levels(), (f, pl, err.max())
            assert err.max() <= H.reg_97_levels(), (f, pl, err.max())
    assert s.sync_status() == 0


def test_batch_over_both_code_forms_equals_single_decodes():
    from paper_2208_10859_gb300 import wv
    streams = {n: _stream(n) for n in ("wideq97", "yuv97")}
    poses = [(0.3, 0.2, math.radians(100)), (-2.0, -0.5, math.radians(80))]
    reqs, refs = [], []
    for n, s in streams.items():
        for k, (yaw, pitch, fov) in enumerate(poses):
            out = torch.zeros((48, 64, 4), dtype=torch.uint8, device="cuda")
            reqs.append(wv.ViewRequest(s, k % 2, yaw, pitch, fov, out))
            ref = torch.zeros_like(out)
            _stream(n).decode_viewport(k % 2, yaw, pitch, fov, ref)
            refs.append(ref)
    b = wv.Batch()
    b.decode(reqs)
    assert b.sync_status() == 0
    torch.cuda.synchronize()
    for r, ref in zip(reqs, refs):
        np.testing.assert_array_equal(r.out.cpu().numpy(), ref.cpu().numpy())
    b.close()
    # the untranscoded stream's viewports against the oracle
    _, p, _, _ = H.case("wideq97")
    for k, (yaw, pitch, fov) in enumerate(poses):
        got = reqs[k].out.cpu().numpy()
        bad, exc = H.viewport_mismatches(H.oracle_planes("wideq97", k % 2), p, got, yaw, pitch, fov)
        assert bad == 0 and exc <= 0.01 * got.shape[0] * got.shape[1]
