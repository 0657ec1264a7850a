"""GPU parity of the viewport path: projection, footprint, resampling and the
end-to-end viewport against the oracle."""
import math

import numpy as np
import pytest

import oracle as O
import synth
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POSES = [(0.0, 0.0, math.radians(110)), (2.9, 0.3, math.radians(90)),      # near the seam
         (-1.2, 1.2, math.radians(110)), (0.4, -1.45, math.radians(100)),  # poles in view
         (-3.1, -0.2, math.radians(60))]


def _stream(name):
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case(name)
    return wv.Stream(data)


def test_projection_within_float32_error_bound():
    _, p, _, _ = H.case("yuv97")
    s = _stream("yuv97")
    for yaw, pitch, fov in POSES:
        uv = s.debug_project(yaw, pitch, fov, 96, 80).cpu().numpy().astype(np.float64)
        u, v = O.project(96, 80, yaw, pitch, fov, p.width, p.height)
        eu, ev = H.position_error_bound(p, 96, 80, yaw, pitch, fov)
        du = np.abs(((uv[..., 0] - u) + p.width / 2) % p.width - p.width / 2)   # seam-aware
        assert np.all(du <= eu), float((du / eu).max())
        assert np.all(np.abs(uv[..., 1] - v) <= ev), float((np.abs(uv[..., 1] - v) / ev).max())


def _grow(m, r):
    """Grow a cell mask by r cells in x (wrapping) and y (clamped)."""
    out = m.copy()
    for _ in range(r):
        g = out.copy()
        for dx in (-1, 1):
            g |= np.roll(out, dx, axis=1)
        g[1:] |= out[:-1]
        g[:-1] |= out[1:]
        out = g
    return out


@pytest.mark.parametrize("name", ["yuv97", "ragged53"])
def test_footprint_between_core_and_dilated(name):
    """The GPU mask contains every cell a bilinear tap of an fp64 position
    touches (the oracle's core) and stays within three cells of it: the GPU
    marks cells whose 3-pixel-grown extent meets the viewport frustum, bounding
    each cell by a spherical cap, which may add cells near frustum corners."""
    _, p, _, _ = H.case(name)
    s = _stream(name)
    for yaw, pitch, fov in POSES:
        for ow, oh in ((64, 64), (200, 120)):
            mask, tiles = s.debug_footprint(yaw, pitch, fov, ow, oh)
            core, _ = O.footprint(p, ow, oh, yaw, pitch, fov)
            m = mask.astype(bool)
            assert np.all(m[core]), (yaw, pitch, int((core & ~m).sum()))
            assert np.all(_grow(core, 3)[m]), (yaw, pitch, int((m & ~_grow(core, 3)).sum()))
            assert tiles > 0


def test_resample_arithmetic_bit_exact_at_given_positions():
    """Bilinear fixed point, wrap/clamp and BT.709 conversion: with the same
    float32 positions (seeded, covering the seam and both poles) the GPU
    result equals the oracle's bit for bit."""
    _, p, _, _ = H.case("yuv53")
    s = _stream("yuv53")
    for pl in range(3):
        s.decode_full(1, pl)
    planes = [u8 for (_, u8) in H.oracle_planes("yuv53", 1)]
    rng = np.random.default_rng(31)
    oh, ow = 48, 64
    u = rng.uniform(-3.0, p.width + 3.0, (oh, ow)).astype(np.float32)
    v = rng.uniform(-2.0, p.height + 1.0, (oh, ow)).astype(np.float32)
    u[0, :8] = [0.0, -0.5, p.width - 0.5, p.width - 0.001, 0.999, 1.0 / 512, 255.5 / 256, -1e-4]
    uv = torch.from_numpy(np.stack([u, v], -1)).cuda()
    out = torch.zeros((oh, ow, 4), dtype=torch.uint8, device="cuda")
    s.resample_at(uv, out)
    torch.cuda.synchronize()
    ref = O.resample(planes, p, u.astype(np.float64), v.astype(np.float64))
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("name", ["yuv53", "yuv97", "ragged97"])
def test_viewport_equals_full_decode_then_resample(name):
    """The viewport decoded through footprint -> tiles -> fused decode ->
    resample equals decoding the whole frame and resampling at the same device
    positions: the selected tiles cover every sample the mapping reads."""
    _, p, _, _ = H.case(name)
    for k, (yaw, pitch, fov) in enumerate(POSES):
        s = _stream(name)          # fresh: reconstruction planes start at zero
        frame = k % p.num_frames
        out = torch.zeros((72, 88, 4), dtype=torch.uint8, device="cuda")
        s.decode_viewport(frame, yaw, pitch, fov, out)
        uv = s.debug_project(yaw, pitch, fov, 88, 72)
        for pl in range(p.planes):
            s.decode_full(frame, pl)
        ref = torch.zeros_like(out)
        s.resample_at(uv, ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
        assert s.sync_status() == 0


@pytest.mark.parametrize("name", ["yuv53", "yuv97", "ragged97"])
def test_viewport_matches_oracle_candidates(name):
    """End to end against the oracle's plain definition (full decode, then
    reprojection): every viewport pixel equals the oracle's bilinear value at
    one of the 1/256 positions within the float32 error bound of the fp64
    position.  Pixels whose bound spans more than four quanta per axis (rays
    within a fraction of a degree of a pole) are excused and counted.  For
    9/7, a sample within 2e-3 of a rounding boundary may take either 8-bit
    value."""
    _, p, _, _ = H.case(name)
    s = _stream(name)
    ow, oh = 96, 64
    excused = total = 0
    for k, (yaw, pitch, fov) in enumerate(POSES):
        frame = (3 * k + 1) % p.num_frames
        out = torch.zeros((oh, ow, 4), dtype=torch.uint8, device="cuda")
        s.decode_viewport(frame, yaw, pitch, fov, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(-1, 4)
        ref = H.oracle_planes(name, frame)
        planes = [u8 for (_, u8) in ref]
        u, v = O.project(ow, oh, yaw, pitch, fov, p.width, p.height)
        eu, ev = H.position_error_bound(p, ow, oh, yaw, pitch, fov)
        u, v, eu, ev = u.ravel(), v.ravel(), eu.ravel(), ev.ravel()
        cand, flag = H.rgba_candidates(planes, p, u, v, eu, ev)
        ok = np.any(np.all(cand == got[:, None, :], axis=-1), axis=-1)
        if p.wavelet == O.WAVELET_97:
            # samples within 2e-3 of k + 1/2 may round either way in float32:
            # their other rounding gives a second candidate set
            alt = [H.other_rounding(x) for (x, _) in ref]
            cand2, _ = H.rgba_candidates(alt, p, u, v, eu, ev)
            ok |= np.any(np.all(cand2 == got[:, None, :], axis=-1), axis=-1)
        skip = flag
        bad = ~ok & ~skip
        assert not np.any(bad), (yaw, pitch, int(bad.sum()), np.nonzero(bad)[0][:5])
        excused += int(skip.sum())
        total += skip.size
    print(f"{name}: {excused} of {total} pixels excused")
    assert excused <= 0.01 * total


def test_cone_bytes_match_oracle():
    """Host-side accounting of the coefficient bytes a mask needs equals the
    oracle's cone computation on the same (seeded) mask."""
    for name in ("yuv97", "ragged53"):
        _, p, _, st = H.case(name)
        s = _stream(name)
        for seed in (1, 2):
            mask = synth.random_cell_mask(p.height // 32, p.width // 32, seed=seed, density=0.25)
            for frame in (0, 1):
                assert s.cone_bytes(frame, mask) == O.cone_bytes(st, frame, mask)


def test_foveated_cone_bytes_match_oracle():
    """Host accounting with foveation equals the oracle's cone restricted to
    the kept coefficients, on seeded masks and the oracle's keep masks."""
    _, p, _, st = H.case("fov97")
    s = _stream("fov97")
    for seed, (gx, gy, r1, r2) in [(1, (0.0, 0.0, 0.3, 0.6)), (2, (0.1, -0.05, 0.5, 0.9))]:
        mask = synth.random_cell_mask(p.height // 32, p.width // 32, seed=seed, density=0.4)
        keep = O.fovea_keep(p, 0.2, 0.1, gx, gy, r1, r2)
        bits = keep[1].astype(np.uint8) | (keep[2].astype(np.uint8) << 1)
        for frame in (0, 1):
            assert s.cone_bytes(frame, mask, bits) == O.cone_bytes(st, frame, mask, keep)


def test_batch_equals_single_and_bad_requests():
    from paper_2208_10859_gb300 import wv
    _, p, _, _ = H.case("yuv97")
    s1, s2 = _stream("yuv97"), _stream("ragged97")
    reqs, singles = [], []
    for k, (yaw, pitch, fov) in enumerate(POSES[:4]):
        st = s1 if k % 2 == 0 else s2
        out = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
        reqs.append(wv.ViewRequest(st, k % 2, yaw, pitch, fov, out))
    wv.decode_batch(reqs)
    torch.cuda.synchronize()
    for r in reqs:
        one = torch.zeros_like(r.out)
        r.stream.decode_viewport(r.frame, r.yaw, r.pitch, r.fov, one)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(one.cpu().numpy(), r.out.cpu().numpy())
    out = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    for bad in [(p.num_frames, 0.0, 0.0, 1.0), (-1, 0.0, 0.0, 1.0), (0, 0.0, 0.0, 0.0),
                (0, 0.0, 0.0, 3.2), (0, float("nan"), 0.0, 1.0)]:
        with pytest.raises(wv.WVError) as e:
            s1.decode_viewport(*bad, out)
        assert e.value.code == -1
    assert s1.sync_status() == 0 and s2.sync_status() == 0


def test_back_to_back_viewports_equal_isolated_decodes():
    """Consecutive viewports of one stream, enqueued without synchronising:
    each one's footprint, selection and coarse pass run on the stream's
    internal second CUDA stream while the previous one's fine pass and
    resampling run, alternating two sets of tile lists and LL_2 planes; a
    full-plane decode in between uses the first set.  Every output equals a
    decode of that viewport alone on a fresh stream."""
    _, p, _, _ = H.case("yuv97")
    s = _stream("yuv97")
    poses = POSES + [(1.1, -0.7, math.radians(75)), (-0.4, 0.9, math.radians(120))]
    outs = []
    for k, (yaw, pitch, fov) in enumerate(poses):
        out = torch.zeros((56, 72, 4), dtype=torch.uint8, device="cuda")
        s.decode_viewport(k % p.num_frames, yaw, pitch, fov, out)
        outs.append(out)
        if k == 3:
            full = torch.empty((p.height, p.width), dtype=torch.uint8, device="cuda")
            s.decode_full(1, 0, full)
    torch.cuda.synchronize()
    assert s.sync_status() == 0
    for k, (yaw, pitch, fov) in enumerate(poses):
        ref = torch.zeros((56, 72, 4), dtype=torch.uint8, device="cuda")
        _stream("yuv97").decode_viewport(k % p.num_frames, yaw, pitch, fov, ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[k].cpu().numpy(), ref.cpu().numpy())
    ref_x, ref_u8 = H.oracle_planes("yuv97", 1)[0]
    diff = full.cpu().numpy() != ref_u8
    assert not np.any(diff & ~H.near_half(ref_x))


def test_viewport_captured_in_a_cuda_graph():
    """A viewport decode captured into a CUDA graph (serial path: the stream
    then stops overlapping) replays to the same output as a direct decode,
    and direct decodes on the same stream stay correct afterwards."""
    _, p, _, _ = H.case("yuv97")
    s = _stream("yuv97")
    warm = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
    s.decode_viewport(0, 0.2, 0.1, 1.5, warm)          # kernel attributes set outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    out = torch.zeros((40, 56, 4), dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    s.set_cuda_stream(side)
    with torch.cuda.graph(g, stream=side):
        s.decode_viewport(1, -1.0, 0.4, 1.7, out)
    g.replay()
    torch.cuda.synchronize()
    ref = torch.zeros_like(out)
    _stream("yuv97").decode_viewport(1, -1.0, 0.4, 1.7, ref)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    s.set_cuda_stream(torch.cuda.current_stream())
    after = torch.zeros_like(out)
    s.decode_viewport(0, 0.2, 0.1, 1.5, after)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(after.cpu().numpy(), warm.cpu().numpy())
    assert s.sync_status() == 0
