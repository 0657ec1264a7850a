"""GPU parity of batched decoding (wv_batch_*, wv_decode_batch): a batch of
requests over streams of uneven size, wavelet, field of view and output
size equals the per-viewport decode of each request; tile shapes chosen by
the autotuner change nothing; foveated requests (Sec. 3.7) match the oracle's
foveated decode."""
import math

import numpy as np
import pytest

import oracle as O
import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POSES = [(0.0, 0.0, math.radians(110)), (2.9, 0.3, math.radians(90)),
         (-1.2, 1.2, math.radians(110)), (0.4, -1.45, math.radians(100)),
         (-3.1, -0.2, math.radians(60)), (1.0, 0.2, math.radians(120))]


def _streams(*names):
    from paper_2208_10859_gb300 import wv
    return {n: wv.Stream(H.case(n)[2]) for n in names}


def _requests(streams, n, seed=0):
    """n requests cycling over the streams, poses, frames and output sizes;
    every other request repeats the previous one's stream and frame (a shared
    decode target)."""
    from paper_2208_10859_gb300 import wv
    names = sorted(streams)
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        name = names[(k // 2) % len(names)]
        p = H.case(name)[1]
        frame = ((k // 2) * 3 + 1) % p.num_frames
        yaw, pitch, fov = POSES[(k + seed) % len(POSES)]
        yaw += float(rng.uniform(-0.3, 0.3))
        ow, oh = [(96, 64), (56, 40), (64, 64)][k % 3]
        out = torch.zeros((oh, ow, 4), dtype=torch.uint8, device="cuda")
        reqs.append(wv.ViewRequest(streams[name], frame, yaw, pitch, fov, out))
    return reqs


def _single(r):
    one = torch.zeros_like(r.out)
    r.stream.decode_viewport(r.frame, r.yaw, r.pitch, r.fov, one)
    torch.cuda.synchronize()
    return one.cpu().numpy()


def _assert_same(r, got):
    """Batch output against the single decode: identical (same kernels, same
    arithmetic per sample)."""
    np.testing.assert_array_equal(got, _single(r))


NAMES = ("yuv97", "yuv53", "ragged97", "ragged53", "gray97_L6", "cfg1")


def test_batch_equals_single_decodes():
    from paper_2208_10859_gb300 import wv
    st = _streams(*NAMES)
    reqs = _requests(st, 14)
    b = wv.Batch()
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    info = b.stats()
    targets = {(id(r.stream), r.frame) for r in reqs}
    assert info["requests"] == 14 and info["surfaces"] == len(targets) == 6
    assert info["fine_tiles"] > 0 and info["coarse_tiles"] > 0
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    b.close()


def test_graph_relaunch_takes_new_poses():
    """The second batch of the same shape reuses the captured graph: its
    results follow the new job tables."""
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97", "ragged53")
    b = wv.Batch()
    for seed in (1, 2, 3):
        reqs = _requests(st, 6, seed=seed)
        b.decode(reqs)
        torch.cuda.synchronize()
        for r in reqs:
            _assert_same(r, r.out.cpu().numpy())
    assert b.sync_status() == 0


@pytest.mark.parametrize("shape", [(64, 64, 32), (64, 64, 64), (128, 128, 32), (256, 64, 64), (256, 128, 64),
                                   (256, 128, 32)])
def test_tile_shapes_give_identical_results(shape):
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97", "yuv53", "ragged97", "gray97_L6")
    b = wv.Batch()
    for name in st:
        p = H.case(name)[1]
        b.set_tile_shape(p.wavelet, p.levels, p.width, p.height, *shape)
        assert b.tile_shape(p.wavelet, p.levels, p.width, p.height) == shape
    reqs = _requests(st, 8, seed=4)
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())


def test_autotune_then_decode():
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97", "ragged53")
    reqs = _requests(st, 6, seed=5)
    b = wv.Batch()
    b.autotune(reqs, reps=2)
    for name in st:
        p = H.case(name)[1]
        assert b.tile_shape(p.wavelet, p.levels, p.width, p.height) in [
            (128, 128, 64), (128, 128, 32), (64, 64, 64), (64, 64, 32), (256, 64, 64), (256, 128, 64)]
    b.decode(reqs)
    torch.cuda.synchronize()
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    assert b.sync_status() == 0


def test_unsupported_tile_shapes_are_rejected():
    from paper_2208_10859_gb300 import wv
    b = wv.Batch()
    for shape in [(256, 256, 64), (128, 64, 64), (96, 96, 64), (128, 128, 48)]:
        with pytest.raises(wv.WVError):
            b.set_tile_shape(1, 5, 8192, 8192, *shape)
    b.close()


@pytest.mark.parametrize("part", [0, 3])
def test_waves_under_a_memory_limit_change_nothing(part):
    """Decode targets grouped into waves that reuse one device region: the
    outputs equal the single decodes; with a limit below any target's size
    every target is a wave of its own; requests of an earlier wave complete
    no later than those of a later one."""
    from paper_2208_10859_gb300 import wv
    st = _streams(*NAMES)
    reqs = _requests(st, 14, seed=6)
    one = wv.Batch()
    one.set_memory_limit(0)
    limit = one.device_bytes(reqs) // part if part else 1
    b = wv.Batch()
    b.set_memory_limit(limit)
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    info = b.stats()
    assert info["waves"] > 1
    if limit == 1:
        assert info["waves"] == info["surfaces"]
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    one.decode(reqs)
    torch.cuda.synchronize()
    i1 = one.stats()
    assert i1["waves"] == 1
    assert (i1["fine_tiles"], i1["coarse_tiles"]) == (info["fine_tiles"], info["coarse_tiles"])
    assert info["bytes"] < i1["bytes"]
    # completion times follow the waves (timed mode, direct launches)
    b.set_timing(True)
    b.decode(reqs)
    done = b.completion_ms(len(reqs))
    assert np.all(done > 0)
    targets = []
    for r in reqs:
        k = (id(r.stream), r.frame)
        if k not in targets:
            targets.append(k)
    wave_of = [targets.index((id(r.stream), r.frame)) for r in reqs] if limit == 1 else None
    if wave_of is not None:
        order = np.argsort(wave_of, kind="stable")
        assert np.all(np.diff(done[order]) >= 0)
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    with pytest.raises(wv.WVError):
        b.completion_ms(len(reqs) + 1)
    b.close()
    one.close()


def test_timing_mode_and_default_context():
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97", "gray97_L6")
    reqs = _requests(st, 4, seed=6)
    b = wv.Batch()
    b.set_timing(True)
    b.decode(reqs)
    ms = b.stats()["ms"]
    assert all(v > 0 for v in ms.values()), ms
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    reqs = _requests(st, 4, seed=7)
    wv.decode_batch(reqs)             # the library's per-device context
    torch.cuda.synchronize()
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    assert b.device_bytes(reqs) > 0


def test_bad_requests_are_rejected():
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97")
    s = st["yuv97"]
    out = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    b = wv.Batch()
    bad = [wv.ViewRequest(s, 99, 0.0, 0.0, 1.0, out), wv.ViewRequest(s, 0, 0.0, 0.0, 3.2, out),
           wv.ViewRequest(s, 0, float("nan"), 0.0, 1.0, out),
           wv.ViewRequest(s, 0, 0.0, 0.0, 1.0, out, True, float("inf"), 0.0, 0.2, 0.4),
           wv.ViewRequest(s, 0, 0.0, 0.0, 1.0, out, True, 0.0, 0.0, float("nan"), 0.4)]
    for r in bad:
        with pytest.raises(wv.WVError) as e:
            b.decode([r])
        assert e.value.code == -1
    b.decode([])
    assert b.sync_status() == 0


def _gaze_with_margin(p, yaw, pitch, r1, r2):
    """A gaze near the view centre whose keep decisions are at least 2e-4 rad
    from a tie in every cell (float32 and fp64 then decide alike)."""
    for k in range(50):
        gx, gy = 0.05 * math.sin(1.7 * k), 0.04 * math.cos(2.3 * k)
        if O.fovea_margin(p, yaw, pitch, gx, gy, r1, r2) > 2e-4:
            return gx, gy
    raise AssertionError("no gaze with a decision margin")


FOVEA_POSES = [(0.3, 0.1, math.radians(100), 0.35, 0.7), (2.8, -0.4, math.radians(110), 0.3, 0.6),
               (-1.0, 0.9, math.radians(90), 0.25, 0.5)]


@pytest.mark.parametrize("name", ["fov97", "fov53"])
def test_strip_targets_equal_square_targets(name):
    """The batched strip fine pass (foveated and not, edge strips as halves)
    gives the same viewports as square tiles for every target."""
    from paper_2208_10859_gb300 import wv
    _, p, _, _ = H.case(name)
    s = _streams(name)[name]
    outs = {}
    for strips in (True, False):
        b = wv.Batch()
        b.set_strips(strips)
        reqs = []
        for k, (yaw, pitch, fov, r1, r2) in enumerate(FOVEA_POSES):
            gx, gy = _gaze_with_margin(p, yaw, pitch, r1, r2)
            for fovea in (True, False):
                out = torch.zeros((96, 128, 4), dtype=torch.uint8, device="cuda")
                reqs.append(wv.ViewRequest(s, k % p.num_frames, yaw, pitch, fov, out, fovea, gx, gy, r1, r2))
        b.decode(reqs)
        torch.cuda.synchronize()
        assert b.sync_status() == 0
        outs[strips] = [r.out.cpu().numpy() for r in reqs]
        b.close()
    for a, c in zip(outs[True], outs[False]):
        np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("name", ["fov97", "fov53"])
def test_foveated_matches_oracle(name):
    """Foveated requests against the oracle's foveated decode (coefficients of
    levels 1 and 2 outside the kept cells set to zero, then the plain
    definition), with the float32 position candidates of the plain viewport
    test; foveation visibly changes the periphery; infinite radii give the
    unfoveated result."""
    from paper_2208_10859_gb300 import wv
    _, p, _, ost = H.case(name)
    s = _streams(name)[name]
    ow, oh = 128, 96
    b = wv.Batch()
    for k, (yaw, pitch, fov, r1, r2) in enumerate(FOVEA_POSES):
        frame = k % p.num_frames
        gx, gy = _gaze_with_margin(p, yaw, pitch, r1, r2)
        out = torch.zeros((oh, ow, 4), dtype=torch.uint8, device="cuda")
        full = torch.zeros_like(out)
        same = torch.zeros_like(out)
        b.decode([wv.ViewRequest(s, frame, yaw, pitch, fov, out, True, gx, gy, r1, r2),
                  wv.ViewRequest(s, frame, yaw, pitch, fov, full),
                  wv.ViewRequest(s, frame, yaw, pitch, fov, same, True, gx, gy, math.inf, math.inf)])
        torch.cuda.synchronize()
        assert b.sync_status() == 0
        assert b.stats()["surfaces"] == 3
        got = out.cpu().numpy()
        np.testing.assert_array_equal(same.cpu().numpy(), full.cpu().numpy())
        assert np.any(got != full.cpu().numpy())
        keep = O.fovea_keep(p, yaw, pitch, gx, gy, r1, r2)
        ref = [O.decode_plane(ost, frame, pl, keep) for pl in range(p.planes)]
        planes = [u8 for (_, u8) in ref]
        u, v = O.project(ow, oh, yaw, pitch, fov, p.width, p.height)
        eu, ev = H.position_error_bound(p, ow, oh, yaw, pitch, fov)
        u, v, eu, ev = u.ravel(), v.ravel(), eu.ravel(), ev.ravel()
        cand, flag = H.rgba_candidates(planes, p, u, v, eu, ev)
        g = got.reshape(-1, 4)
        ok = np.any(np.all(cand == g[:, None, :], axis=-1), axis=-1)
        if p.wavelet == O.WAVELET_97:
            alt = [H.other_rounding(x) for (x, _) in ref]
            cand2, _ = H.rgba_candidates(alt, p, u, v, eu, ev)
            ok |= np.any(np.all(cand2 == g[:, None, :], axis=-1), axis=-1)
        bad = ~ok & ~flag
        assert not np.any(bad), (k, int(bad.sum()))
        assert flag.sum() <= 0.01 * flag.size


def test_foveation_keeps_the_tile_set():
    """Foveation keeps the decoded region (the inverse transform still runs
    over every tile the viewport needs; only detail loads are skipped)."""
    from paper_2208_10859_gb300 import wv
    s = _streams("fov97")["fov97"]
    outs = [torch.zeros((96, 128, 4), dtype=torch.uint8, device="cuda") for _ in range(2)]
    b = wv.Batch()
    b.decode([wv.ViewRequest(s, 0, 0.3, 0.1, 1.7, outs[0], True, 0.0, 0.0, 0.2, 0.4)])
    t_fov = b.stats()["fine_tiles"]
    b.decode([wv.ViewRequest(s, 0, 0.3, 0.1, 1.7, outs[1])])
    assert b.stats()["fine_tiles"] == t_fov
    assert b.sync_status() == 0


def test_without_sharing_every_request_has_its_own_target():
    from paper_2208_10859_gb300 import wv
    st = _streams("yuv97", "ragged53")
    reqs = _requests(st, 6, seed=9)
    b = wv.Batch()
    b.set_sharing(False)
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.stats()["surfaces"] == len(reqs)
    for r in reqs:
        _assert_same(r, r.out.cpu().numpy())
    assert b.sync_status() == 0
