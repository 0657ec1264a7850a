"""GPU tests of the serving loop (wv_server_*): each result is the same alone
and in a mix of concurrent traffic, admission by device memory splits
batches, the stream cache evicts and re-uploads, bad requests are refused."""
import math
import threading

import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("yuv97", "ragged53", "fov97")


def _server(**kw):
    from paper_2208_10859_gb300 import wv
    sv = wv.Server(**kw)
    ids = {n: sv.add_stream(H.case(n)[2]) for n in NAMES}
    return sv, ids


def _probe_requests(k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        name = NAMES[i % len(NAMES)]
        p = H.case(name)[1]
        fov = math.radians(float(rng.uniform(80, 120)))
        fovea = name == "fov97" and i % 2 == 1
        out.append(dict(name=name, frame=int(rng.integers(p.num_frames)),
                        yaw=float(rng.uniform(-math.pi, math.pi)), pitch=float(rng.uniform(-1.0, 1.0)),
                        fov=fov, fovea=fovea, gx=0.05, gy=-0.03, r1=0.3, r2=0.6,
                        size=[(64, 48), (96, 64)][i % 2]))
    return out


def _submit(sv, ids, r, out):
    return sv.submit(ids[r["name"]], r["frame"], r["yaw"], r["pitch"], r["fov"], out,
                     r["fovea"], r["gx"], r["gy"], r["r1"], r["r2"])


def _alloc(r):
    w, h = r["size"]
    return torch.zeros((h, w, 4), dtype=torch.uint8, device="cuda")


def test_result_same_alone_and_in_the_mix():
    from paper_2208_10859_gb300 import wv
    sv, ids = _server(slots=2, max_batch=16)
    probes = _probe_requests(9, seed=1)
    alone = []
    for r in probes:                                   # one at a time, idle server
        out = _alloc(r)
        sv.wait(_submit(sv, ids, r, out))
        alone.append(out.cpu().numpy())
    # the unfoveated results also equal the plain per-viewport decode
    streams = {n: wv.Stream(H.case(n)[2]) for n in NAMES}
    for r, a in zip(probes, alone):
        if not r["fovea"]:
            one = _alloc(r)
            streams[r["name"]].decode_viewport(r["frame"], r["yaw"], r["pitch"], r["fov"], one)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(one.cpu().numpy(), a)
    sv.reset_stats()
    # the same probes inside background traffic submitted from two threads
    background = _probe_requests(80, seed=2)
    outs = [_alloc(r) for r in probes]
    bg_outs = [_alloc(r) for r in background]
    tickets, lock = [], threading.Lock()

    def client(reqs, bufs):
        for r, o in zip(reqs, bufs):
            t = _submit(sv, ids, r, o)
            with lock:
                tickets.append(t)

    th = [threading.Thread(target=client, args=(background[:40], bg_outs[:40])),
          threading.Thread(target=client, args=(background[40:], bg_outs[40:]))]
    for t in th:
        t.start()
    probe_tickets = [_submit(sv, ids, r, o) for r, o in zip(probes, outs)]
    for t in th:
        t.join()
    for t in probe_tickets + tickets:
        sv.wait(t)
    for a, o in zip(alone, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), a)
    st = sv.stats()
    assert st["completed"] == len(probes) + len(background) and st["failed"] == 0
    assert st["batched_requests"] == st["completed"]
    assert st["batches"] < st["completed"], st          # requests were batched together
    lat = sv.latencies()
    assert len(lat) == st["completed"] and np.all(lat > 0)
    sv.close()


def test_admission_by_device_memory_splits_batches():
    from paper_2208_10859_gb300 import wv
    reqs = _probe_requests(12, seed=3)
    # the memory of two requests' batch: no batch may hold more
    probe = wv.Batch()
    streams = {n: wv.Stream(H.case(n)[2]) for n in NAMES}
    bufs = [_alloc(r) for r in reqs]
    vr = [wv.ViewRequest(streams[r["name"]], r["frame"], r["yaw"], r["pitch"], r["fov"], b)
          for r, b in zip(reqs, bufs)]
    two = max(probe.device_bytes(vr[i:i + 2]) for i in range(0, len(vr), 2))
    sv, ids = _server(slots=1, max_batch=16, arena_bytes=int(two * 1.3))
    tickets = [_submit(sv, ids, r, b) for r, b in zip(reqs, bufs)]
    for t in tickets:
        sv.wait(t)
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_batch_bytes"] <= int(two * 1.3)
    assert st["batches"] >= len(reqs) // 4
    sv.close()


def test_stream_cache_evicts_and_reuploads():
    from paper_2208_10859_gb300 import wv
    need = {n: wv.query(H.case(n)[2])[1] for n in NAMES}
    sv, ids = _server(slots=1, max_batch=4, cache_bytes=max(need.values()) + 1)
    streams = {n: wv.Stream(H.case(n)[2]) for n in NAMES}
    reqs = _probe_requests(9, seed=4)
    for r in reqs:
        r["fovea"] = False
        out = _alloc(r)
        sv.wait(_submit(sv, ids, r, out))
        one = _alloc(r)
        streams[r["name"]].decode_viewport(r["frame"], r["yaw"], r["pitch"], r["fov"], one)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(one.cpu().numpy(), out.cpu().numpy())
    st = sv.stats()
    assert st["evictions"] >= 2 and st["uploads"] >= 3, st
    assert st["resident_bytes"] <= max(need.values()) + 1
    sv.close()


def test_bad_requests_are_refused():
    from paper_2208_10859_gb300 import wv
    sv, ids = _server(slots=1, max_batch=4)
    out = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    for args in [(99, 0, 0.0, 0.0, 1.0), (ids["yuv97"], 99, 0.0, 0.0, 1.0),
                 (ids["yuv97"], 0, 0.0, 0.0, 3.3)]:
        with pytest.raises(wv.WVError) as e:
            sv.submit(*args, out)
        assert e.value.code == -1
    with pytest.raises(wv.WVError):
        sv.add_stream(b"not a stream")
    sv.close()
