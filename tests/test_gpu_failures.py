"""Failure detection without a GPU fault.

* The batch tile decode's bounded wait (a fine tile waiting for its decode
  target's coarse tiles): with a poll limit of zero every such wait gives up
  at once; the batch completes, reports WV_ERR_TIMEOUT through
  wv_batch_sync_status, and the next batch with the default limit decodes
  exactly as the per-viewport path again.
* Device allocation failures injected on the host (the library's own
  allocations report failure as if the device were full): wv_open_stream
  without caller memory and wv_batch_decode return WV_ERR_OOM, leave nothing
  behind, and work again once the injection is used up."""
import ctypes
import math

import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FOV = math.radians(100)


def _requests(s, n, out):
    from paper_2208_10859_gb300 import wv
    poses = [(0.3 + 0.5 * k, 0.1 - 0.05 * k) for k in range(n)]
    return [wv.ViewRequest(s, k % 2, y, p, FOV, out[k]) for k, (y, p) in enumerate(poses)], poses


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_2208_10859_gb300 import wv
    _, p, data, _ = H.case("yuv97")           # 4 levels: coarse and fine tiles, so fine tiles wait
    s = wv.Stream(data)
    outs = [torch.zeros((48, 48, 4), dtype=torch.uint8, device="cuda") for _ in range(3)]
    reqs, poses = _requests(s, 3, outs)
    b = wv.Batch()
    b.set_strips(False)   # square fine tiles: they wait for their target's coarse tiles in the same launch
    b.set_wait_limit(0)
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.sync_status() == -6            # WV_ERR_TIMEOUT
    assert b.sync_status() == 0             # the word was cleared by the read
    # the default limit again: the same requests decode as the per-viewport path
    b.set_wait_limit(1 << 21)
    b.decode(reqs)
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    for k, (yaw, pitch) in enumerate(poses):
        ref = torch.zeros_like(outs[k])
        s.decode_viewport(k % 2, yaw, pitch, FOV, ref)
        torch.cuda.synchronize()
        assert torch.equal(ref, outs[k])
    with pytest.raises(wv.WVError):
        b.set_wait_limit(-1)
    b.close()
    assert s.sync_status() == 0


def test_injected_allocation_failures_report_oom():
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    _, p, data, _ = H.case("yuv97")
    buf = np.frombuffer(data, np.uint8)
    h = ctypes.c_void_p()
    # wv_open_stream with no caller memory allocates the stream store itself
    lib.wv_debug_fail_device_allocs(1)
    rc = lib.wv_open_stream(buf.ctypes.data_as(ctypes.c_void_p), len(data), None, 0, None, ctypes.byref(h))
    assert rc == -3 and not h.value          # WV_ERR_OOM, no stream returned
    rc = lib.wv_open_stream(buf.ctypes.data_as(ctypes.c_void_p), len(data), None, 0, None, ctypes.byref(h))
    assert rc == 0 and h.value               # the injection is used up
    lib.wv_close_stream(h)
    # a batch allocates its arena on first use
    s = wv.Stream(data)
    outs = [torch.zeros((32, 32, 4), dtype=torch.uint8, device="cuda") for _ in range(2)]
    reqs, _ = _requests(s, 2, outs)
    b = wv.Batch()
    lib.wv_debug_fail_device_allocs(1)
    with pytest.raises(wv.WVError) as ei:
        b.decode(reqs)
    assert ei.value.code == -3
    b.decode(reqs)                           # allocation succeeds now
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    lib.wv_debug_fail_device_allocs(0)
    b.close()
    assert s.sync_status() == 0
