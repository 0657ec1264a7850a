"""The allocation-free whole-plane decode (wv_decode_plane_static).

Some callers of this library may not allocate GPU memory themselves (a
plug-in whose host application owns every device allocation), but hold a
stream's block table and coefficient blocks on the device already.  These
tests give the entry point exactly that: device copies of the table and
payload that the test owns, and an output buffer.  They call it through the
C ABI twice in a row and compare each result with the fp64 oracle's decode
of the same plane (bit-exact for 5/3; 9/7 float32 samples within the 9/7
tolerance of the other tests, 8-bit samples equal except next to a rounding
boundary) and with the regular wv_decode_full, and check the error word it
hands back.  The file name makes pytest collect it last."""
import ctypes
import struct

import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _device_table_and_payload(data: bytes):
    """Device copies of a stream's table and payload, and its block count."""
    nf, nbpf = struct.unpack_from("<I", data, 32)[0], struct.unpack_from("<I", data, 56)[0]
    n_payload, toff, poff = struct.unpack_from("<QQQ", data, 64)
    block = struct.unpack_from("<I", data, 40)[0]
    table = np.frombuffer(data, np.int32, nf * nbpf, toff)
    payload = np.frombuffer(data, np.int16, max(1, n_payload) * block * block if n_payload else 1,
                            poff if n_payload else 0)
    return (torch.from_numpy(table.copy()).cuda(), torch.from_numpy(payload.copy()).cuda(), max(1, n_payload))


def _desc(desc: dict):
    from paper_2208_10859_gb300 import wv
    return wv.StreamDesc(**{k: desc[k] for k, _ in wv.StreamDesc._fields_})


def _call(lib, d, payload, n_blocks, table, frame, plane, out, as_float, cs, status):
    return lib.wv_decode_plane_static(ctypes.byref(d), ctypes.c_void_p(payload.data_ptr()), n_blocks,
                                      ctypes.c_void_p(table.data_ptr()), frame, plane,
                                      ctypes.c_void_p(out.data_ptr()), as_float, cs, ctypes.byref(status))


@pytest.mark.parametrize("name", ["yuv53", "yuv97", "ragged97"])
def test_static_plane_decode_matches_oracle(name):
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    _, p, data, _ = H.case(name)
    table, payload, n_blocks = _device_table_and_payload(data)
    s = wv.Stream(data)
    d = _desc(s.desc)
    cs = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for frame in (0, p.num_frames - 1):
        ref = H.oracle_planes(name, frame)
        for plane in range(p.planes):
            ref_x, ref_u8 = ref[plane]
            h, w = ref_x.shape
            for as_float in (0, 1):
                dt = torch.float32 if as_float else torch.uint8
                full = torch.empty((h, w), dtype=dt, device="cuda")
                s.decode_full(frame, plane, full, as_float=bool(as_float))
                for _call_no in range(2):
                    out = torch.full((h, w), 7, dtype=dt, device="cuda")
                    status = ctypes.c_int(-99)
                    rc = _call(lib, d, payload, n_blocks, table, frame, plane, out, as_float, cs, status)
                    assert rc == 0 and status.value == 0, (rc, status.value)
                    a = out.cpu().numpy()
                    if as_float and p.wavelet == 1:
                        err = np.abs(a.astype(np.float64) - ref_x)
                        assert err.max() <= H.tol_97_levels() and err.max() <= H.reg_97_levels(), err.max()
                        assert np.abs(a - full.cpu().numpy()).max() <= H.reg_97_levels()
                    elif as_float:
                        np.testing.assert_array_equal(a, ref_x.astype(np.float32))
                    elif p.wavelet == 1:
                        assert not np.any((a != ref_u8) & ~H.near_half(ref_x))
                    else:
                        np.testing.assert_array_equal(a, ref_u8)
    assert s.sync_status() == 0


def test_static_plane_decode_reports_bad_table_entries():
    """A table entry at or above the payload's block count is read as an
    absent (all-zero) block and reported through the status word; nothing
    outside the payload is read."""
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    _, p, data, st = H.case("yuv97")
    table, payload, n_blocks = _device_table_and_payload(data)
    d = _desc(wv.Stream(data).desc)
    cs = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the first stored block of frame 0 now points past the payload
    tab = table.cpu().numpy()
    k = int(np.nonzero(tab >= 0)[0][0])
    bad = table.clone()
    bad[k] = n_blocks + 5
    h, w = p.height, p.width
    out = torch.empty((h, w), dtype=torch.float32, device="cuda")
    status = ctypes.c_int(-99)
    assert _call(lib, d, payload, n_blocks, bad, 0, 0, out, 1, cs, status) == 0
    assert status.value == -2   # WV_ERR_FORMAT
    # the next call with the intact table starts from a clear word
    assert _call(lib, d, payload, n_blocks, table, 0, 0, out, 1, cs, status) == 0
    assert status.value == 0


def test_static_plane_decode_rejects_oversized_planes():
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    d = wv.StreamDesc(16384, 16384, 1, 0, 5, 1, 2, 1, 256, 0, 4.0)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    status = ctypes.c_int(0)
    rc = lib.wv_decode_plane_static(ctypes.byref(d), ptr, 1, ptr, 0, 0, ptr, 0, None, ctypes.byref(status))
    assert rc == -5
    d.levels = 9
    assert lib.wv_decode_plane_static(ctypes.byref(d), ptr, 1, ptr, 0, 0, ptr, 0, None, None) == -1
    d.levels = 5
    d.width = d.height = 1024
    assert lib.wv_decode_plane_static(ctypes.byref(d), ptr, 0, ptr, 0, 0, ptr, 0, None, None) == -1
