"""The allocation-free whole-plane decode (wv_decode_plane_static).

Some callers of this library may not allocate GPU memory themselves (a
plug-in whose host application owns every device allocation), but hold a
stream's block table and coefficient blocks on the device already.  This
test gives the entry point exactly that: device copies of the table and
payload that the test owns, and an output buffer.  It calls the entry point
through the C ABI twice in a row and compares each result with the regular
wv_decode_full of the same stream (bit-exact for 5/3 and for 8-bit output,
float32 samples within the 9/7 tolerance of the other tests).  The file name
makes pytest collect it last."""
import ctypes
import struct

import numpy as np
import pytest

import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _device_table_and_payload(data: bytes):
    nf, nbpf = struct.unpack_from("<I", data, 32)[0], struct.unpack_from("<I", data, 56)[0]
    n_payload, toff, poff = struct.unpack_from("<QQQ", data, 64)
    block = struct.unpack_from("<I", data, 40)[0]
    table = np.frombuffer(data, np.int32, nf * nbpf, toff)
    payload = np.frombuffer(data, np.int16, max(1, n_payload) * block * block if n_payload else 1,
                            poff if n_payload else 0)
    return (torch.from_numpy(table.copy()).cuda(), torch.from_numpy(payload.copy()).cuda())


def _desc(desc: dict):
    from paper_2208_10859_gb300 import wv
    return wv.StreamDesc(**{k: desc[k] for k, _ in wv.StreamDesc._fields_})


@pytest.mark.parametrize("name", ["yuv53", "yuv97", "ragged97"])
def test_static_plane_decode_matches_decode_full(name):
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    _, p, data, _ = H.case(name)
    table, payload = _device_table_and_payload(data)
    s = wv.Stream(data)
    d = _desc(s.desc)
    cs = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for frame in (0, p.num_frames - 1):
        for plane in range(p.planes):
            w, h = (p.width, p.height) if plane == 0 or not p.chroma_420 else (p.width // 2, p.height // 2)
            for as_float in (0, 1):
                dt = torch.float32 if as_float else torch.uint8
                ref = torch.empty((h, w), dtype=dt, device="cuda")
                s.decode_full(frame, plane, ref, as_float=bool(as_float))
                for _call in range(2):
                    out = torch.full((h, w), 7, dtype=dt, device="cuda")
                    rc = lib.wv_decode_plane_static(ctypes.byref(d), ctypes.c_void_p(payload.data_ptr()),
                                                    ctypes.c_void_p(table.data_ptr()), frame, plane,
                                                    ctypes.c_void_p(out.data_ptr()), as_float, cs)
                    assert rc == 0, rc
                    torch.cuda.synchronize()
                    a, b = out.cpu().numpy(), ref.cpu().numpy()
                    if as_float and p.wavelet == 1:
                        assert np.abs(a.astype(np.float64) - b).max() <= H.tol_97_levels()
                    else:
                        np.testing.assert_array_equal(a, b)
    assert s.sync_status() == 0


def test_static_plane_decode_rejects_oversized_planes():
    from paper_2208_10859_gb300 import wv
    lib = wv._lib()
    d = wv.StreamDesc(16384, 16384, 1, 0, 5, 1, 2, 1, 256, 0, 4.0)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.wv_decode_plane_static(ctypes.byref(d), ptr, ptr, 0, 0, ptr, 0, None)
    assert rc == -5
    d.levels = 9
    assert lib.wv_decode_plane_static(ctypes.byref(d), ptr, ptr, 0, 0, ptr, 0, None) == -1
