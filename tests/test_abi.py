"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/wv.h declares, validates stream bytes, and refuses to run
without a CUDA device instead of falling back to the CPU."""
import ctypes
import os
import re
import struct

import pytest

import oracle as O
import helpers as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_10859_gb300 import build, wv
    build.build()
    return wv._lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wv_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    from paper_2208_10859_gb300 import wv
    assert sorted(wv.exported_symbols()) == names


def test_strerror_names_every_code(lib):
    for code in range(0, -8, -1):
        assert lib.wv_strerror(code).decode() not in ("", "unknown error")
    assert lib.wv_strerror(-99).decode() == "unknown error"


def test_query_parses_oracle_streams(lib):
    from paper_2208_10859_gb300 import wv
    for name in ("cfg1", "yuv97", "ragged53"):
        _, p, data, _ = H.case(name)
        desc, need = wv.query(data)
        assert (desc["width"], desc["height"], desc["planes"], desc["levels"], desc["wavelet"],
                desc["num_frames"], desc["tlevels"], desc["block"]) == \
            (p.width, p.height, p.planes, p.levels, p.wavelet, p.num_frames, p.tlevels, p.block)
        assert need >= len(data) - 128


def test_query_with_host_payload_excludes_the_store(lib):
    """WV_OPEN_HOST_PAYLOAD: the device size drops by at least the stored
    blocks (host memory holds them); unknown flags are refused."""
    from paper_2208_10859_gb300 import wv
    for name in ("yuv97", "ragged53"):
        _, p, data, st = H.case(name)
        d0, dev = wv.query(data)
        d1, host = wv.query(data, wv.WV_OPEN_HOST_PAYLOAD)
        assert d0 == d1
        assert dev - host >= st.payload.size * 2
    with pytest.raises(wv.WVError) as e:
        wv.query(data, 4)
    assert e.value.code == -1


def test_open_with_unknown_flags_is_refused(lib):
    _, _, data, _ = H.case("yuv97")
    h = ctypes.c_void_p()
    rc = lib.wv_open_stream_ex(ctypes.c_char_p(data), len(data), None, 0, None, 8, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_query_rejects_corrupt_streams(lib):
    from paper_2208_10859_gb300 import wv
    _, _, data, _ = H.case("yuv97")
    bad_cases = [data[:100], b"XXXX" + data[4:], data[: len(data) // 2]]
    toff = struct.unpack_from("<Q", data, 72)[0]
    b = bytearray(data)
    struct.pack_into("<i", b, toff + 8, 10 ** 6)          # slot beyond the payload
    bad_cases.append(bytes(b))
    b = bytearray(data)
    struct.pack_into("<I", b, 24, 9)                       # 9 levels: unsupported
    bad_cases.append(bytes(b))
    b = bytearray(data)
    struct.pack_into("<I", b, 40, 48)                      # block not a power of two
    bad_cases.append(bytes(b))
    for bad in bad_cases:
        with pytest.raises(wv.WVError) as e:
            wv.query(bad)
        assert e.value.code == -2


def test_open_without_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    _, _, data, _ = H.case("cfg1")
    h = ctypes.c_void_p()
    rc = lib.wv_open_stream(ctypes.c_char_p(data), len(data), None, 0, None, ctypes.byref(h))
    assert rc == -4 and not h.value


def test_encode_sizes(lib):
    from paper_2208_10859_gb300 import wv
    d = wv.StreamDesc(8192, 8192, 3, 1, 5, 1, 8, 1, 256, 0, 4.0)
    scratch, cap = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.wv_encode_sizes(ctypes.byref(d), ctypes.byref(scratch), ctypes.byref(cap)) == 0
    assert cap.value >= 8 * 1536 * 256 * 256 * 2
    d.levels = 7
    assert lib.wv_encode_sizes(ctypes.byref(d), ctypes.byref(scratch), ctypes.byref(cap)) == -1


def test_null_stream_arguments_are_rejected(lib):
    assert lib.wv_launches_per_viewport(None) == -1
    assert lib.wv_set_decode_mode(None, 0) == -1
    assert lib.wv_decode_viewport(None, 0, 0.0, 0.0, 1.0, None) == -1
    assert lib.wv_stream_sync_status(None) == -1


def test_query_parses_and_rejects_paper_streams(lib):
    import struct
    import synth
    from oracle import paper_format as PF
    from paper_2208_10859_gb300 import wv
    fr = synth.equirect_gop(64, 4, seed=9, n_discs=2)
    data = PF.encode(fr, PF.PaperParams(64, 64, 3, 1, 2, 4, 2, alpha=0.0, alpha_t=0.0))
    desc, need = wv.query(data)
    assert (desc["quant"], desc["block"], desc["tlevels"], desc["wavelet"]) == (1, 32, 2, 1)
    assert need > 0
    off = struct.unpack_from("<Q", data, 128)[0]
    b = bytearray(data)
    struct.pack_into("<I", b, off, 10 ** 8)                  # record count past the end
    bad = [data[:200], bytes(b)]
    b = bytearray(data)
    nbpf = struct.unpack_from("<I", data, 40)[0]
    ends = off + 8 + 16 * 3
    struct.pack_into("<I", b, ends, 10 ** 6)                 # BlockEnd beyond the record count
    bad.append(bytes(b))
    for x in bad:
        with pytest.raises(wv.WVError) as e:
            wv.query(x)
        assert e.value.code == -2
