"""The C ABI's host code under AddressSanitizer and UndefinedBehaviorSanitizer
(libwv_san.so; device code unchanged, no GPU needed): the stream parsers
of both formats take valid streams, every truncation of them, seeded byte
corruptions and random bytes, and answer WV_OK or a negative error code
without a sanitizer report; the ABI's argument checks and the refusal to
run without a CUDA device hold in that build too."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)
from paper_2208_10859_gb300 import build, wv
assert wv.lib_path() == build.LIB_SAN
L = wv._lib()
import oracle as O
from oracle import paper_format as PF
import synth

fr = synth.equirect_gop(64, 4, seed=9, n_discs=2)
streams = [
    O.encode(fr[:2], O.Params(64, 64, 3, 1, 3, O.WAVELET_97, 2, 1, 32, 4.0)),
    O.encode(fr, O.Params(64, 64, 3, 1, 2, O.WAVELET_53, 4, 2, 16, 1.0)),
    PF.encode(fr, PF.PaperParams(64, 64, 3, 1, 2, 4, 2, alpha=0.1, alpha_t=0.005)),
]
desc = wv.StreamDesc()
need = ctypes.c_size_t()
rng = np.random.default_rng(17)
calls = bad = 0

def query(b):
    global calls, bad
    buf = ctypes.create_string_buffer(bytes(b), len(b))   # exactly the bytes: overreads are caught
    for flags in (0, 1):
        rc = L.wv_stream_query_ex(buf, len(b), flags, ctypes.byref(desc), ctypes.byref(need))
        assert rc == 0 or -8 < rc < 0, rc
        calls += 1
        bad += rc != 0

for s in streams:
    query(s)
    assert L.wv_stream_query(ctypes.create_string_buffer(s, len(s)), len(s), ctypes.byref(desc), None) == 0
    for n in sorted(set([0, 1, 4, 87, 88, 127, 128, 129] + list(range(0, len(s), max(1, len(s) // 97))))):
        query(s[:n])
    for _ in range(300):
        b = bytearray(s)
        for _ in range(int(rng.integers(1, 5))):
            i = int(rng.integers(0, min(len(b), 4096)))
            b[i] = int(rng.integers(0, 256))
        query(b)
for n in (16, 128, 1000, 5000):
    query(rng.integers(0, 256, n, dtype=np.uint8).tobytes())
# stream descriptions of every shape, valid or not: the geometry builder
scratch, biggest = ctypes.c_size_t(), ctypes.c_size_t()
ok_desc = 0
for _ in range(400):
    d = wv.StreamDesc()
    d.width, d.height = (int(x) for x in rng.choice([0, 2, 30, 32, 64, 96, 320, 2048, 16384, 16416, -32], 2))
    d.planes = int(rng.choice([0, 1, 2, 3, 4]))
    d.chroma_420 = int(rng.integers(-1, 3))
    d.levels = int(rng.integers(-1, 9))
    d.wavelet = int(rng.integers(-1, 3))
    d.num_frames = int(rng.choice([0, 1, 2, 3, 4, 8]))
    d.tlevels = int(rng.integers(-1, 5))
    d.block = int(rng.choice([0, 8, 16, 24, 32, 256, 512]))
    d.quant = int(rng.integers(-1, 3))
    d.step = float(rng.choice([0.0, 1.0, 2.5, 4.0, -1.0, float("nan")]))
    d.stereo = int(rng.integers(-1, 3))
    rc = L.wv_encode_sizes(ctypes.byref(d), ctypes.byref(scratch), ctypes.byref(biggest))
    assert rc == 0 or -8 < rc < 0, rc
    ok_desc += rc == 0
for s in streams[:2]:   # the descriptions of valid streams
    assert L.wv_stream_query(ctypes.create_string_buffer(s, len(s)), len(s), ctypes.byref(desc), None) == 0
    assert L.wv_encode_sizes(ctypes.byref(desc), ctypes.byref(scratch), ctypes.byref(biggest)) == 0
    assert biggest.value > 0
# argument checks and no CUDA device: errors, never a CPU fallback
assert L.wv_stream_query(None, 0, None, None) < 0
assert L.wv_decode_viewport(None, 0, 0.0, 0.0, 1.0, None) == -1
assert L.wv_stream_sync_status(None) == -1
print("done", calls, bad)
'''


def test_host_code_is_clean_under_asan_and_ubsan():
    from paper_2208_10859_gb300 import build
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["gcc", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("no sanitizer runtimes")
    build.build(sanitize=True)
    env = dict(os.environ, WV_SANITIZE="1", LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:exitcode=23:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1:exitcode=24",
               CUDA_VISIBLE_DEVICES="")
    script = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", script], env=env, cwd=HERE, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0 and "done" in r.stdout, (r.returncode, r.stdout[-1000:], r.stderr[-4000:])
    calls, bad = (int(x) for x in r.stdout.split("done")[1].split())
    assert calls > 2000 and 0 < bad < calls
