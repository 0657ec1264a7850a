"""The oracle's C core under host-side sanitizers (AddressSanitizer and
UndefinedBehaviorSanitizer; the GPU side has its bounds-check build
instead): in a child process that loads the sanitized build, 1D and 2D
transforms of every length and level count the tests use, and whole
encode/decode round trips of small streams, run without a report and give
the same results as the normal build."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle as O
import synth
rng = np.random.default_rng(5)
out = []
for n in (2, 4, 6, 8, 10, 16, 30, 64, 130, 256):
    for wav in (O.WAVELET_53, O.WAVELET_97):
        x = rng.integers(-300, 300, n) if wav == O.WAVELET_53 else rng.normal(0, 50, n)
        y = O.fwd1d(x, wav)
        out.append(y)
        out.append(O.inv1d(y, wav))
for (w, h, lev) in ((8, 8, 2), (64, 32, 4), (320, 192, 4), (96, 64, 3), (512, 256, 6)):
    for wav in (O.WAVELET_53, O.WAVELET_97):
        img = rng.integers(0, 256, (h, w)).astype(np.float64)
        c = O.fwd2d(img, lev, wav)
        out.append(c)
        out.append(O.inv2d(c, lev, wav))
frames = synth.equirect_gop(64, 2, seed=8, n_discs=2)
for wav, step in ((O.WAVELET_97, 4.0), (O.WAVELET_53, 1.0)):
    p = O.Params(64, 64, 3, 1, 3, wav, 2, 1, 32, step)
    st = O.Stream(O.encode(frames, p))
    for f in range(2):
        for pl in range(3):
            out.append(O.decode_plane(st, f, pl)[0])
np.savez(OUT, *[np.asarray(a, np.float64) for a in out])
print("done")
'''


def _run(tmp_path, sanitize: bool):
    import oracle as O
    env = dict(os.environ)
    outp = str(tmp_path / ("san.npz" if sanitize else "plain.npz"))
    if sanitize:
        O.build_sanitized()
        asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(asan) or not os.path.exists(asan):
            pytest.skip("no AddressSanitizer runtime")
        env.update(WV_ORACLE_SANITIZE="1", LD_PRELOAD=asan,
                   ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:abort_on_error=0:exitcode=23",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1:exitcode=24")
    script = f"ROOT = {ROOT!r}\nOUT = {outp!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", script], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "done" in r.stdout, (r.returncode, r.stdout[-1000:], r.stderr[-4000:])
    return outp


def test_oracle_core_is_clean_under_asan_and_ubsan(tmp_path):
    import numpy as np
    plain = np.load(_run(tmp_path, False))
    san = np.load(_run(tmp_path, True))
    assert sorted(plain.files) == sorted(san.files)
    for k in plain.files:
        np.testing.assert_array_equal(plain[k], san[k])
