"""The WV_CHECKED build (the bounds-check substitute for a sanitizer): the
kernels test the indices their data decide (table entries against the
payload's block count, output, LL_2 and tap offsets against their planes),
record WV_ERR_DEVICE and skip the access instead of faulting.  On small
valid streams the checked library must decode exactly what the oracle
decodes and leave every error word at 0.  It runs in a child process with
WV_CHECKED=1, which loads libwv_checked.so (built on first use)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import math, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)
from paper_2208_10859_gb300 import build, wv
assert wv.lib_path() == build.LIB_CHECKED
build.build(checked=True)
import oracle as O
import helpers as H
import synth

def cases():
    for name in ("yuv97", "cfg1", "ragged97", "fov97"):
        frames, p, data, st = H.case(name)
        yield name, p, data, st
    fr = synth.equirect_gop(64, 2, seed=41, n_discs=2)
    p = O.Params(64, 64, 3, 1, 3, O.WAVELET_97, 2, 1, 32, 4.0)
    data = O.encode(fr, p)
    yield "64x64", p, data, O.Stream(data)

for name, p, data, st in cases():
    s = wv.Stream(data)
    for pl in range(p.planes):
        w, h = O.plane_dims(p, pl)
        u8 = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        s.decode_full(p.num_frames - 1, pl, u8)
        torch.cuda.synchronize()
        x, ref = O.decode_plane(st, p.num_frames - 1, pl)
        diff = u8.cpu().numpy() != ref
        if p.wavelet == O.WAVELET_53:
            assert not diff.any(), (name, pl)
        else:
            assert not np.any(diff & ~H.near_half(x)), (name, pl, int(diff.sum()))
    for k, (yaw, pitch) in enumerate([(0.3, 0.2), (3.0, -1.3)]):
        out = torch.zeros((48, 64, 4), dtype=torch.uint8, device="cuda")
        s.decode_viewport(k % p.num_frames, yaw, pitch, math.radians(100), out)
        reqs = [wv.ViewRequest(s, k % p.num_frames, yaw, pitch, math.radians(100),
                               torch.zeros_like(out), fovea, 0.0, 0.0, 0.3, 0.6) for fovea in (False, True)]
        wv.decode_batch(reqs)
        torch.cuda.synchronize()
        assert torch.equal(reqs[0].out, out), name
    assert s.sync_status() == 0, name
    s.close()
print("checked ok")
'''


def test_checked_build_decodes_small_streams_without_errors():
    env = dict(os.environ, WV_CHECKED="1")
    script = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", script], env=env, cwd=HERE, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
