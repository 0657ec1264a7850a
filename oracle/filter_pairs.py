"""Training pairs for the learned post-filter, made by the oracle codec.

Test and data infrastructure, like the rest of oracle/: the library never
imports it.  It writes, per quantiser step, (decoded, original) viewport
luma pairs that the post-filter trainer
(paper_2208_10859_gb300/train_postfilter.py --pairs) reads from disk.

Recipe (the stream shape of the benchmark):
* frames: seeded synthetic 8192 x 8192 equirectangular groups of 8 frames
  (synth.equirect_gop, 50 discs), seeds disjoint from the benchmark's;
  crops of 2048 x 2048 luma (1024 x 1024 chroma) at seeded 32-aligned
  origins keep the texture statistics of the 8192 frames (the noise spectrum
  and the disc textures are defined per pixel);
* coding: the oracle encoder and decoder (this package) with YCbCr 4:2:0,
  5-level CDF 9/7, one inter-frame Haar level over the 8 frames, 256 x 256
  blocks, dead-zone step Delta;
* viewports: a crop is projected as an equirectangular frame (Sec. 3.6),
  540 x 540 pixels at 110 degrees, which samples the 2048-wide crop as a
  2160 x 2160 viewport at 110 degrees samples the 8192-wide frame (the same
  ratio of viewport to frame pixel angle everywhere in the image);
  random yaw, pitch uniform in [-45, 45] degrees; luma of both the decoded
  and the original planes by the oracle's fixed-point bilinear filter at
  the same positions (what the filtered decode feeds the network and what
  the lossless reference shows).

    python -m oracle.filter_pairs --out DIR --step 4 --step 12 [--seeds 11,12] [--crops 4] [--views 6]
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import WAVELET_97, Params, Stream, bilinear, decode_plane, encode, project

FRAME, CROP, VIEW, FOV_DEG, FRAMES = 8192, 2048, 540, 110.0, 8


def crop_origins(n: int, seed: int):
    """n crop origins (x, y) in the 8192 frame, multiples of 32."""
    rng = np.random.default_rng(seed + 555)
    k = (FRAME - CROP) // 32
    return [(32 * int(rng.integers(0, k + 1)), 32 * int(rng.integers(0, k + 1))) for _ in range(n)]


def crop_gop(frames, x0: int, y0: int):
    """The 2048 x 2048 crop (4:2:0 chroma 1024 x 1024) of every frame."""
    return [(f[0][y0:y0 + CROP, x0:x0 + CROP].copy(),
             f[1][y0 // 2:y0 // 2 + CROP // 2, x0 // 2:x0 // 2 + CROP // 2].copy(),
             f[2][y0 // 2:y0 // 2 + CROP // 2, x0 // 2:x0 // 2 + CROP // 2].copy()) for f in frames]


def view_pairs(gop, step: float, views: int, seed: int):
    """(decoded, original) viewport luma, uint8 arrays (n, VIEW, VIEW), of a
    cropped group coded at `step` by the oracle codec."""
    p = Params(CROP, CROP, 3, 1, 5, WAVELET_97, FRAMES, 1, 256, float(step))
    st = Stream(encode(gop, p))
    rng = np.random.default_rng(seed)
    fov = math.radians(FOV_DEG)
    dec, org = [], []
    for f in range(FRAMES):
        y_dec = decode_plane(st, f, 0)[1]
        for _ in range(views):
            yaw = float(rng.uniform(-math.pi, math.pi))
            pitch = float(rng.uniform(-math.pi / 4, math.pi / 4))
            u, v = project(VIEW, VIEW, yaw, pitch, fov, CROP, CROP)
            dec.append(bilinear(y_dec, u, v))
            org.append(bilinear(gop[f][0], u, v))
    return np.stack(dec), np.stack(org)


def make(out: str, steps, seeds, crops: int, views: int) -> list:
    """Write pairs_q{step}.npz (arrays dec, org) under out for every step;
    returns the paths."""
    import synth
    os.makedirs(out, exist_ok=True)
    dec = {s: [] for s in steps}
    org = {s: [] for s in steps}
    for seed in seeds:
        frames = synth.equirect_gop(FRAME, FRAMES, seed=seed, n_discs=50)
        for c, (x0, y0) in enumerate(crop_origins(crops, seed)):
            gop = crop_gop(frames, x0, y0)
            for step in steps:
                d, o = view_pairs(gop, step, views, seed * 100 + c)
                dec[step].append(d)
                org[step].append(o)
        del frames
    paths = []
    for step in steps:
        path = os.path.join(out, f"pairs_q{int(step)}.npz")
        np.savez(path, dec=np.concatenate(dec[step]), org=np.concatenate(org[step]))
        paths.append(path)
    return paths


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--step", type=float, action="append", required=True)
    ap.add_argument("--seeds", default="11,12")
    ap.add_argument("--crops", type=int, default=4)
    ap.add_argument("--views", type=int, default=6)
    args = ap.parse_args()
    seeds = [int(s) for s in args.seeds.split(",")]
    t = time.time()
    for path in make(args.out, args.step, seeds, args.crops, args.views):
        print(path, flush=True)
    print(f"{time.time() - t:.1f} s", flush=True)


if __name__ == "__main__":
    main()
