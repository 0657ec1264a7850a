"""Seeded synthetic inputs: 8-bit frames, head poses and reconstruction masks.

This module is the only code shared by the CPU oracle tests and the GPU path.
It draws pixels, angles and masks from seeded generators and holds none of the
codec's arithmetic (no wavelet, no quantiser, no projection).

The paper evaluates on 8192x8192 360-degree videos (Sec. 4.1: CGI scenes and
real recordings) that are not available here.  The frames below stand in for
them with the same shape: equirectangular 8-bit YCbCr 4:2:0, a band-limited
noise background with a natural-image-like 1/f^1.5 spectrum, and textured discs
that move a few pixels per frame so that the inter-frame (temporal) transform
of Sec. 3.2 sees realistic small motion.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gradient_rects_frame",
    "bandlimited_noise",
    "disc_params",
    "equirect_gop",
    "random_poses",
    "random_cell_mask",
]


def gradient_rects_frame(size: int = 512, seed: int = 1, n_rects: int = 20,
                         noise_sigma: float = 8.0) -> np.ndarray:
    """One 8-bit grayscale frame: a smooth gradient a*x + b*y + c, 20 filled
    rectangles of random grey level, then Gaussian noise (sigma 8) over all of
    it, clipped to 0..255.  Used for the lossless 5/3 round-trip workload."""
    rng = np.random.default_rng(seed)
    h = w = int(size)
    a, b = rng.uniform(-0.2, 0.2, 2)
    c = rng.uniform(80.0, 176.0)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = a * (xx - w / 2) + b * (yy - h / 2) + c
    for _ in range(n_rects):
        x0, y0 = rng.integers(0, w, 2)
        rw, rh = rng.integers(max(2, w // 64), max(3, w // 4), 2)
        img[y0:y0 + rh, x0:x0 + rw] = rng.uniform(0.0, 255.0)
    img += rng.normal(0.0, noise_sigma, (h, w))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def bandlimited_noise(h: int, w: int, seed: int, mean: float, std: float,
                      cutoff: float = 1.0 / 16.0, slope: float = 1.5) -> np.ndarray:
    """White Gaussian noise shaped by a 1/f^slope amplitude spectrum and cut
    off at `cutoff` cycles/pixel (1/16 = one eighth of Nyquist), rescaled to
    the given mean and standard deviation.  Returns float32."""
    from scipy import fft as sfft

    rng = np.random.default_rng(seed)
    white = rng.standard_normal((h, w), dtype=np.float32)
    spec = sfft.rfft2(white, workers=-1)
    fy = np.fft.fftfreq(h).astype(np.float32)[:, None]
    fx = np.fft.rfftfreq(w).astype(np.float32)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    gain = np.zeros_like(f)
    nz = (f > 0) & (f <= cutoff)
    gain[nz] = f[nz] ** (-slope)
    spec *= gain
    out = sfft.irfft2(spec, s=(h, w), workers=-1).astype(np.float32)
    out -= out.mean()
    sd = float(out.std())
    if sd > 0:
        out *= std / sd
    out += mean
    return out


def disc_params(n: int, size: int, seed: int) -> list[dict]:
    """Parameters of n textured discs on a size x size equirectangular frame.
    Radii scale with the frame (64..512 px at 8192)."""
    rng = np.random.default_rng(seed)
    s = size / 8192.0
    discs = []
    for _ in range(n):
        discs.append(dict(
            cx=float(rng.uniform(0, size)), cy=float(rng.uniform(0, size)),
            r=float(rng.uniform(64, 512) * s),
            theta=float(rng.uniform(0, 2 * math.pi)),
            k=float(rng.uniform(1 / 64, 1 / 12)),
            phi=float(rng.uniform(0, math.pi)),
            psi=float(rng.uniform(0, 2 * math.pi)),
            amp=float(rng.uniform(20, 60)),
            y=float(rng.uniform(40, 215)),
            cb=float(rng.uniform(64, 192)),
            cr=float(rng.uniform(64, 192)),
        ))
    return discs


def _paint_disc(img: np.ndarray, cx: float, cy: float, r: float, value_fn) -> None:
    h, w = img.shape
    y0 = max(0, int(math.floor(cy - r)))
    y1 = min(h, int(math.ceil(cy + r)) + 1)
    if y1 <= y0:
        return
    x0 = int(math.floor(cx - r))
    x1 = int(math.ceil(cx + r)) + 1
    ys = np.arange(y0, y1, dtype=np.float32)[:, None]
    xs = np.arange(x0, x1, dtype=np.float32)[None, :]
    dx = xs - np.float32(cx)
    dy = ys - np.float32(cy)
    inside = (dx * dx + dy * dy) <= np.float32(r * r)
    vals = value_fn(dx, dy)
    cols = np.arange(x0, x1) % w          # longitude wraps around the seam
    sub = img[y0:y1][:, cols]
    sub[inside] = np.broadcast_to(vals, inside.shape)[inside]
    img[y0:y1, cols] = sub


def equirect_gop(size: int = 8192, n_frames: int = 8, seed: int = 2,
                 n_discs: int = 50, speed: float = 2.0, chroma: bool = True):
    """A group of frames of an equirectangular 360-degree video.

    Returns a list of n_frames tuples (Y, Cb, Cr) of uint8 arrays (Cb/Cr at
    half resolution, 4:2:0), or (Y,) when chroma is False.  The background is
    static band-limited noise; the discs move `speed` px/frame in random
    directions, wrapping in longitude."""
    h = w = int(size)
    ybg = bandlimited_noise(h, w, seed * 1000 + 1, 128.0, 40.0)
    if chroma:
        cbg = bandlimited_noise(h // 2, w // 2, seed * 1000 + 2, 128.0, 14.0)
        crg = bandlimited_noise(h // 2, w // 2, seed * 1000 + 3, 128.0, 14.0)
    discs = disc_params(n_discs, size, seed * 1000 + 4)
    frames = []
    for t in range(n_frames):
        Y = ybg.copy()
        if chroma:
            Cb = cbg.copy()
            Cr = crg.copy()
        for d in discs:
            cx = (d["cx"] + t * speed * math.cos(d["theta"])) % w
            cy = d["cy"] + t * speed * math.sin(d["theta"])
            kx = np.float32(2 * math.pi * d["k"] * math.cos(d["phi"]))
            ky = np.float32(2 * math.pi * d["k"] * math.sin(d["phi"]))

            def yfn(dx, dy, d=d, kx=kx, ky=ky):
                return np.float32(d["y"]) + np.float32(d["amp"]) * np.sin(kx * dx + ky * dy + np.float32(d["psi"]))

            _paint_disc(Y, cx, cy, d["r"], yfn)
            if chroma:
                _paint_disc(Cb, cx / 2, cy / 2, d["r"] / 2, lambda dx, dy, d=d: np.float32(d["cb"]))
                _paint_disc(Cr, cx / 2, cy / 2, d["r"] / 2, lambda dx, dy, d=d: np.float32(d["cr"]))
        planes = [Y] + ([Cb, Cr] if chroma else [])
        frames.append(tuple(np.clip(np.rint(p), 0, 255).astype(np.uint8) for p in planes))
    return frames


def random_poses(n: int = 64, seed: int = 3, pitch_max: float = math.pi / 4):
    """n head poses (yaw, pitch) in radians: yaw uniform in [-pi, pi), pitch
    uniform in [-pitch_max, pitch_max]."""
    rng = np.random.default_rng(seed)
    yaw = rng.uniform(-math.pi, math.pi, n)
    pitch = rng.uniform(-pitch_max, pitch_max, n)
    return [(float(a), float(b)) for a, b in zip(yaw, pitch)]


def random_cell_mask(rows: int, cols: int, seed: int, density: float = 0.3) -> np.ndarray:
    """A random binary reconstruction mask (uint8 0/1) made of a few random
    rectangles, for testing dependency computations on arbitrary shapes."""
    rng = np.random.default_rng(seed)
    m = np.zeros((rows, cols), np.uint8)
    target = density * rows * cols
    while m.sum() < target:
        r0 = int(rng.integers(0, rows)); c0 = int(rng.integers(0, cols))
        rh = int(rng.integers(1, max(2, rows // 3))); cw = int(rng.integers(1, max(2, cols // 3)))
        m[r0:r0 + rh, c0:c0 + cw] = 1
    return m
