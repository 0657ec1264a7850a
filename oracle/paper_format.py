"""Paper-faithful stream format -- TEST INFRASTRUCTURE (CPU oracle).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may use this module; the CUDA library never calls it.

The paper's own coding of the wavelet coefficients, written step by step:

* samples normalised to [0, 1] (x = (Y - 128) / 255 around zero), CDF 9/7
  frame-wise transform (Sec. 3.1);
* thresholding twice (Sec. 3.3): after the frame-wise transform with
  T = alpha ((l_max - l) / l_max)^2 + H (Eq. 3), and after the inter-frame
  transform (Sec. 3.2, run to the last level) with the same form, the
  inter-frame constant and the temporal level; H(y) = 1 - sin(pi y / S_y)
  (Sec. 3.6) with y the row inside the subband and S_y its height, added on
  the detail bands only (the approximation band takes l = l_max, so its
  threshold is 0; the temporal low band likewise); a coefficient survives
  when |W| > T;
* quantisation to one byte (Sec. 3.3): c_d = round((c - c_min) / (c_max -
  c_min) * 255) with the extremes of the surviving coefficients, separately
  for the approximation band and for all detail bands, per coefficient frame
  and plane; dropped coefficients are absent and decode as 0;
* file format (Sec. 3.4): header, per-frame offsets, then per coefficient
  frame a metadata package (record count, extremes), the BlockEnd package
  (one end pointer per block of 32 x 32 coefficients) and the records (block
  after block, blocks level-wise from the lowest frequency; one record = the
  coefficient's index inside its block and its byte).

Record: uint32 = index (y * 32 + x, bits 0-15) | byte << 16.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass

import numpy as np

from . import (WAVELET_97, block_list, fwd2d, haar_forward, haar_inverse, haar_needed_slots, haar_slots,
               inv2d, plane_dims, subbands, Params)

MAGIC = b"WVP1"
HEADER_FMT = "<4s" + "I" * 10 + "ff"      # 52 bytes, padded to 128
HEADER_SIZE = 128
BLOCK = 32


@dataclass
class PaperParams:
    width: int
    height: int
    planes: int = 1
    chroma_420: int = 0
    levels: int = 4
    num_frames: int = 4
    tlevels: int = 2            # inter-frame sets of 2^tlevels frames, to the last level
    alpha: float = 0.1          # frame-wise threshold constant (Eq. 3)
    alpha_t: float = 0.005      # inter-frame threshold constant

    def codec(self) -> Params:
        """The geometry as a Params of the main codec (9/7, 32 x 32 blocks)."""
        return Params(self.width, self.height, self.planes, self.chroma_420, self.levels, WAVELET_97,
                      self.num_frames, self.tlevels, BLOCK, 1.0)


def mapping_factor(rows: int) -> np.ndarray:
    """H(y) = 1 - sin(pi y / S_y) for the rows of a subband of S_y rows."""
    return 1.0 - np.sin(math.pi * np.arange(rows) / rows)


def threshold_map(w: int, h: int, levels: int, alpha: float) -> np.ndarray:
    """Per-coefficient threshold of a Mallat plane (Eq. 3): a detail band of
    level l takes alpha ((l_max - l) / l_max)^2 + H(y), y its row inside the
    subband; the approximation band (l = l_max) takes the level term alone,
    i.e. 0.  H (Sec. 3.6) thins the detail that the equirectangular mapping
    oversamples toward the poles; applied to the approximation band it
    would remove the image itself there."""
    T = np.zeros((h, w))
    for (name, lev, x0, y0, sw, sh) in subbands(w, h, levels):
        l = levels if name == "LL" else lev
        t = alpha * ((levels - l) / levels) ** 2
        T[y0:y0 + sh, x0:x0 + sw] = t if name == "LL" else t + mapping_factor(sh)[:, None]
    return T


def temporal_threshold_map(w: int, h: int, levels: int, alpha_t: float, j: int, k: int) -> np.ndarray:
    """Inter-frame threshold of a coefficient frame of temporal level j (0 =
    the low band, treated as level k): alpha_t ((k - j) / k)^2, plus H(y) on
    the spatial detail bands of the temporal detail frames (j >= 1)."""
    jj = k if j == 0 else j
    T = np.zeros((h, w))
    for (name, lev, x0, y0, sw, sh) in subbands(w, h, levels):
        t = alpha_t * ((k - jj) / k) ** 2
        T[y0:y0 + sh, x0:x0 + sw] = t if (name == "LL" or j == 0) else t + mapping_factor(sh)[:, None]
    return T


def approx_mask(w: int, h: int, levels: int) -> np.ndarray:
    m = np.zeros((h, w), bool)
    m[:h >> levels, :w >> levels] = True
    return m


def quantize_bytes(c: np.ndarray, keep: np.ndarray, approx: np.ndarray):
    """Byte codes of the surviving coefficients and the (c_min, c_max) of the
    approximation and the detail class."""
    codes = np.zeros(c.shape, np.int64)
    ext = []
    for cls in (approx, ~approx):
        sel = keep & cls
        if not np.any(sel):
            ext.append((0.0, 0.0))
            continue
        lo, hi = float(c[sel].min()), float(c[sel].max())
        if hi > lo:
            codes[sel] = np.floor((c[sel] - lo) / (hi - lo) * 255.0 + 0.5).astype(np.int64)
        ext.append((lo, hi))
    return codes, ext


def dequantize_bytes(codes: np.ndarray, present: np.ndarray, approx: np.ndarray, ext) -> np.ndarray:
    out = np.zeros(codes.shape)
    for cls, (lo, hi) in zip((approx, ~approx), ext):
        sel = present & cls
        out[sel] = lo + codes[sel] / 255.0 * (hi - lo)
    return out


def encode(frames, pp: PaperParams) -> bytes:
    """frames: num_frames tuples of uint8 planes."""
    p = pp.codec()
    k = pp.tlevels
    n = 1 << k
    if pp.num_frames % n:
        raise ValueError("num_frames must be a multiple of the set size")
    blocks = block_list(p)
    nbpf = len(blocks)
    slots = haar_slots(k)
    packages = []
    for s in range(pp.num_frames // n):
        per_plane = []
        for pl in range(pp.planes):
            w, h = plane_dims(p, pl)
            T = threshold_map(w, h, pp.levels, pp.alpha)
            coefs = []
            for j in range(n):
                x = (np.asarray(frames[s * n + j][pl], np.float64) - 128.0) / 255.0
                c = fwd2d(x, pp.levels, WAVELET_97)
                coefs.append(np.where(np.abs(c) > T, c, 0.0))
            bands = haar_forward(coefs, k, False) if k else coefs
            out = []
            for (j, _i), c in zip(slots, bands):
                Tt = temporal_threshold_map(w, h, pp.levels, pp.alpha_t, j, k) if k else np.zeros_like(c)
                keep = (np.abs(c) > Tt) & (c != 0.0)
                out.append(quantize_bytes(np.where(keep, c, 0.0), keep, approx_mask(w, h, pp.levels)) + (keep,))
            per_plane.append(out)
        for t in range(n):
            ext, ends, recs = [], [], []
            for pl in range(pp.planes):
                ext.extend(per_plane[pl][t][1])
            count = 0
            for (pl, name, lev, x0, y0, bw, bh) in blocks:
                codes, _, keep = per_plane[pl][t]
                kb = keep[y0:y0 + bh, x0:x0 + bw]
                yy, xx = np.nonzero(kb)
                vals = codes[y0:y0 + bh, x0:x0 + bw][yy, xx]
                recs.append(((yy * BLOCK + xx) | (vals << 16)).astype(np.uint32))
                count += len(yy)
                ends.append(count)
            meta = struct.pack("<II", count, 0) + np.asarray(ext, np.float32).ravel().tobytes()
            body = meta + np.asarray(ends, np.uint32).tobytes() + (np.concatenate(recs).tobytes() if recs else b"")
            body += b"\0" * ((-len(body)) % 16)
            packages.append(body)
    table_off = HEADER_SIZE
    offs, o = [], table_off + 8 * pp.num_frames
    o = (o + 15) // 16 * 16
    for b in packages:
        offs.append(o)
        o += len(b)
    hdr = struct.pack(HEADER_FMT, MAGIC, 1, pp.width, pp.height, pp.planes, pp.chroma_420, pp.levels,
                      pp.num_frames, pp.tlevels, BLOCK, nbpf, pp.alpha, pp.alpha_t)
    out = bytearray(o)
    out[:len(hdr)] = hdr
    out[table_off:table_off + 8 * pp.num_frames] = np.asarray(offs, np.uint64).tobytes()
    for off, b in zip(offs, packages):
        out[off:off + len(b)] = b
    return bytes(out)


class PaperStream:
    def __init__(self, data: bytes):
        f = struct.unpack_from(HEADER_FMT, data, 0)
        magic, version, w, h, planes, c420, levels, nf, tl, blk, nbpf, alpha, alpha_t = f
        if magic != MAGIC or version != 1 or blk != BLOCK:
            raise ValueError("not a paper-format stream")
        self.pp = PaperParams(w, h, planes, c420, levels, nf, tl, alpha, alpha_t)
        self.p = self.pp.codec()
        self.blocks = block_list(self.p)
        if nbpf != len(self.blocks):
            raise ValueError("block count mismatch")
        self.data = data
        self.offs = np.frombuffer(data, np.uint64, nf, HEADER_SIZE)

    def frame_package(self, t: int):
        """(extremes per plane and class, BlockEnd pointers, records) of coefficient frame t."""
        o = int(self.offs[t])
        count, _ = struct.unpack_from("<II", self.data, o)
        ne = 2 * 2 * self.pp.planes
        ext = np.frombuffer(self.data, np.float32, ne, o + 8).reshape(self.pp.planes, 2, 2).astype(np.float64)
        o2 = o + 8 + 4 * ne
        ends = np.frombuffer(self.data, np.uint32, len(self.blocks), o2)
        recs = np.frombuffer(self.data, np.uint32, count, o2 + 4 * len(self.blocks))
        return ext, ends, recs

    def coef_plane(self, t: int, plane: int) -> np.ndarray:
        """Dequantised Mallat plane of coefficient frame t (absent -> 0)."""
        w, h = plane_dims(self.p, plane)
        ext, ends, recs = self.frame_package(t)
        codes = np.zeros((h, w), np.int64)
        present = np.zeros((h, w), bool)
        start = 0
        for b, (pl, name, lev, x0, y0, bw, bh) in enumerate(self.blocks):
            end = int(ends[b])
            if pl == plane and end > start:
                r = recs[start:end]
                idx, val = r & 0xFFFF, r >> 16
                yy, xx = idx // BLOCK, idx % BLOCK
                codes[y0 + yy, x0 + xx] = val
                present[y0 + yy, x0 + xx] = True
            start = end
        return dequantize_bytes(codes, present, approx_mask(w, h, self.pp.levels),
                                [tuple(ext[plane, 0]), tuple(ext[plane, 1])])

    def decode_plane(self, frame: int, plane: int):
        """(x, u8): samples in 8-bit units before rounding (DC included) and the
        8-bit result clip(floor(x + 1/2))."""
        k, n = self.pp.tlevels, 1 << self.pp.tlevels
        s, fl = divmod(frame, n)
        bands = [self.coef_plane(s * n + slot, plane) for (slot, j, bit) in haar_needed_slots(k, fl)]
        c = haar_inverse(bands, k, fl, False) if k else bands[0]
        x = inv2d(c, self.pp.levels, WAVELET_97) * 255.0 + 128.0
        return x, np.clip(np.floor(x + 0.5), 0, 255).astype(np.uint8)
