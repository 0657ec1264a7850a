"""CPU oracle of the wavelet 360-degree video codec -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA decoder never calls it, and it shares no
code with the CUDA library: the lifting loops live in ``wv_oracle.c`` (plain C,
fp64 / exact integers), everything else below is plain numpy written step by
step from the paper (Groth, Fricke, Castillo, Magnor: "Wavelet-Based Fast
Decoding of 360 deg Videos").

What is computed, with the passage each part follows:

* ``fwd2d`` / ``inv2d`` -- frame-wise 2D FWT / iFWT, Sec. 3.1 Eq. 1, CDF 9/7
  (Sec. 3.1) or LeGall 5/3 (Sec. 2.2), Mallat layout, level 1 finest.
* ``haar_forward`` / ``haar_inverse`` -- inter-frame Haar transform over sets
  of n = 2^k frames, to the last level, applied to the 2D coefficients (Sec.
  3.2); the inverse adds log2(n) detail coefficients with sign -1 or +1.
* ``quantize`` / ``dequantize`` -- dead-zone uniform quantiser with step D;
  the paper's own min/max byte quantiser (Sec. 3.3, "Quantization") is not
  used by this stream format.  The decoder inverts the quantisation (Sec. 3.3).
* ``encode`` / ``Stream`` -- block-structured stream: header (Sec. 3.4: frame
  count, frame size, levels), per-frame block table (the BlockEnd pointers of
  Sec. 3.4 as one slot index per block, -1 for an all-zero block), payload of
  dense int16 blocks, ordered level-wise from the lowest frequency (Sec. 3.4).
* ``decode_plane`` -- rebuild of one frame: dequantise, inverse inter-frame
  Haar, 2D iFWT (Sec. 3.5), DC unshift and rounding to 8 bit.
* ``project`` -- viewport pixel -> equirectangular position (Sec. 3.6).
* ``footprint`` -- the low-resolution binary reconstruction mask (Sec. 3.1:
  256x256 cells for an 8k frame, i.e. 32-pixel cells).
* ``cone`` -- coefficients the masked iFWT needs (Sec. 3.1/3.4).
* ``fovea_distance`` / ``fovea_keep`` / ``fovea_coef_mask`` -- foveated
  decoding (Sec. 3.7): finer levels' details only near the gaze, rectilinear
  regions, dropped coefficients taken as zero.
* ``resample`` / ``ycbcr_to_rgba`` / ``viewport`` -- reprojection of the
  decoded region into the viewport (Sec. 3.6) with bilinear filtering and a
  BT.709 colour conversion (the paper itself does none, Sec. 5).

Readings of silent or ambiguous passages are listed in the repository's design
notes; the constants used here are restated from their published sources.

Parity pins: every function above is checked in ``tests/test_oracle_*.py``
against closed forms, published filter taps, brute force or textbook
identities.
"""
from __future__ import annotations

import ctypes
import math
import os
import struct
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# host-side sanitizers: with WV_ORACLE_SANITIZE=1 the oracle loads a build
# of its C core with AddressSanitizer and UndefinedBehaviorSanitizer (the
# process must preload the ASan runtime)
_SAN_PATH = os.path.join(_BUILD, "liboracle_san.so")
_lib = None

WAVELET_53 = 0
WAVELET_97 = 1


# --------------------------------------------------------------------------
# native lifting core
# --------------------------------------------------------------------------

def build_sanitized() -> str:
    """Compile wv_oracle.c with AddressSanitizer and UndefinedBehaviorSanitizer
    (single-threaded) into oracle/_build/liboracle_san.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(_SAN_PATH) or os.path.getmtime(_SAN_PATH) < os.path.getmtime(_SRC):
        tmp = _SAN_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O1", "-g", "-fPIC", "-shared", "-std=c99",
                               "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                               "-fno-omit-frame-pointer", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SAN_PATH)
    return _SAN_PATH


def build() -> str:
    """Compile wv_oracle.c with gcc into oracle/_build/liboracle.so (with
    OpenMP where the compiler has it, else single-threaded)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:5] + ["-fopenmp"] + base[5:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def set_threads(n: int) -> int:
    """Host threads the 2D transforms use (n <= 0 keeps the current count);
    returns the count in effect (1 without OpenMP)."""
    return int(_load().or_set_threads(int(n)))


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_sanitized() if os.environ.get("WV_ORACLE_SANITIZE") == "1" else build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        L = ctypes.c_long
        for name, p in (("or_fwd97_1d", dp), ("or_inv97_1d", dp),
                        ("or_fwd53_1d", ip), ("or_inv53_1d", ip)):
            f = getattr(lib, name)
            f.argtypes = [p, p, L]
            f.restype = None
        for name, p in (("or_fwd2d_97", dp), ("or_inv2d_97", dp),
                        ("or_fwd2d_53", ip), ("or_inv2d_53", ip)):
            f = getattr(lib, name)
            f.argtypes = [p, L, L, ctypes.c_int]
            f.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def fwd1d(x, wavelet: int) -> np.ndarray:
    """One-level 1D analysis of an even-length line: returns [s | d]."""
    lib = _load()
    if wavelet == WAVELET_97:
        x = np.ascontiguousarray(x, np.float64)
        out = np.empty_like(x)
        lib.or_fwd97_1d(_ptr(x, ctypes.c_double), _ptr(out, ctypes.c_double), x.size)
    else:
        x = np.ascontiguousarray(x, np.int64)
        out = np.empty_like(x)
        lib.or_fwd53_1d(_ptr(x, ctypes.c_int64), _ptr(out, ctypes.c_int64), x.size)
    return out


def inv1d(c, wavelet: int) -> np.ndarray:
    """One-level 1D synthesis of [s | d] back to samples."""
    lib = _load()
    if wavelet == WAVELET_97:
        c = np.ascontiguousarray(c, np.float64)
        out = np.empty_like(c)
        lib.or_inv97_1d(_ptr(c, ctypes.c_double), _ptr(out, ctypes.c_double), c.size)
    else:
        c = np.ascontiguousarray(c, np.int64)
        out = np.empty_like(c)
        lib.or_inv53_1d(_ptr(c, ctypes.c_int64), _ptr(out, ctypes.c_int64), c.size)
    return out


def fwd2d(img, levels: int, wavelet: int) -> np.ndarray:
    """Frame-wise 2D FWT (Sec. 3.1, Eq. 1) into the Mallat layout."""
    lib = _load()
    h, w = img.shape
    if w % (1 << levels) or h % (1 << levels):
        raise ValueError("frame sides must be divisible by 2^levels")
    if wavelet == WAVELET_97:
        a = np.array(img, np.float64, order="C")
        rc = lib.or_fwd2d_97(_ptr(a, ctypes.c_double), w, h, levels)
    else:
        a = np.array(img, np.int64, order="C")
        rc = lib.or_fwd2d_53(_ptr(a, ctypes.c_int64), w, h, levels)
    if rc:
        raise MemoryError("oracle fwd2d")
    return a


def inv2d(coef, levels: int, wavelet: int) -> np.ndarray:
    """2D iFWT of a Mallat-layout plane (Sec. 3.1 / 3.5)."""
    lib = _load()
    h, w = coef.shape
    if wavelet == WAVELET_97:
        a = np.array(coef, np.float64, order="C")
        rc = lib.or_inv2d_97(_ptr(a, ctypes.c_double), w, h, levels)
    else:
        a = np.array(coef, np.int64, order="C")
        rc = lib.or_inv2d_53(_ptr(a, ctypes.c_int64), w, h, levels)
    if rc:
        raise MemoryError("oracle inv2d")
    return a


# --------------------------------------------------------------------------
# inter-frame Haar transform (Sec. 3.2)
# --------------------------------------------------------------------------

def haar_slots(k: int) -> list[tuple[int, int]]:
    """Slot order of the 2^k coefficient frames of one inter-frame set:
    slot 0 = L_k, then H_k[0], H_(k-1)[0..1], ..., H_1[0..n/2).  Returns a list
    of (level j, index i) with j = 0 meaning the low band L_k."""
    slots = [(0, 0)]
    for j in range(k, 0, -1):
        for i in range(1 << (k - j)):
            slots.append((j, i))
    return slots


def haar_forward(frames: list, k: int, integer: bool) -> list:
    """Forward inter-frame Haar over n = 2^k coefficient frames, executed to
    the last level (Sec. 3.2).  Float: L = (a+b)/2, H = (b-a)/2.  Integer
    (S-transform, for the reversible 5/3 codec): H = b-a, L = a + floor(H/2)."""
    n = 1 << k
    assert len(frames) == n
    low = list(frames)
    highs = {}
    for j in range(1, k + 1):
        nxt = []
        hj = []
        for i in range(len(low) // 2):
            a, b = low[2 * i], low[2 * i + 1]
            if integer:
                hh = b - a
                ll = a + np.floor_divide(hh, 2)
            else:
                ll = (a + b) / 2.0
                hh = (b - a) / 2.0
            nxt.append(ll)
            hj.append(hh)
        highs[j] = hj
        low = nxt
    out = []
    for (j, i) in haar_slots(k):
        out.append(low[0] if j == 0 else highs[j][i])
    return out


def haar_needed_slots(k: int, f_local: int) -> list[tuple[int, int, int]]:
    """Coefficient frames needed to rebuild frame f_local of a set, as
    (slot, level j, bit) from the coarsest level down; bit 1 means '+H'."""
    need = [(0, 0, 0)]
    for j in range(k, 0, -1):
        i = f_local >> j
        bit = (f_local >> (j - 1)) & 1
        need.append(((1 << (k - j)) + i, j, bit))
    return need


def haar_inverse(bands: list, k: int, f_local: int, integer: bool):
    """Rebuild one frame from L_k and one detail band per level (Sec. 3.2):
    float: L + sum of +-H; integer: S-transform inverse level by level."""
    need = haar_needed_slots(k, f_local)
    v = bands[0]
    for (slot, j, bit), h in zip(need[1:], bands[1:]):
        if integer:
            a = v - np.floor_divide(h, 2)
            v = a + h if bit else a
        else:
            v = v + h if bit else v - h
    return v


# --------------------------------------------------------------------------
# dead-zone quantiser
# --------------------------------------------------------------------------

def quantize(c, step: float, integer: bool) -> np.ndarray:
    """q = sign(c) * floor(|c| / step) (fp64, or exact integers for 5/3)."""
    if integer:
        c = np.asarray(c, np.int64)
        s = int(step)
        return np.sign(c) * (np.abs(c) // s)
    c = np.asarray(c, np.float64)
    return (np.sign(c) * np.floor(np.abs(c) / step)).astype(np.int64)


def dequantize(q, step: float, integer: bool):
    """Inverse of the quantiser (Sec. 3.3: the normalisation is inverted at
    reconstruction).  Float: sign(q)(|q| + 1/2) step, 0 for q = 0.  Integer
    (5/3): sign(q)(|q| step + floor(step/2)), which is q itself at step 1."""
    q = np.asarray(q, np.int64)
    if integer:
        s = int(step)
        return np.sign(q) * (np.abs(q) * s + s // 2)
    return np.sign(q) * (np.abs(q) + 0.5) * float(step)


# --------------------------------------------------------------------------
# stream format (Sec. 3.4)
# --------------------------------------------------------------------------

MAGIC = b"WVS1"
HEADER_FMT = "<4s" + "I" * 12 + "fII" + "QQQ"   # 88 bytes, padded to 128
HEADER_SIZE = 128


@dataclass
class Params:
    width: int
    height: int
    planes: int = 1            # 1 (grey) or 3 (Y, Cb, Cr)
    chroma_420: int = 0        # 1: Cb/Cr at half width and height
    levels: int = 3
    wavelet: int = WAVELET_53
    num_frames: int = 1
    tlevels: int = 0           # inter-frame Haar levels k (set size n = 2^k)
    block: int = 256
    step: float = 1.0
    stereo: int = 0            # 1: top/bottom stereo, each eye an equirect of height / 2


def plane_dims(p: Params, plane: int) -> tuple[int, int]:
    if plane > 0 and p.chroma_420:
        return p.width // 2, p.height // 2
    return p.width, p.height


def subbands(w: int, h: int, levels: int):
    """Subbands of a Mallat plane in stream order: LL_L, then for l = L..1:
    HL_l, LH_l, HH_l.  Yields (name, level, x0, y0, sw, sh)."""
    sw, sh = w >> levels, h >> levels
    yield ("LL", levels, 0, 0, sw, sh)
    for l in range(levels, 0, -1):
        sw, sh = w >> l, h >> l
        yield ("HL", l, sw, 0, sw, sh)
        yield ("LH", l, 0, sh, sw, sh)
        yield ("HH", l, sw, sh, sw, sh)


def block_list(p: Params):
    """All blocks of one coefficient frame in stream order, as tuples
    (plane, subband name, level, x0, y0, bw, bh) in Mallat coordinates."""
    out = []
    B = p.block
    for pl in range(p.planes):
        w, h = plane_dims(p, pl)
        for (name, lev, x0, y0, sw, sh) in subbands(w, h, p.levels):
            for by in range(0, sh, B):
                for bx in range(0, sw, B):
                    out.append((pl, name, lev, x0 + bx, y0 + by,
                                min(B, sw - bx), min(B, sh - by)))
    return out


def _check_params(p: Params):
    if p.planes not in (1, 3):
        raise ValueError("planes must be 1 or 3")
    if p.wavelet not in (WAVELET_53, WAVELET_97):
        raise ValueError("wavelet")
    if p.num_frames % (1 << p.tlevels):
        raise ValueError("num_frames must be a multiple of the set size")
    for pl in range(p.planes):
        w, h = plane_dims(p, pl)
        if w % (1 << p.levels) or h % (1 << p.levels) or (w >> p.levels) < 2 or (h >> p.levels) < 2:
            raise ValueError("plane sides must be divisible by 2^levels")
    if p.wavelet == WAVELET_53 and (p.step != int(p.step) or p.step < 1):
        raise ValueError("5/3 needs an integer step >= 1")
    if p.stereo not in (0, 1) or (p.stereo and p.height % (2 * CELL)):
        raise ValueError("stereo frames need a height divisible by 64")


def encode(frames, p: Params) -> bytes:
    """Oracle encoder: per frame and plane DC shift and 2D FWT (Sec. 3.1),
    per inter-frame set the Haar transform along time (Sec. 3.2), dead-zone
    quantisation, blocking with all-zero blocks omitted (Sec. 3.4).

    frames: list of num_frames tuples of uint8 planes."""
    _check_params(p)
    integer = p.wavelet == WAVELET_53
    n = 1 << p.tlevels
    blocks = block_list(p)
    nbpf = len(blocks)
    table = np.full((p.num_frames, nbpf), -1, np.int32)
    payload = []
    B = p.block
    for s in range(p.num_frames // n):
        per_plane = []
        for pl in range(p.planes):
            coefs = []
            for j in range(n):
                x = np.asarray(frames[s * n + j][pl])
                x = x.astype(np.int64) - 128 if integer else x.astype(np.float64) - 128.0
                coefs.append(fwd2d(x, p.levels, p.wavelet))
            bands = haar_forward(coefs, p.tlevels, integer) if p.tlevels else coefs
            qs = []
            for c in bands:
                q = quantize(c, p.step, integer)
                if q.size and (q.max() > 32767 or q.min() < -32768):
                    raise OverflowError("quantised coefficient out of int16 range")
                qs.append(q.astype(np.int16))
            per_plane.append(qs)
        for j in range(n):
            t = s * n + j
            for b, (pl, name, lev, x0, y0, bw, bh) in enumerate(blocks):
                blk = per_plane[pl][j][y0:y0 + bh, x0:x0 + bw]
                if np.any(blk):
                    full = np.zeros((B, B), np.int16)
                    full[:bh, :bw] = blk
                    table[t, b] = len(payload)
                    payload.append(full)
    table_off = HEADER_SIZE
    payload_off = table_off + table.nbytes
    payload_off = (payload_off + 255) // 256 * 256
    hdr = struct.pack(HEADER_FMT, MAGIC, 1, p.width, p.height, p.planes, p.chroma_420,
                      p.levels, p.wavelet, p.num_frames, p.tlevels, p.block, 0, p.stereo,
                      float(p.step), nbpf, 0, len(payload), table_off, payload_off)
    out = bytearray(payload_off + len(payload) * B * B * 2)
    out[:len(hdr)] = hdr
    out[table_off:table_off + table.nbytes] = table.tobytes()
    if payload:
        out[payload_off:] = np.stack(payload).tobytes()
    return bytes(out)


class Stream:
    """Parsed stream (header + block table preloaded, as in Sec. 3.4)."""

    def __init__(self, data: bytes):
        if len(data) < HEADER_SIZE:
            raise ValueError("truncated header")
        f = struct.unpack_from(HEADER_FMT, data, 0)
        (magic, version, w, h, planes, c420, levels, wavelet, nf, tl, blk, quant,
         stereo, step, nbpf, _r1, npay, toff, poff) = f
        if magic != MAGIC or version != 1 or quant != 0 or stereo not in (0, 1):
            raise ValueError("bad magic/version/quantiser/stereo flag")
        self.p = Params(w, h, planes, c420, levels, wavelet, nf, tl, blk, step, stereo)
        _check_params(self.p)
        self.blocks = block_list(self.p)
        if nbpf != len(self.blocks):
            raise ValueError("block count mismatch")
        self.table = np.frombuffer(data, np.int32, nf * nbpf, toff).reshape(nf, nbpf)
        self.payload = np.frombuffer(data, np.int16, npay * blk * blk, poff).reshape(npay, blk, blk)
        if self.table.size and (self.table.max() >= npay or self.table.min() < -1):
            raise ValueError("block slot out of range")

    def coef_plane(self, t: int, plane: int) -> np.ndarray:
        """Quantised Mallat plane of coefficient frame t (zero blocks -> 0)."""
        w, h = plane_dims(self.p, plane)
        out = np.zeros((h, w), np.int64)
        for b, (pl, name, lev, x0, y0, bw, bh) in enumerate(self.blocks):
            if pl != plane:
                continue
            slot = self.table[t, b]
            if slot >= 0:
                out[y0:y0 + bh, x0:x0 + bw] = self.payload[slot, :bh, :bw]
        return out

    def present_mask(self, t: int, plane: int) -> np.ndarray:
        """Boolean Mallat-plane mask of coefficients that lie in stored blocks."""
        w, h = plane_dims(self.p, plane)
        out = np.zeros((h, w), bool)
        for b, (pl, name, lev, x0, y0, bw, bh) in enumerate(self.blocks):
            if pl == plane and self.table[t, b] >= 0:
                out[y0:y0 + bh, x0:x0 + bw] = True
        return out


def frame_slots(p: Params, frame: int) -> list[tuple[int, int]]:
    """Coefficient frames (t, bit) needed to rebuild `frame` (Sec. 3.2)."""
    n = 1 << p.tlevels
    s, fl = divmod(frame, n)
    return [(s * n + slot, bit) for (slot, j, bit) in haar_needed_slots(p.tlevels, fl)]


def decode_coefs(st: Stream, frame: int, plane: int, keep=None):
    """Dequantised, temporally rebuilt Mallat plane of one frame (Sec. 3.5).
    keep: optional foveation cell masks (see ``fovea_keep``); coefficients
    they drop are taken as zero (Sec. 3.7)."""
    p = st.p
    integer = p.wavelet == WAVELET_53
    n = 1 << p.tlevels
    bands = [dequantize(st.coef_plane(t, plane), p.step, integer)
             for (t, bit) in frame_slots(p, frame)]
    if keep is not None:
        m = fovea_coef_mask(p, plane, keep)
        bands = [b * m for b in bands]
    if p.tlevels == 0:
        return bands[0]
    return haar_inverse(bands, p.tlevels, frame % n, integer)


def decode_plane(st: Stream, frame: int, plane: int, keep=None):
    """Full-frame reconstruction of one plane.  Returns (x, u8): x are the
    samples in 8-bit units before rounding (float64 for 9/7, int64 for 5/3,
    DC unshifted) and u8 the 8-bit result: clip(floor(x + 1/2)) for 9/7,
    clip(x) for 5/3.  keep: optional foveation cell masks."""
    p = st.p
    c = decode_coefs(st, frame, plane, keep)
    x = inv2d(c, p.levels, p.wavelet) + 128
    if p.wavelet == WAVELET_97:
        u8 = np.clip(np.floor(x + 0.5), 0, 255).astype(np.uint8)
    else:
        u8 = np.clip(x, 0, 255).astype(np.uint8)
    return x, u8


# --------------------------------------------------------------------------
# projection, footprint, dependency cone (Sec. 3.1, 3.6)
# --------------------------------------------------------------------------

def rotation(yaw: float, pitch: float) -> np.ndarray:
    """World-from-camera rotation R_y(yaw) R_x(pitch): positive pitch looks
    up (+y), positive yaw turns from +z toward +x."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    rx = np.array([[1, 0, 0], [0, cp, sp], [0, -sp, cp]])
    return ry @ rx


def project(out_w: int, out_h: int, yaw: float, pitch: float, fov: float,
            eq_w: int, eq_h: int, row0: int = 0):
    """Equirectangular position (u, v), in pixels of an eq_w x eq_h frame with
    pixel centres at integers, seen by each viewport pixel (fp64).  The
    viewport is a pinhole camera with the same full field of view `fov` on
    both axes; pixel (i, j) looks through its centre (i + 1/2, j + 1/2).
    row0 places the equirect at rows row0 .. row0 + eq_h - 1 of a larger
    frame (an eye of a top/bottom stereo frame)."""
    t = math.tan(fov / 2)
    xn = (2 * (np.arange(out_w) + 0.5) / out_w - 1) * t
    yn = (1 - 2 * (np.arange(out_h) + 0.5) / out_h) * t
    X, Yn = np.meshgrid(xn, yn)
    cam = np.stack([X, Yn, np.ones_like(X)], axis=-1)
    d = cam @ rotation(yaw, pitch).T
    lon = np.arctan2(d[..., 0], d[..., 2])
    lat = np.arctan2(d[..., 1], np.hypot(d[..., 0], d[..., 2]))
    u = (lon / (2 * math.pi) + 0.5) * eq_w - 0.5
    v = (0.5 - lat / math.pi) * eq_h - 0.5 + row0
    return u, v


def eye_rows(p: Params, eye: int = 0) -> tuple[int, int]:
    """(first row, rows) of the luma equirect an eye sees: the whole frame for
    mono streams; the top (eye 0) or bottom (eye 1) half for stereo ones."""
    if not p.stereo:
        if eye != 0:
            raise ValueError("mono streams have one eye")
        return 0, p.height
    if eye not in (0, 1):
        raise ValueError("eye must be 0 or 1")
    return eye * p.height // 2, p.height // 2


def _fixed(t):
    """Split a coordinate into integer part and a fraction in 1/256 steps
    (round half up), carrying into the integer part at 256."""
    i = np.floor(t).astype(np.int64)
    f = np.floor((t - i) * 256 + 0.5).astype(np.int64)
    carry = f >= 256
    i = i + carry
    f = np.where(carry, 0, f)
    return i, f


def taps(u, v, w: int, h: int, rows=None):
    """Integer positions of the 2x2 bilinear taps (x wraps, y clamps to the
    rows (first, count) of the image, default all)."""
    lo, n = (0, h) if rows is None else rows
    x0, fx = _fixed(np.asarray(u))
    y0, fy = _fixed(np.asarray(v))
    xa = np.mod(x0, w)
    xb = np.mod(x0 + 1, w)
    ya = np.clip(y0, lo, lo + n - 1)
    yb = np.clip(y0 + 1, lo, lo + n - 1)
    return xa, xb, ya, yb, fx, fy


def bilinear(img: np.ndarray, u, v, rows=None) -> np.ndarray:
    """Fixed-point bilinear sample: weights in 1/256 steps that sum to 65536,
    result (sum + 32768) >> 16; rows limits the clamp (stereo eyes)."""
    h, w = img.shape
    xa, xb, ya, yb, fx, fy = taps(u, v, w, h, rows)
    P = img.astype(np.int64)
    acc = ((256 - fx) * (256 - fy) * P[ya, xa] + fx * (256 - fy) * P[ya, xb]
           + (256 - fx) * fy * P[yb, xa] + fx * fy * P[yb, xb])
    return ((acc + 32768) >> 16).astype(np.uint8)


def chroma_coords(u, v):
    """Centre-sited 4:2:0: chroma sample c covers luma samples 2c, 2c+1."""
    return (np.asarray(u) + 0.5) / 2 - 0.5, (np.asarray(v) + 0.5) / 2 - 0.5


CELL = 32  # luma pixels per mask cell: 256x256 cells for 8192x8192 (Sec. 3.1)


def footprint(p: Params, out_w: int, out_h: int, yaw: float, pitch: float,
              fov: float, cell: int = CELL, eye: int = 0):
    """Low-resolution binary mask of the frame region the viewport reads
    (Sec. 3.1): cell (r, c) is set when a bilinear tap of some viewport pixel,
    of luma or (mapped to luma) of chroma, falls in it.  Returns (core,
    dilated): core from the fp64 positions, dilated = core grown by one cell
    in each direction (x wraps, y clamps)."""
    W, H = p.width, p.height
    rows, cols = H // cell, W // cell
    r0, nr = eye_rows(p, eye)
    u, v = project(out_w, out_h, yaw, pitch, fov, W, nr, r0)
    core = np.zeros((rows, cols), bool)
    xa, xb, ya, yb, _, _ = taps(u, v, W, H, (r0, nr))
    for xx in (xa, xb):
        for yy in (ya, yb):
            core[yy // cell, xx // cell] = True
    if p.planes == 3 and p.chroma_420:
        uc, vc = chroma_coords(u, v)
        cw, chh = W // 2, H // 2
        xa, xb, ya, yb, _, _ = taps(uc, vc, cw, chh, (r0 // 2, nr // 2))
        half = cell // 2
        for xx in (xa, xb):
            for yy in (ya, yb):
                core[yy // half, xx // half] = True
    dil = core.copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            sh = np.roll(core, dx, axis=1)
            if dy == -1:
                sh = np.vstack([sh[1:], np.zeros((1, cols), bool)])
            elif dy == 1:
                sh = np.vstack([np.zeros((1, cols), bool), sh[:-1]])
            dil |= sh
    return core, dil


def synthesis_support(wavelet: int, parity: int) -> tuple[int, int]:
    """Interleaved input offsets [lo, hi] that synthesis output i reads,
    for i of the given parity.  9/7: the four lifting steps reach 3 samples
    to each side of an even output and 4 of an odd one; 5/3: 1 and 2."""
    if wavelet == WAVELET_97:
        return (-3, 3) if parity == 0 else (-4, 4)
    return (-1, 1) if parity == 0 else (-2, 2)


def _reflect_idx(i, n):
    i = np.asarray(i)
    period = 2 * (n - 1)
    i = np.mod(i, period)
    return np.where(i >= n, period - i, i)


def _dilate_axis(m: np.ndarray, wavelet: int, axis: int) -> np.ndarray:
    """Positions along `axis` read by the 1D synthesis of the set positions,
    reflected into range."""
    n = m.shape[axis]
    out = np.zeros_like(m)
    idx = np.arange(n)
    for parity in (0, 1):
        lo, hi = synthesis_support(wavelet, parity)
        src = idx[idx % 2 == parity]
        sel = np.take(m, src, axis=axis)
        for off in range(lo, hi + 1):
            dst = _reflect_idx(src + off, n)
            if axis == 0:
                np.logical_or.at(out, (dst[:, None], np.arange(m.shape[1])[None, :]), sel)
            else:
                np.logical_or.at(out, (np.arange(m.shape[0])[:, None], dst[None, :]), sel)
    return out


def cone(pix_mask: np.ndarray, levels: int, wavelet: int) -> dict:
    """Dependency cone of the masked iFWT (Sec. 3.1): for each level l and
    subband, the boolean mask of coefficients needed to reconstruct the
    pixels set in `pix_mask` (full plane resolution).  Returns
    {(name, l): mask over that subband}, names LL (level L only), HL, LH, HH."""
    need = {}
    R = pix_mask.astype(bool)
    for l in range(1, levels + 1):
        X = _dilate_axis(_dilate_axis(R, wavelet, 1), wavelet, 0)
        need[("HL", l)] = X[0::2, 1::2]
        need[("LH", l)] = X[1::2, 0::2]
        need[("HH", l)] = X[1::2, 1::2]
        R = X[0::2, 0::2]
    need[("LL", levels)] = R
    return need


def cell_mask_to_pixels(mask: np.ndarray, w: int, h: int) -> np.ndarray:
    """Expand a cell mask to a pixel mask of a w x h plane."""
    ry, rx = h // mask.shape[0], w // mask.shape[1]
    return np.repeat(np.repeat(mask.astype(bool), ry, axis=0), rx, axis=1)


def cone_bytes(st: Stream, frame: int, mask: np.ndarray, keep=None) -> int:
    """Coefficient bytes the viewport needs: the cone of the mask in every
    plane, restricted to stored (non-zero) blocks, 2 bytes per coefficient,
    summed over the coefficient frames the inter-frame rebuild reads.  With
    foveation cell masks `keep`, coefficients they drop are not read."""
    p = st.p
    total = 0
    for pl in range(p.planes):
        w, h = plane_dims(p, pl)
        need = cone(cell_mask_to_pixels(mask, w, h), p.levels, p.wavelet)
        full = np.zeros((h, w), bool)
        for (name, lev, x0, y0, sw, sh) in subbands(w, h, p.levels):
            full[y0:y0 + sh, x0:x0 + sw] = need[(name, lev)]
        if keep is not None:
            full &= fovea_coef_mask(p, pl, keep)
        for (t, _bit) in frame_slots(p, frame):
            total += 2 * int(np.count_nonzero(full & st.present_mask(t, pl)))
    return total


# --------------------------------------------------------------------------
# foveated decoding (Sec. 3.7)
# --------------------------------------------------------------------------
#
# The full viewport is reconstructed from the coarse levels; each finer level
# adds its details only over a smaller, rectilinear region around the gaze,
# and the inverse transform treats the dropped details as zero.  The regions
# are unions of mask cells: a cell keeps the details of level l when its
# centre lies within r_l of the gaze, the distance being the larger of the
# horizontal and vertical angle differences seen from the viewer (squares in
# angle, i.e. rectilinear regions).  Level 1 (finest) uses r1, level 2 uses
# r2; coarser levels are always complete.  A detail coefficient belongs to the
# cell of its nominal position: coefficient (kx, ky) of a level-l subband of a
# plane subsampled by s sits at luma pixel (s kx 2^l, s ky 2^l).


def fovea_distance(p: Params, yaw: float, pitch: float, gaze_x: float, gaze_y: float,
                   cell: int = CELL, eye: int = 0) -> np.ndarray:
    """Per mask cell (rows x cols), the angular distance (radians) of the
    cell centre from the gaze direction: max(|theta_x - gaze_x|,
    |theta_y - gaze_y|), theta_x = atan2(x, z) and theta_y = atan2(y, z) in
    viewer coordinates (x right, y up, z forward; gaze angles relative to the
    view centre).  Cells behind the viewer (z <= 0) are infinitely far."""
    W, H = p.width, p.height
    rows, cols = H // cell, W // cell
    r0, nr = eye_rows(p, eye)              # cells of the other eye are infinitely far
    lon = 2 * math.pi * ((np.arange(cols) + 0.5) * cell / W - 0.5)
    lat = math.pi * (0.5 - ((np.arange(rows) + 0.5) * cell - r0) / nr)
    LON, LAT = np.meshgrid(lon, lat)
    d = np.stack([np.cos(LAT) * np.sin(LON), np.sin(LAT), np.cos(LAT) * np.cos(LON)], axis=-1)
    cam = d @ rotation(yaw, pitch)          # rows of R^T d: world -> viewer
    tx = np.arctan2(cam[..., 0], cam[..., 2])
    ty = np.arctan2(cam[..., 1], cam[..., 2])
    dist = np.maximum(np.abs(tx - gaze_x), np.abs(ty - gaze_y))
    inside = ((np.arange(rows) * cell >= r0) & (np.arange(rows) * cell < r0 + nr))[:, None]
    return np.where((cam[..., 2] > 0) & inside, dist, np.inf)


def fovea_keep(p: Params, yaw: float, pitch: float, gaze_x: float, gaze_y: float,
               r1: float, r2: float, eye: int = 0) -> dict:
    """Cell masks of the detail levels foveation keeps: {1: dist <= r1,
    2: dist <= r2}; other levels are complete."""
    d = fovea_distance(p, yaw, pitch, gaze_x, gaze_y, eye=eye)
    return {1: d <= r1, 2: d <= r2}


def fovea_coef_mask(p: Params, plane: int, keep: dict) -> np.ndarray:
    """Boolean Mallat-plane mask of the coefficients foveation keeps."""
    w, h = plane_dims(p, plane)
    s = 2 if (plane > 0 and p.chroma_420) else 1
    out = np.ones((h, w), bool)
    for (name, lev, x0, y0, sw, sh) in subbands(w, h, p.levels):
        if name == "LL" or lev not in keep:
            continue
        cx = (np.arange(sw) * s << lev) // CELL
        cy = (np.arange(sh) * s << lev) // CELL
        out[y0:y0 + sh, x0:x0 + sw] = keep[lev][np.ix_(cy, cx)]
    return out


def fovea_margin(p: Params, yaw: float, pitch: float, gaze_x: float, gaze_y: float,
                 r1: float, r2: float) -> float:
    """Smallest |distance - radius| over all cells (radians): how far the
    keep decisions are from a tie."""
    d = fovea_distance(p, yaw, pitch, gaze_x, gaze_y)
    d = d[np.isfinite(d)]
    return float(min(np.abs(d - r1).min(), np.abs(d - r2).min())) if d.size else math.inf


# --------------------------------------------------------------------------
# resampling and colour (Sec. 3.6; colour conversion per BT.709)
# --------------------------------------------------------------------------

KR, KB = 0.2126, 0.0722  # ITU-R BT.709 luma weights


def colour_coefficients():
    """Integer (x 2^16) BT.709 full-range YCbCr -> RGB coefficients:
    R = Y + 2(1-Kr) Cr', G = Y - 2Kb(1-Kb)/Kg Cb' - 2Kr(1-Kr)/Kg Cr',
    B = Y + 2(1-Kb) Cb'."""
    kg = 1 - KR - KB
    return dict(rcr=round(2 * (1 - KR) * 65536), gcb=round(2 * KB * (1 - KB) / kg * 65536),
                gcr=round(2 * KR * (1 - KR) / kg * 65536), bcb=round(2 * (1 - KB) * 65536))


def ycbcr_to_rgba(Y, Cb, Cr) -> np.ndarray:
    c = colour_coefficients()
    y = np.asarray(Y, np.int64) * 65536 + 32768
    cb = np.asarray(Cb, np.int64) - 128
    cr = np.asarray(Cr, np.int64) - 128
    r = np.clip((y + c["rcr"] * cr) >> 16, 0, 255)
    g = np.clip((y - c["gcb"] * cb - c["gcr"] * cr) >> 16, 0, 255)
    b = np.clip((y + c["bcb"] * cb) >> 16, 0, 255)
    a = np.full_like(r, 255)
    return np.stack([r, g, b, a], axis=-1).astype(np.uint8)


def resample(planes, p: Params, u, v, eye: int = 0) -> np.ndarray:
    """Viewport RGBA from decoded 8-bit planes at luma positions (u, v);
    rows clamp to the eye's part of the frame."""
    r0, nr = eye_rows(p, eye)
    Y = bilinear(planes[0], u, v, (r0, nr))
    if p.planes == 1:
        return ycbcr_to_rgba(Y, np.full_like(Y, 128), np.full_like(Y, 128))
    if p.chroma_420:
        uc, vc = chroma_coords(u, v)
        crows = (r0 // 2, nr // 2)
    else:
        uc, vc = u, v
        crows = (r0, nr)
    return ycbcr_to_rgba(Y, bilinear(planes[1], uc, vc, crows), bilinear(planes[2], uc, vc, crows))


def viewport(st: Stream, frame: int, yaw: float, pitch: float, fov: float,
             out_w: int, out_h: int, planes=None, fovea=None, eye: int = 0) -> np.ndarray:
    """Reference viewport decode by the plain definition: reconstruct the
    whole frame, then reproject it into the viewport.  fovea = (gaze_x,
    gaze_y, r1, r2) decodes with foveation (Sec. 3.7); eye selects the half of
    a top/bottom stereo frame.  Returns RGBA uint8 (out_h, out_w, 4)."""
    p = st.p
    if planes is None:
        keep = None if fovea is None else fovea_keep(p, yaw, pitch, *fovea)
        planes = [decode_plane(st, frame, pl, keep)[1] for pl in range(p.planes)]
    r0, nr = eye_rows(p, eye)
    u, v = project(out_w, out_h, yaw, pitch, fov, p.width, nr, r0)
    return resample(planes, p, u, v, eye)


def viewport_candidates(planes, p: Params, u, v, eps: float):
    """All RGBA values a viewport pixel may take when its position is known
    only to within +-eps pixels: each of the luma and chroma coordinates can
    fall into at most two 1/256 quantisation cells, so up to 16 candidates
    per pixel.  Returns an array (..., 16, 4)."""
    if p.planes == 3 and p.chroma_420:
        uc, vc = chroma_coords(u, v)
    else:
        uc, vc = u, v
    outs = []
    for su in (-eps, eps):
        for sv in (-eps, eps):
            Y = bilinear(planes[0], u + su, v + sv)
            for scu in (-eps, eps):
                for scv in (-eps, eps):
                    if p.planes == 1:
                        outs.append(ycbcr_to_rgba(Y, np.full_like(Y, 128), np.full_like(Y, 128)))
                    else:
                        Cb = bilinear(planes[1], uc + scu, vc + scv)
                        Cr = bilinear(planes[2], uc + scu, vc + scv)
                        outs.append(ycbcr_to_rgba(Y, Cb, Cr))
    return np.stack(outs, axis=-2)
