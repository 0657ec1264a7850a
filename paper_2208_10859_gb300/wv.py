"""Thin Python binding of the C ABI in include/wv.h (ctypes).

Argument marshalling only: every step of the decode runs in libwv.so's CUDA
kernels.  PyTorch supplies device memory (tensors) and CUDA streams.  There
is no CPU fallback: importing this module on a machine without the built
library raises, and calls without a CUDA device return WV_ERR_CUDA.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

WV_OK = 0
WV_OPEN_HOST_PAYLOAD = 1
ERRORS = {-1: "WV_ERR_ARG", -2: "WV_ERR_FORMAT", -3: "WV_ERR_OOM", -4: "WV_ERR_CUDA",
          -5: "WV_ERR_RANGE", -6: "WV_ERR_TIMEOUT", -7: "WV_ERR_DEVICE"}
WAVELET_53 = 0
WAVELET_97 = 1


class WVError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({_lib().wv_strerror(code).decode()})")


class StreamDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("planes", ctypes.c_int),
                ("chroma_420", ctypes.c_int), ("levels", ctypes.c_int), ("wavelet", ctypes.c_int),
                ("num_frames", ctypes.c_int), ("tlevels", ctypes.c_int), ("block", ctypes.c_int),
                ("quant", ctypes.c_int), ("step", ctypes.c_float), ("stereo", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Image(ctypes.Structure):
    _fields_ = [("dptr", ctypes.c_void_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("pitch_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("s", ctypes.c_void_p), ("frame", ctypes.c_int), ("yaw", ctypes.c_float),
                ("pitch", ctypes.c_float), ("fov", ctypes.c_float), ("out", Image),
                ("fovea", ctypes.c_int), ("gaze_x", ctypes.c_float), ("gaze_y", ctypes.c_float),
                ("r1", ctypes.c_float), ("r2", ctypes.c_float), ("eye", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int), ("surfaces", ctypes.c_int), ("coarse_tiles", ctypes.c_int),
                ("fine_tiles", ctypes.c_int), ("bytes", ctypes.c_size_t), ("ms", ctypes.c_double * 4),
                ("waves", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_batch", ctypes.c_int), ("cache_bytes", ctypes.c_size_t),
                ("arena_bytes", ctypes.c_size_t), ("reserve_bytes", ctypes.c_size_t)]


class ServerRequest(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int), ("frame", ctypes.c_int), ("yaw", ctypes.c_float),
                ("pitch", ctypes.c_float), ("fov", ctypes.c_float), ("out", Image),
                ("fovea", ctypes.c_int), ("gaze_x", ctypes.c_float), ("gaze_y", ctypes.c_float),
                ("r1", ctypes.c_float), ("r2", ctypes.c_float), ("eye", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_ulonglong) for n in
                ("submitted", "completed", "failed", "batches", "batched_requests", "uploads", "evictions",
                 "max_batch_bytes", "resident_bytes", "arena_bytes")]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int * 8), ("tiles", ctypes.c_int)]


KERNEL_NAMES = ["footprint", "select_tiles", "decode_coarse", "decode_fine", "resample"]

_LIB = None


def lib_path() -> str:
    """The library the binding loads: libwv.so, the WV_CHECKED build when the
    environment variable WV_CHECKED is 1, or the host-sanitizer build when
    WV_SANITIZE is 1."""
    if os.environ.get("WV_CHECKED") == "1":
        return _build.LIB_CHECKED
    if os.environ.get("WV_SANITIZE") == "1":
        return _build.LIB_SAN
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"{os.path.basename(path)} is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        c_int, c_size, vp, fl = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_float
        sig = {
            "wv_strerror": (ctypes.c_char_p, [c_int]),
            "wv_stream_query": (c_int, [vp, c_size, ctypes.POINTER(StreamDesc), ctypes.POINTER(c_size)]),
            "wv_open_stream": (c_int, [vp, c_size, vp, c_size, vp, ctypes.POINTER(vp)]),
            "wv_stream_query_ex": (c_int, [vp, c_size, c_int, ctypes.POINTER(StreamDesc), ctypes.POINTER(c_size)]),
            "wv_open_stream_ex": (c_int, [vp, c_size, vp, c_size, vp, c_int, ctypes.POINTER(vp)]),
            "wv_set_cuda_stream": (c_int, [vp, vp]),
            "wv_close_stream": (None, [vp]),
            "wv_decode_viewport": (c_int, [vp, c_int, fl, fl, fl, ctypes.POINTER(Image)]),
            "wv_decode_viewport_eye": (c_int, [vp, c_int, c_int, fl, fl, fl, ctypes.POINTER(Image)]),
            "wv_decode_batch": (c_int, [ctypes.POINTER(Request), c_int, vp]),
            "wv_decode_full": (c_int, [vp, c_int, c_int, vp, c_int]),
            "wv_stream_sync_status": (c_int, [vp]),
            "wv_debug_footprint": (c_int, [vp, fl, fl, fl, c_int, c_int, vp, ctypes.POINTER(c_int)]),
            "wv_debug_project": (c_int, [vp, fl, fl, fl, c_int, c_int, vp]),
            "wv_resample_at": (c_int, [vp, vp, ctypes.POINTER(Image)]),
            "wv_cone_bytes": (c_int, [vp, c_int, vp, ctypes.POINTER(ctypes.c_ulonglong)]),
            "wv_profile_begin": (c_int, [vp]),
            "wv_profile_end": (c_int, [vp, ctypes.POINTER(Profile)]),
            "wv_launches_per_viewport": (c_int, [vp]),
            "wv_set_decode_mode": (c_int, [vp, c_int]),
            "wv_encode_sizes": (c_int, [ctypes.POINTER(StreamDesc), ctypes.POINTER(c_size), ctypes.POINTER(c_size)]),
            "wv_encode": (c_int, [ctypes.POINTER(StreamDesc), vp, vp, c_size, vp, c_size,
                                  ctypes.POINTER(c_size), vp]),
            "wv_decode_plane_static": (c_int, [ctypes.POINTER(StreamDesc), vp, c_size, vp, c_int, c_int, vp,
                                               c_int, vp, ctypes.POINTER(c_int)]),
            "wv_release_default_batch": (None, []),
            "wv_encode_paper": (c_int, [ctypes.POINTER(StreamDesc), vp, vp, c_size, fl, fl, vp, c_size,
                                        ctypes.POINTER(c_size), vp]),
            "wv_cnn_param_count": (c_size, []),
            "wv_cnn_create": (c_int, [vp, ctypes.POINTER(vp)]),
            "wv_cnn_close": (None, [vp]),
            "wv_cnn_get_params": (c_int, [vp, vp]),
            "wv_cnn_set_params": (c_int, [vp, vp]),
            "wv_cnn_get_state": (c_int, [vp, vp, vp, ctypes.POINTER(c_int)]),
            "wv_cnn_set_state": (c_int, [vp, vp, vp, c_int]),
            "wv_cnn_forward": (c_int, [vp, vp, vp, c_int, c_int, c_int, vp]),
            "wv_cnn_gradients": (c_int, [vp, vp, vp, c_int, c_int, c_int, vp, ctypes.POINTER(fl), vp]),
            "wv_cnn_train_step": (c_int, [vp, vp, vp, c_int, c_int, c_int, fl, ctypes.POINTER(fl), vp]),
            "wv_cnn_sync_status": (c_int, [vp]),
            "wv_decode_viewport_filtered": (c_int, [vp, c_int, fl, fl, fl, vp, ctypes.POINTER(Image)]),
            "wv_server_create": (c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
            "wv_server_add_stream": (c_int, [vp, vp, c_size, ctypes.POINTER(c_int)]),
            "wv_server_submit": (c_int, [vp, ctypes.POINTER(ServerRequest), ctypes.POINTER(ctypes.c_uint64)]),
            "wv_server_poll": (c_int, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
            "wv_server_wait": (c_int, [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
            "wv_server_drain": (c_int, [vp, ctypes.c_double]),
            "wv_server_get_stats": (c_int, [vp, ctypes.POINTER(ServerStats)]),
            "wv_server_latencies": (c_int, [vp, ctypes.POINTER(ctypes.c_double), c_int, ctypes.POINTER(c_int)]),
            "wv_server_reset_stats": (c_int, [vp]),
            "wv_server_close": (None, [vp]),
            "wv_cone_bytes_fovea": (c_int, [vp, c_int, vp, vp, ctypes.POINTER(ctypes.c_ulonglong)]),
            "wv_cone_bytes_split": (c_int, [vp, c_int, vp, ctypes.POINTER(ctypes.c_ulonglong),
                                            ctypes.POINTER(ctypes.c_ulonglong)]),
            "wv_request_bytes": (c_int, [ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_ulonglong),
                                         ctypes.POINTER(ctypes.c_ulonglong)]),
            "wv_batch_create": (c_int, [vp, ctypes.POINTER(vp)]),
            "wv_batch_close": (None, [vp]),
            "wv_batch_decode": (c_int, [vp, ctypes.POINTER(Request), c_int]),
            "wv_batch_set_cuda_stream": (c_int, [vp, vp]),
            "wv_batch_device_bytes": (c_int, [vp, ctypes.POINTER(Request), c_int, ctypes.POINTER(c_size)]),
            "wv_batch_sync_status": (c_int, [vp]),
            "wv_batch_stats": (c_int, [vp, ctypes.POINTER(BatchInfo)]),
            "wv_batch_set_timing": (c_int, [vp, c_int]),
            "wv_batch_set_sharing": (c_int, [vp, c_int]),
            "wv_batch_set_wait_limit": (c_int, [vp, c_int]),
            "wv_batch_set_strips": (c_int, [vp, c_int]),
            "wv_debug_fail_device_allocs": (None, [c_int]),
            "wv_batch_set_tile_shape": (c_int, [vp, c_int, c_int, c_int, c_int, c_int, c_int, c_int]),
            "wv_batch_tile_shape": (c_int, [vp, c_int, c_int, c_int, c_int, ctypes.POINTER(c_int),
                                            ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
            "wv_batch_completion_ms": (c_int, [vp, ctypes.POINTER(ctypes.c_double), c_int]),
            "wv_batch_set_memory_limit": (c_int, [vp, c_size]),
            "wv_batch_autotune": (c_int, [vp, ctypes.POINTER(Request), c_int, c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols() -> list[str]:
    """Names of the ABI functions the binding resolves (all of include/wv.h)."""
    _lib()
    return ["wv_strerror", "wv_stream_query", "wv_open_stream", "wv_stream_query_ex", "wv_open_stream_ex",
            "wv_set_cuda_stream",
            "wv_close_stream", "wv_decode_viewport", "wv_decode_viewport_eye", "wv_decode_batch",
            "wv_decode_full",
            "wv_stream_sync_status", "wv_debug_footprint", "wv_debug_project", "wv_resample_at",
            "wv_cone_bytes", "wv_profile_begin", "wv_profile_end", "wv_launches_per_viewport",
            "wv_set_decode_mode",
            "wv_encode_sizes", "wv_encode", "wv_decode_plane_static", "wv_release_default_batch",
            "wv_cone_bytes_fovea", "wv_cone_bytes_split", "wv_request_bytes", "wv_encode_paper",
            "wv_cnn_param_count", "wv_cnn_create", "wv_cnn_close", "wv_cnn_get_params", "wv_cnn_set_params",
            "wv_cnn_get_state", "wv_cnn_set_state",
            "wv_cnn_forward", "wv_cnn_gradients", "wv_cnn_train_step", "wv_cnn_sync_status",
            "wv_decode_viewport_filtered",
            "wv_server_create", "wv_server_add_stream", "wv_server_submit", "wv_server_poll",
            "wv_server_wait", "wv_server_drain", "wv_server_get_stats", "wv_server_latencies",
            "wv_server_reset_stats", "wv_server_close",
            "wv_batch_create", "wv_batch_close", "wv_batch_decode", "wv_batch_set_cuda_stream",
            "wv_batch_device_bytes", "wv_batch_sync_status", "wv_batch_stats", "wv_batch_set_timing",
            "wv_batch_set_sharing", "wv_batch_set_wait_limit", "wv_debug_fail_device_allocs",
            "wv_batch_set_tile_shape", "wv_batch_tile_shape", "wv_batch_autotune", "wv_batch_completion_ms",
            "wv_batch_set_memory_limit", "wv_batch_set_strips"]


def _check(rc: int, what: str):
    if rc != WV_OK:
        raise WVError(rc, what)


def _cuda_stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _image(t) -> Image:
    import torch
    if not (t.is_cuda and t.dtype == torch.uint8 and t.dim() == 3 and t.shape[2] == 4):
        raise ValueError("output must be a CUDA uint8 tensor of shape (H, W, 4)")
    if t.stride(2) != 1 or t.stride(1) != 4:
        raise ValueError("output rows must be packed RGBA")
    return Image(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0))


def query(data: bytes, flags: int = 0) -> tuple[dict, int]:
    d = StreamDesc()
    need = ctypes.c_size_t()
    buf = ctypes.c_char_p(data)
    _check(_lib().wv_stream_query_ex(buf, len(data), flags, ctypes.byref(d), ctypes.byref(need)),
           "wv_stream_query_ex")
    return d.as_dict(), need.value


class Stream:
    """An open wavelet video stream resident on the GPU."""

    def __init__(self, data: bytes, cuda_stream=None, host_payload: bool = False):
        """host_payload: keep the coefficient store in pinned, device-mapped
        host memory (WV_OPEN_HOST_PAYLOAD) instead of device memory."""
        import torch
        flags = WV_OPEN_HOST_PAYLOAD if host_payload else 0
        self.desc, need = query(data, flags)
        # device store supplied by PyTorch's allocator (256-byte aligned)
        self._mem = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        base = self._mem.data_ptr()
        aligned = (base + 255) & ~255
        self._handle = ctypes.c_void_p()
        self._cuda_stream = cuda_stream
        _check(_lib().wv_open_stream_ex(ctypes.c_char_p(data), len(data), ctypes.c_void_p(aligned), need,
                                        ctypes.c_void_p(_cuda_stream_handle(cuda_stream)), flags,
                                        ctypes.byref(self._handle)), "wv_open_stream_ex")
        self.device_bytes = need

    @property
    def handle(self) -> int:
        return self._handle.value

    def set_cuda_stream(self, stream) -> None:
        self._cuda_stream = stream
        _check(_lib().wv_set_cuda_stream(self._handle, ctypes.c_void_p(_cuda_stream_handle(stream))),
               "wv_set_cuda_stream")

    def decode_viewport(self, frame: int, yaw: float, pitch: float, fov: float, out, eye: int = 0) -> None:
        img = _image(out)
        if eye == 0:
            _check(_lib().wv_decode_viewport(self._handle, frame, yaw, pitch, fov, ctypes.byref(img)),
                   "wv_decode_viewport")
        else:
            _check(_lib().wv_decode_viewport_eye(self._handle, frame, eye, yaw, pitch, fov, ctypes.byref(img)),
                   "wv_decode_viewport_eye")

    def decode_full(self, frame: int, plane: int, out=None, as_float: bool = False) -> None:
        ptr = None if out is None else ctypes.c_void_p(out.data_ptr())
        _check(_lib().wv_decode_full(self._handle, frame, plane, ptr, int(as_float)), "wv_decode_full")

    def sync_status(self) -> int:
        return _lib().wv_stream_sync_status(self._handle)

    def debug_footprint(self, yaw, pitch, fov, out_w, out_h):
        d = self.desc
        mask = np.zeros((d["height"] // 32, d["width"] // 32), np.uint8)
        tiles = ctypes.c_int()
        _check(_lib().wv_debug_footprint(self._handle, yaw, pitch, fov, out_w, out_h,
                                         mask.ctypes.data_as(ctypes.c_void_p), ctypes.byref(tiles)),
               "wv_debug_footprint")
        return mask, tiles.value

    def debug_project(self, yaw, pitch, fov, out_w, out_h):
        import torch
        uv = torch.empty((out_h, out_w, 2), dtype=torch.float32, device="cuda")
        _check(_lib().wv_debug_project(self._handle, yaw, pitch, fov, out_w, out_h,
                                       ctypes.c_void_p(uv.data_ptr())), "wv_debug_project")
        return uv

    def resample_at(self, uv, out) -> None:
        img = _image(out)
        if not (uv.is_cuda and uv.is_contiguous() and tuple(uv.shape) == (out.shape[0], out.shape[1], 2)
                and str(uv.dtype) == "torch.float32"):
            raise ValueError("uv must be a contiguous CUDA float32 tensor of shape (H, W, 2)")
        _check(_lib().wv_resample_at(self._handle, ctypes.c_void_p(uv.data_ptr()), ctypes.byref(img)),
               "wv_resample_at")

    def cone_bytes_split(self, frame: int, mask: np.ndarray) -> tuple[int, int]:
        """Coefficient cone bytes read by the fine pass (levels 1-2) and by the
        coarse pass (levels 3 and above)."""
        m = np.ascontiguousarray(mask, np.uint8)
        fine, coarse = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        _check(_lib().wv_cone_bytes_split(self._handle, frame, m.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(fine), ctypes.byref(coarse)), "wv_cone_bytes_split")
        return int(fine.value), int(coarse.value)

    def cone_bytes(self, frame: int, mask: np.ndarray, fovea: np.ndarray | None = None) -> int:
        m = np.ascontiguousarray(mask, np.uint8)
        out = ctypes.c_ulonglong()
        if fovea is None:
            _check(_lib().wv_cone_bytes(self._handle, frame, m.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(out)), "wv_cone_bytes")
        else:
            f = np.ascontiguousarray(fovea, np.uint8)
            _check(_lib().wv_cone_bytes_fovea(self._handle, frame, m.ctypes.data_as(ctypes.c_void_p),
                                              f.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)),
                   "wv_cone_bytes_fovea")
        return out.value

    def decode_viewport_filtered(self, frame: int, yaw: float, pitch: float, fov: float, cnn, out) -> None:
        img = _image(out)
        _check(_lib().wv_decode_viewport_filtered(self._handle, frame, yaw, pitch, fov, cnn.handle,
                                                  ctypes.byref(img)), "wv_decode_viewport_filtered")

    def set_decode_mode(self, mode: int) -> None:
        _check(_lib().wv_set_decode_mode(self._handle, mode), "wv_set_decode_mode")

    def launches_per_viewport(self) -> int:
        return _lib().wv_launches_per_viewport(self._handle)

    def profile_begin(self) -> None:
        _check(_lib().wv_profile_begin(self._handle), "wv_profile_begin")

    def profile_end(self) -> dict:
        p = Profile()
        _check(_lib().wv_profile_end(self._handle, ctypes.byref(p)), "wv_profile_end")
        out = {n: (p.ms[i], p.launches[i]) for i, n in enumerate(KERNEL_NAMES)}
        out["tiles"] = p.tiles
        return out

    def close(self) -> None:
        if self._handle.value:
            _lib().wv_close_stream(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class ViewRequest:
    stream: Stream
    frame: int
    yaw: float
    pitch: float
    fov: float
    out: object
    fovea: bool = False
    gaze_x: float = 0.0
    gaze_y: float = 0.0
    r1: float = float("inf")
    r2: float = float("inf")
    eye: int = 0


def _requests(requests: list):
    arr = (Request * len(requests))()
    for i, r in enumerate(requests):
        arr[i] = Request(r.stream.handle, r.frame, r.yaw, r.pitch, r.fov, _image(r.out),
                         1 if r.fovea else 0, r.gaze_x, r.gaze_y, r.r1, r.r2, r.eye)
    return arr


def request_bytes(request) -> tuple:
    """(coefficient cone bytes, decoded region bytes) of one request."""
    arr = _requests([request])
    cone, region = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    _check(_lib().wv_request_bytes(arr, ctypes.byref(cone), ctypes.byref(region)), "wv_request_bytes")
    return cone.value, region.value


def decode_batch(requests: list, cuda_stream=None) -> None:
    arr = _requests(requests)
    _check(_lib().wv_decode_batch(arr, len(requests), ctypes.c_void_p(_cuda_stream_handle(cuda_stream))),
           "wv_decode_batch")


class Batch:
    """A batch context (wv_batch_*): batched, graph-launched decoding of many
    viewport requests with an autotuned tile shape per stream class."""

    def __init__(self, cuda_stream=None):
        h = ctypes.c_void_p()
        _check(_lib().wv_batch_create(ctypes.c_void_p(_cuda_stream_handle(cuda_stream)), ctypes.byref(h)),
               "wv_batch_create")
        self._h = h

    def decode(self, requests: list) -> None:
        arr = _requests(requests)
        _check(_lib().wv_batch_decode(self._h, arr, len(requests)), "wv_batch_decode")

    def set_cuda_stream(self, stream) -> None:
        _check(_lib().wv_batch_set_cuda_stream(self._h, ctypes.c_void_p(_cuda_stream_handle(stream))),
               "wv_batch_set_cuda_stream")

    def device_bytes(self, requests: list) -> int:
        n = ctypes.c_size_t()
        _check(_lib().wv_batch_device_bytes(self._h, _requests(requests), len(requests), ctypes.byref(n)),
               "wv_batch_device_bytes")
        return n.value

    def sync_status(self) -> int:
        return _lib().wv_batch_sync_status(self._h)

    def stats(self) -> dict:
        info = BatchInfo()
        _check(_lib().wv_batch_stats(self._h, ctypes.byref(info)), "wv_batch_stats")
        return {"requests": info.requests, "surfaces": info.surfaces, "coarse_tiles": info.coarse_tiles,
                "fine_tiles": info.fine_tiles, "bytes": info.bytes, "waves": info.waves,
                "ms": dict(zip(["footprint", "select", "decode", "resample"], list(info.ms)))}

    def completion_ms(self, n: int) -> np.ndarray:
        """With timing on: completion time of each request of the last batch
        (ms from the batch's start; caller order)."""
        out = np.zeros(n, np.float64)
        _check(_lib().wv_batch_completion_ms(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n),
               "wv_batch_completion_ms")
        return out

    def set_memory_limit(self, nbytes: int) -> None:
        """Device bytes of decode targets per wave (0: one wave)."""
        _check(_lib().wv_batch_set_memory_limit(self._h, int(nbytes)), "wv_batch_set_memory_limit")

    def set_timing(self, on: bool) -> None:
        _check(_lib().wv_batch_set_timing(self._h, 1 if on else 0), "wv_batch_set_timing")

    def set_strips(self, on: bool) -> None:
        """Strip fine pass for the targets it takes (default), or square tiles for all."""
        _check(_lib().wv_batch_set_strips(self._h, 1 if on else 0), "wv_batch_set_strips")

    def set_sharing(self, on: bool) -> None:
        _check(_lib().wv_batch_set_sharing(self._h, 1 if on else 0), "wv_batch_set_sharing")

    def set_wait_limit(self, polls: int) -> None:
        """Polls of the tile decode's bounded wait before it gives up."""
        _check(_lib().wv_batch_set_wait_limit(self._h, int(polls)), "wv_batch_set_wait_limit")

    def set_tile_shape(self, wavelet, levels, width, height, tile_w, tile_h, ctile) -> None:
        _check(_lib().wv_batch_set_tile_shape(self._h, wavelet, levels, width, height, tile_w, tile_h, ctile),
               "wv_batch_set_tile_shape")

    def tile_shape(self, wavelet, levels, width, height) -> tuple:
        """(output tile width, output tile height, coarse tile side)."""
        tw, th, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().wv_batch_tile_shape(self._h, wavelet, levels, width, height, ctypes.byref(tw),
                                          ctypes.byref(th), ctypes.byref(c)), "wv_batch_tile_shape")
        return tw.value, th.value, c.value

    def autotune(self, requests: list, reps: int = 3) -> None:
        _check(_lib().wv_batch_autotune(self._h, _requests(requests), len(requests), reps), "wv_batch_autotune")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib().wv_batch_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode_paper(frames, desc: dict, alpha: float, alpha_t: float, cuda_stream=None) -> bytes:
    """Encode frames (as for encode) into the paper-faithful format on the GPU."""
    d = dict(desc, quant=1, wavelet=WAVELET_97, block=32, step=1.0)
    return _encode(frames, d, cuda_stream, lambda L, sd, arr, base, scratch, out, cap, n, cs:
                   L.wv_encode_paper(sd, arr, base, scratch, alpha, alpha_t, out, cap, n, cs), "wv_encode_paper")


def encode(frames, desc: dict, cuda_stream=None) -> bytes:
    return _encode(frames, desc, cuda_stream, lambda L, sd, arr, base, scratch, out, cap, n, cs:
                   L.wv_encode(sd, arr, base, scratch, out, cap, n, cs), "wv_encode")


def _encode(frames, desc: dict, cuda_stream, call, what) -> bytes:
    """Encode frames (list of num_frames tuples of CUDA uint8 plane tensors) on
    the GPU into stream bytes."""
    import torch
    d = StreamDesc(**{k: desc.get(k, 0) for k, _ in StreamDesc._fields_})
    scratch = ctypes.c_size_t()
    cap = ctypes.c_size_t()
    _check(_lib().wv_encode_sizes(ctypes.byref(d), ctypes.byref(scratch), ctypes.byref(cap)), "wv_encode_sizes")
    mem = torch.empty(scratch.value + 256, dtype=torch.uint8, device="cuda")
    base = (mem.data_ptr() + 255) & ~255
    ptrs = []
    keep = []
    for fr in frames:
        for p in fr:
            t = p.contiguous()
            keep.append(t)
            ptrs.append(t.data_ptr())
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    out = np.empty(cap.value, np.uint8)
    n = ctypes.c_size_t()
    torch.cuda.current_stream().synchronize()
    _check(call(_lib(), ctypes.byref(d), arr, ctypes.c_void_p(base), scratch.value,
                out.ctypes.data_as(ctypes.c_void_p), cap.value, ctypes.byref(n),
                ctypes.c_void_p(_cuda_stream_handle(cuda_stream))), what)
    del mem, keep
    return out[:n.value].tobytes()


class Server:
    """Request loop with continuous batching (wv_server_*): register coded
    streams, submit viewport requests from any thread, poll or wait."""

    def __init__(self, slots: int = 2, max_batch: int = 64, cache_bytes: int = 0, arena_bytes: int = 0,
                 reserve_bytes: int = 1 << 30):
        h = ctypes.c_void_p()
        cfg = ServerConfig(slots, max_batch, cache_bytes, arena_bytes, reserve_bytes)
        _check(_lib().wv_server_create(ctypes.byref(cfg), ctypes.byref(h)), "wv_server_create")
        self._h = h
        self._keep = {}

    def add_stream(self, data: bytes) -> int:
        sid = ctypes.c_int()
        _check(_lib().wv_server_add_stream(self._h, ctypes.c_char_p(data), len(data), ctypes.byref(sid)),
               "wv_server_add_stream")
        return sid.value

    def submit(self, stream_id: int, frame: int, yaw: float, pitch: float, fov: float, out,
               fovea: bool = False, gaze_x: float = 0.0, gaze_y: float = 0.0,
               r1: float = float("inf"), r2: float = float("inf"), eye: int = 0) -> int:
        r = ServerRequest(stream_id, frame, yaw, pitch, fov, _image(out), 1 if fovea else 0,
                          gaze_x, gaze_y, r1, r2, eye)
        t = ctypes.c_uint64()
        _check(_lib().wv_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "wv_server_submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending; the latency in ms once done (raises on failure)."""
        lat = ctypes.c_double()
        rc = _lib().wv_server_poll(self._h, ticket, ctypes.byref(lat))
        if rc == 1:
            return None
        _check(rc, "wv_server_poll")
        return lat.value

    def wait(self, ticket: int, timeout_ms: float = 10000.0) -> float:
        lat = ctypes.c_double()
        _check(_lib().wv_server_wait(self._h, ticket, timeout_ms, ctypes.byref(lat)), "wv_server_wait")
        return lat.value

    def drain(self, timeout_ms: float = 60000.0) -> None:
        _check(_lib().wv_server_drain(self._h, timeout_ms), "wv_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib().wv_server_get_stats(self._h, ctypes.byref(st)), "wv_server_get_stats")
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def latencies(self) -> np.ndarray:
        n = ctypes.c_int()
        _check(_lib().wv_server_latencies(self._h, None, 0, ctypes.byref(n)), "wv_server_latencies")
        buf = (ctypes.c_double * max(1, n.value))()
        _check(_lib().wv_server_latencies(self._h, buf, n.value, ctypes.byref(n)), "wv_server_latencies")
        return np.array(buf[:n.value])

    def reset_stats(self) -> None:
        _check(_lib().wv_server_reset_stats(self._h), "wv_server_reset_stats")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib().wv_server_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned post-filter
# ---------------------------------------------------------------------------

CNN_SHAPES = [(32, 1), (32, 32), (32, 32), (32, 32), (1, 32)]   # (c_out, c_in) per layer


def cnn_init_params(seed: int = 0) -> np.ndarray:
    """Flat parameters: He-normal weights (the last layer scaled by 0.1, so the
    untrained network is close to the identity), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (co, ci) in enumerate(CNN_SHAPES):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if k == len(CNN_SHAPES) - 1 else 1.0)
        parts.append((rng.standard_normal((co, ci, 3, 3)) * std).ravel())
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def _fptr(t) -> ctypes.c_void_p:
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return ctypes.c_void_p(t.data_ptr())


class CNN:
    """The residual post-filter network (wv_cnn_*): forward, gradients and
    Adam training steps on the library's tensor-core kernels."""

    def __init__(self, params=None, seed: int = 0):
        p = cnn_init_params(seed) if params is None else np.ascontiguousarray(params, np.float32)
        if p.size != self.param_count():
            raise ValueError("wrong parameter count")
        h = ctypes.c_void_p()
        _check(_lib().wv_cnn_create(p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)), "wv_cnn_create")
        self.handle = h

    @staticmethod
    def param_count() -> int:
        return int(_lib().wv_cnn_param_count())

    def params(self) -> np.ndarray:
        out = np.empty(self.param_count(), np.float32)
        _check(_lib().wv_cnn_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "wv_cnn_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, np.float32)
        _check(_lib().wv_cnn_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)), "wv_cnn_set_params")

    def state(self) -> tuple[np.ndarray, np.ndarray, int]:
        """Adam moments (m, v) and the number of steps taken."""
        m = np.empty(self.param_count(), np.float32)
        v = np.empty(self.param_count(), np.float32)
        k = ctypes.c_int()
        _check(_lib().wv_cnn_get_state(self.handle, m.ctypes.data_as(ctypes.c_void_p),
                                       v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)), "wv_cnn_get_state")
        return m, v, int(k.value)

    def set_state(self, m, v, steps: int) -> None:
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        _check(_lib().wv_cnn_set_state(self.handle, m.ctypes.data_as(ctypes.c_void_p),
                                       v.ctypes.data_as(ctypes.c_void_p), int(steps)), "wv_cnn_set_state")

    def forward(self, x, stream=None):
        import torch
        n, h, w = x.shape
        y = torch.empty_like(x)
        _check(_lib().wv_cnn_forward(self.handle, _fptr(x), _fptr(y), n, h, w,
                                     ctypes.c_void_p(_cuda_stream_handle(stream))), "wv_cnn_forward")
        return y

    def gradients(self, x, t, stream=None):
        n, h, w = x.shape
        g = np.empty(self.param_count(), np.float32)
        loss = ctypes.c_float()
        _check(_lib().wv_cnn_gradients(self.handle, _fptr(x), _fptr(t), n, h, w, g.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(loss), ctypes.c_void_p(_cuda_stream_handle(stream))),
               "wv_cnn_gradients")
        return float(loss.value), g

    def train_step(self, x, t, lr: float, want_loss: bool = False, stream=None):
        n, h, w = x.shape
        loss = ctypes.c_float()
        _check(_lib().wv_cnn_train_step(self.handle, _fptr(x), _fptr(t), n, h, w, lr,
                                        ctypes.byref(loss) if want_loss else None,
                                        ctypes.c_void_p(_cuda_stream_handle(stream))), "wv_cnn_train_step")
        return float(loss.value) if want_loss else None

    def sync_status(self) -> int:
        return _lib().wv_cnn_sync_status(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None) and self.handle.value:
            _lib().wv_cnn_close(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
