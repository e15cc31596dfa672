"""Thin ctypes binding of the C ABI in include/isx.h (argument marshalling only).

Every step of encode and decode runs in the CUDA library
``libisx_gb300.so``; this module converts torch tensors / numpy arrays into
pointers and maps status codes to exceptions.  There is no CPU fallback:
loading fails loudly when the library is missing or CUDA is unavailable.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libisx_gb300.so")

ISX_OK, ISX_ERR_ARG, ISX_ERR_CAPACITY, ISX_ERR_CORRUPT, ISX_ERR_OOM, ISX_ERR_CUDA, ISX_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "ISX_OK", 1: "ISX_ERR_ARG", 2: "ISX_ERR_CAPACITY", 3: "ISX_ERR_CORRUPT", 4: "ISX_ERR_OOM",
                5: "ISX_ERR_CUDA", 6: "ISX_ERR_TIMEOUT", 7: "ISX_ERR_INTERNAL"}

# every entry point declared in include/isx.h
EXPORTS = ["isx_create", "isx_destroy", "isx_encode_tiles", "isx_decode_region", "isx_encode_tiles_host",
           "isx_decode_region_host", "isx_forward_coefficients", "isx_sync_status", "isx_last_launch_count",
           "isx_last_error", "isx_set_timing", "isx_stage_times", "isx_encode_tile_static", "isx_decode_jobs",
           "isx_get_schedule", "isx_set_schedule", "isx_autotune", "isx_plan_encode", "isx_plan_decode",
           "isx_plan_launch_encode", "isx_plan_launch_decode", "isx_plan_sync_status", "isx_plan_device_bytes",
           "isx_plan_launch_count", "isx_plan_last_error", "isx_plan_destroy", "isx_decode_jobs_scratch",
           "isx_reserve_scratch", "isx_scratch_bytes", "isx_decode_path", "isx_set_tile_stamps", "isx_copy_rects"]

SIZE_CLASSES = 5

# colour transform selectors (isx_tile_desc.transform, ISX_CT_*)
CT_DEFAULT, CT_NONE, CT_RCT, CT_YCOCG_R = 0, 1, 2, 3

# size of the library's static device scratch (ISX_STATIC_SCRATCH_BYTES)
STATIC_SCRATCH_BYTES = 16 << 20


class IsxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class TileDescC(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("bits", ctypes.c_int32), ("levels", ctypes.c_int32), ("x0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("qstep_log2", ctypes.c_uint8 * 16), ("pixels", ctypes.c_void_p), ("row_pitch_bytes", ctypes.c_int64),
                ("transform", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class DecodeJobC(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("rx", ctypes.c_int32), ("ry", ctypes.c_int32), ("rw", ctypes.c_int32),
                ("rh", ctypes.c_int32), ("d_out", ctypes.c_void_p), ("out_pitch_bytes", ctypes.c_int64)]


# numpy layout of isx_decode_job (for building many jobs without Python loops)
JOB_DTYPE = np.dtype([("tile", "<i4"), ("rx", "<i4"), ("ry", "<i4"), ("rw", "<i4"), ("rh", "<i4"), ("_pad", "<i4"),
                      ("d_out", "<u8"), ("out_pitch_bytes", "<i8")])


# numpy layout of isx_rect_copy
COPY_DTYPE = np.dtype([("src", "<u8"), ("src_pitch", "<i8"), ("dst", "<u8"), ("dst_pitch", "<i8"), ("row_bytes", "<i4"),
                       ("rows", "<i4")])


class ScheduleC(ctypes.Structure):
    _fields_ = [("forward_threads", ctypes.c_int32 * 5), ("inverse_threads", ctypes.c_int32 * 5)]


@dataclass
class Tile:
    """One tile: geometry, coding parameters and where its pixels live."""
    width: int
    height: int
    channels: int
    bits: int
    levels: int
    qstep_log2: Sequence[int] = ()
    x0: int = 0
    y0: int = 0
    pixels: int = 0            # device (or, for the *_host calls, host) address
    row_pitch_bytes: int = 0
    keep: object = field(default=None, repr=False)   # keeps the pixel buffer alive
    transform: int = CT_DEFAULT

    def to_c(self) -> TileDescC:
        t = TileDescC()
        t.width, t.height, t.channels, t.bits, t.levels = self.width, self.height, self.channels, self.bits, self.levels
        t.x0, t.y0 = self.x0, self.y0
        q = list(self.qstep_log2) + [0] * (16 - len(self.qstep_log2))
        for i in range(16):
            t.qstep_log2[i] = q[i]
        t.pixels = self.pixels
        t.row_pitch_bytes = self.row_pitch_bytes
        t.transform = self.transform
        return t


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libisx_gb300.so (building it in-tree with nvcc when absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH) and build_if_missing:
            from . import _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        st = ctypes.c_int
        lib.isx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, sz]
        lib.isx_create.restype = st
        lib.isx_destroy.argtypes = [vp]
        lib.isx_destroy.restype = None
        lib.isx_encode_tiles.argtypes = [vp, vp, i32, vp, sz, vp, vp]
        lib.isx_encode_tiles.restype = st
        lib.isx_decode_region.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, i64, vp]
        lib.isx_decode_region.restype = st
        lib.isx_encode_tiles_host.argtypes = [vp, vp, i32, vp, sz, vp, vp]
        lib.isx_encode_tiles_host.restype = st
        lib.isx_decode_region_host.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, i64, vp]
        lib.isx_decode_region_host.restype = st
        lib.isx_forward_coefficients.argtypes = [vp, vp, i32, vp, vp]
        lib.isx_forward_coefficients.restype = st
        lib.isx_sync_status.argtypes = [vp, vp]
        lib.isx_sync_status.restype = st
        lib.isx_last_launch_count.argtypes = [vp]
        lib.isx_last_launch_count.restype = i32
        lib.isx_set_timing.argtypes = [vp, i32]
        lib.isx_set_timing.restype = st
        lib.isx_stage_times.argtypes = [vp, ctypes.c_char_p, i64, vp, vp, i32]
        lib.isx_stage_times.restype = i32
        lib.isx_last_error.argtypes = [vp]
        lib.isx_last_error.restype = ctypes.c_char_p
        lib.isx_encode_tile_static.argtypes = [vp, vp, sz, ctypes.POINTER(sz), vp, ctypes.c_char_p, sz]
        lib.isx_encode_tile_static.restype = st
        lib.isx_decode_jobs.argtypes = [vp, vp, vp, vp, i32, vp, i32, i32, i32, vp]
        lib.isx_decode_jobs.restype = st
        lib.isx_get_schedule.argtypes = [vp, vp]
        lib.isx_get_schedule.restype = st
        lib.isx_set_schedule.argtypes = [vp, vp]
        lib.isx_set_schedule.restype = st
        lib.isx_autotune.argtypes = [vp, vp, i32, i32, vp]
        lib.isx_autotune.restype = st
        lib.isx_plan_encode.argtypes = [vp, vp, i32, ctypes.POINTER(vp)]
        lib.isx_plan_encode.restype = st
        lib.isx_plan_decode.argtypes = [vp, vp, i32, vp, i32, i32, i32, ctypes.POINTER(vp)]
        lib.isx_plan_decode.restype = st
        lib.isx_plan_launch_encode.argtypes = [vp, vp, sz, vp, vp]
        lib.isx_plan_launch_encode.restype = st
        lib.isx_plan_launch_decode.argtypes = [vp, vp, vp, vp]
        lib.isx_plan_launch_decode.restype = st
        lib.isx_plan_sync_status.argtypes = [vp, vp]
        lib.isx_plan_sync_status.restype = st
        lib.isx_plan_device_bytes.argtypes = [vp]
        lib.isx_plan_device_bytes.restype = sz
        lib.isx_plan_launch_count.argtypes = [vp]
        lib.isx_plan_launch_count.restype = i32
        lib.isx_plan_last_error.argtypes = [vp]
        lib.isx_plan_last_error.restype = ctypes.c_char_p
        lib.isx_plan_destroy.argtypes = [vp]
        lib.isx_plan_destroy.restype = None
        lib.isx_decode_jobs_scratch.argtypes = [vp, vp, i32, vp, i32, i32, i32, ctypes.POINTER(sz)]
        lib.isx_decode_jobs_scratch.restype = st
        lib.isx_reserve_scratch.argtypes = [vp, sz]
        lib.isx_reserve_scratch.restype = st
        lib.isx_scratch_bytes.argtypes = [vp]
        lib.isx_scratch_bytes.restype = sz
        lib.isx_decode_path.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_double)]
        lib.isx_decode_path.restype = i32
        lib.isx_set_tile_stamps.argtypes = [vp, vp, i32]
        lib.isx_set_tile_stamps.restype = st
        lib.isx_copy_rects.argtypes = [vp, vp, i32, vp]
        lib.isx_copy_rects.restype = st
        _lib = lib
        return lib


def decode_path(tile: Tile, level: int = 0, drop_lsb_planes: int = 0):
    """(path, bound) of isx_decode_path: path 1 = fused int16 inverse, 0 = global int32 inverse,
    -1 = invalid; bound = proven magnitude bound of the inverse's values (host computation only)."""
    lib = load()
    desc = tile.to_c()
    b = ctypes.c_double(0.0)
    path = int(lib.isx_decode_path(ctypes.byref(desc), level, drop_lsb_planes, ctypes.byref(b)))
    return path, float(b.value)


def encode_tile_static(tile: Tile, out, stream=None) -> int:
    """Encode one tile with the no-allocation entry point (isx_encode_tile_static).

    out: uint8 CUDA tensor (its size is the capacity).  Synchronous; returns
    the stream size.  On ISX_ERR_CAPACITY the raised error's ``needed``
    attribute holds the capacity the stream needs."""
    lib = load()
    desc = tile.to_c()
    size = ctypes.c_size_t(0)
    err = ctypes.create_string_buffer(512)
    rc = lib.isx_encode_tile_static(ctypes.byref(desc), out.data_ptr(), out.numel() * out.element_size(),
                                    ctypes.byref(size), _stream_ptr(stream), err, 512)
    if rc != ISX_OK:
        e = IsxError(rc, err.value.decode())
        e.needed = int(size.value)
        raise e
    return int(size.value)


class TileArray:
    """Tiles marshalled once into the C descriptor array (reuse it across calls)."""

    def __init__(self, tiles: Sequence[Tile]):
        self.tiles = list(tiles)
        self.c = (TileDescC * len(self.tiles))(*[t.to_c() for t in self.tiles])

    def __len__(self):
        return len(self.tiles)

    def __getitem__(self, i):
        return self.tiles[i]


def _tiles_c(tiles):
    if isinstance(tiles, TileArray):
        return tiles.c
    return (TileDescC * len(tiles))(*[t.to_c() for t in tiles])


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Codec:
    """A library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        self.ctx = ctypes.c_void_p()
        rc = self.lib.isx_create(ctypes.byref(self.ctx), device, hbm_budget_bytes)
        if rc != ISX_OK:
            raise IsxError(rc, "isx_create failed (no usable CUDA device?)")
        self.device = device

    def close(self):
        if self.ctx:
            self.lib.isx_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != ISX_OK:
            raise IsxError(rc, self.lib.isx_last_error(self.ctx).decode())

    @property
    def last_launch_count(self) -> int:
        return int(self.lib.isx_last_launch_count(self.ctx))

    def set_timing(self, enable: bool):
        self._check(self.lib.isx_set_timing(self.ctx, 1 if enable else 0))

    def stage_times(self) -> dict:
        """{stage name: (total ms, calls)} accumulated since timing was enabled."""
        names = ctypes.create_string_buffer(8192)
        ms = np.zeros(64, np.float64)
        cnt = np.zeros(64, np.int64)
        n = self.lib.isx_stage_times(self.ctx, names, 8192, ms.ctypes.data, cnt.ctypes.data, 64)
        keys = names.value.decode().split("\n")[:n]
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(keys)}

    def sync_status(self, stream=None) -> int:
        return int(self.lib.isx_sync_status(self.ctx, _stream_ptr(stream)))

    def set_tile_stamps(self, stamps=None):
        """stamps: uint64/int64 CUDA tensor of 4 * n_tiles (None: off); see isx_set_tile_stamps."""
        if stamps is None:
            self._check(self.lib.isx_set_tile_stamps(self.ctx, None, 0))
        else:
            assert stamps.numel() % 4 == 0
            self._check(self.lib.isx_set_tile_stamps(self.ctx, stamps.data_ptr(), stamps.numel() // 4))

    # ---------------------------------------------------------- device calls
    def encode_tiles(self, tiles: Sequence[Tile], out, offsets, stream=None):
        """out: uint8 CUDA tensor (capacity = its size); offsets: int64/uint64 CUDA tensor of n+1."""
        arr = _tiles_c(tiles)
        self._check(self.lib.isx_encode_tiles(self.ctx, arr, len(tiles), out.data_ptr(), out.numel() * out.element_size(),
                                              offsets.data_ptr(), _stream_ptr(stream)))

    def decode_region(self, stream_buf, offsets, tiles: Sequence[Tile], level, rect, out, drop_lsb_planes=0, stream=None):
        rx, ry, rw, rh = rect
        arr = _tiles_c(tiles)
        pitch = out.stride(0) * out.element_size()
        self._check(self.lib.isx_decode_region(self.ctx, stream_buf.data_ptr(), offsets.data_ptr(), arr, len(tiles), level, rx, ry,
                                               rw, rh, drop_lsb_planes, out.data_ptr(), pitch, _stream_ptr(stream)))

    def decode_jobs(self, stream_buf, offsets, tiles: Sequence[Tile], jobs, level=0, drop_lsb_planes=0, stream=None):
        """jobs: sequence of (tile index, (rx, ry, rw, rh), out tensor whose [0, 0] is pixel (rx, ry))."""
        arr = _tiles_c(tiles)
        jc = _jobs_c(jobs)
        self._check(self.lib.isx_decode_jobs(self.ctx, stream_buf.data_ptr(), offsets.data_ptr(), arr, len(tiles), jc, len(jobs),
                                             level, drop_lsb_planes, _stream_ptr(stream)))

    def decode_jobs_array(self, stream_buf, offsets, tiles, jobs: np.ndarray, level=0, drop_lsb_planes=0, stream=None):
        """jobs: contiguous numpy array of JOB_DTYPE (the C struct layout)."""
        assert jobs.dtype == JOB_DTYPE and jobs.flags["C_CONTIGUOUS"]
        self._check(self.lib.isx_decode_jobs(self.ctx, stream_buf.data_ptr(), offsets.data_ptr(), _tiles_c(tiles), len(tiles),
                                             jobs.ctypes.data, len(jobs), level, drop_lsb_planes, _stream_ptr(stream)))

    def decode_jobs_scratch(self, tiles, jobs: np.ndarray, level=0, drop_lsb_planes=0) -> int:
        assert jobs.dtype == JOB_DTYPE and jobs.flags["C_CONTIGUOUS"]
        n = ctypes.c_size_t(0)
        self._check(self.lib.isx_decode_jobs_scratch(self.ctx, _tiles_c(tiles), len(tiles), jobs.ctypes.data, len(jobs), level,
                                                     drop_lsb_planes, ctypes.byref(n)))
        return int(n.value)

    def copy_rects(self, copies: np.ndarray, stream=None):
        """copies: contiguous numpy array of COPY_DTYPE (device addresses); one launch (isx_copy_rects)."""
        assert copies.dtype == COPY_DTYPE and copies.flags["C_CONTIGUOUS"]
        self._check(self.lib.isx_copy_rects(self.ctx, copies.ctypes.data, len(copies), _stream_ptr(stream)))

    def reserve_scratch(self, nbytes: int):
        self._check(self.lib.isx_reserve_scratch(self.ctx, nbytes))

    @property
    def scratch_bytes(self) -> int:
        return int(self.lib.isx_scratch_bytes(self.ctx))

    def get_schedule(self) -> dict:
        sc = ScheduleC()
        self._check(self.lib.isx_get_schedule(self.ctx, ctypes.byref(sc)))
        return {"forward_threads": list(sc.forward_threads), "inverse_threads": list(sc.inverse_threads)}

    def set_schedule(self, forward_threads, inverse_threads):
        sc = ScheduleC()
        for k in range(SIZE_CLASSES):
            sc.forward_threads[k] = forward_threads[k]
            sc.inverse_threads[k] = inverse_threads[k]
        self._check(self.lib.isx_set_schedule(self.ctx, ctypes.byref(sc)))

    def autotune(self, tiles: Sequence[Tile], reps: int = 3, stream=None) -> dict:
        arr = _tiles_c(tiles)
        self._check(self.lib.isx_autotune(self.ctx, arr, len(tiles), reps, _stream_ptr(stream)))
        return self.get_schedule()

    def plan_encode(self, tiles: Sequence[Tile]) -> "Plan":
        arr = _tiles_c(tiles)
        h = ctypes.c_void_p()
        self._check(self.lib.isx_plan_encode(self.ctx, arr, len(tiles), ctypes.byref(h)))
        return Plan(self.lib, h, "encode", keep=(tiles,))

    def plan_decode(self, tiles: Sequence[Tile], jobs, level=0, drop_lsb_planes=0) -> "Plan":
        arr = _tiles_c(tiles)
        jc = _jobs_c(jobs)
        h = ctypes.c_void_p()
        self._check(self.lib.isx_plan_decode(self.ctx, arr, len(tiles), jc, len(jobs), level, drop_lsb_planes, ctypes.byref(h)))
        return Plan(self.lib, h, "decode", keep=(tiles, jobs))

    def forward_coefficients(self, tiles: Sequence[Tile], out, stream=None):
        arr = _tiles_c(tiles)
        self._check(self.lib.isx_forward_coefficients(self.ctx, arr, len(tiles), out.data_ptr(), _stream_ptr(stream)))

    # ------------------------------------------------------------ host calls
    def encode_tiles_host(self, tiles: Sequence[Tile], out: np.ndarray, offsets: np.ndarray, stream=None):
        arr = _tiles_c(tiles)
        assert out.dtype == np.uint8 and offsets.dtype == np.uint64 and offsets.size == len(tiles) + 1
        self._check(self.lib.isx_encode_tiles_host(self.ctx, arr, len(tiles), out.ctypes.data, out.nbytes, offsets.ctypes.data,
                                                   _stream_ptr(stream)))

    def decode_region_host(self, stream_buf: np.ndarray, offsets: np.ndarray, tiles: Sequence[Tile], level, rect, out: np.ndarray,
                           drop_lsb_planes=0, stream=None):
        rx, ry, rw, rh = rect
        arr = _tiles_c(tiles)
        self._check(self.lib.isx_decode_region_host(self.ctx, stream_buf.ctypes.data, offsets.ctypes.data, arr, len(tiles), level,
                                                    rx, ry, rw, rh, drop_lsb_planes, out.ctypes.data, out.strides[0],
                                                    _stream_ptr(stream)))


def _jobs_c(jobs):
    arr = (DecodeJobC * max(1, len(jobs)))()
    for k, (ti, rect, out) in enumerate(jobs):
        rx, ry, rw, rh = rect
        arr[k].tile, arr[k].rx, arr[k].ry, arr[k].rw, arr[k].rh = ti, rx, ry, rw, rh
        arr[k].d_out = out.data_ptr()
        arr[k].out_pitch_bytes = out.stride(0) * out.element_size()
    return arr


class Plan:
    """A prepared encode or decode (isx_plan_*): launches enqueue kernels only, so they can be graph-captured."""

    def __init__(self, lib, handle, kind, keep=()):
        self.lib, self.h, self.kind, self.keep = lib, handle, kind, keep

    def _check(self, rc):
        if rc != ISX_OK:
            raise IsxError(rc, self.lib.isx_plan_last_error(self.h).decode())

    def launch_encode(self, out, offsets, stream=None):
        self._check(self.lib.isx_plan_launch_encode(self.h, out.data_ptr(), out.numel() * out.element_size(), offsets.data_ptr(),
                                                    _stream_ptr(stream)))

    def launch_decode(self, stream_buf, offsets, stream=None):
        self._check(self.lib.isx_plan_launch_decode(self.h, stream_buf.data_ptr(), offsets.data_ptr(), _stream_ptr(stream)))

    def sync_status(self, stream=None) -> int:
        return int(self.lib.isx_plan_sync_status(self.h, _stream_ptr(stream)))

    @property
    def device_bytes(self) -> int:
        return int(self.lib.isx_plan_device_bytes(self.h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.isx_plan_launch_count(self.h))

    def close(self):
        if self.h:
            self.lib.isx_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ helpers
def level_dim(n: int, z: int) -> int:
    for _ in range(z):
        n = (n + 1) // 2
    return n


def tile_from_tensor(t, levels: int, bits: int, qstep_log2=(), x0: int = 0, y0: int = 0, transform: int = CT_DEFAULT) -> Tile:
    """Tile over an HWC (or HW) CUDA tensor view (uint8, or int16/uint16 storage for bits > 8)."""
    h, w = int(t.shape[0]), int(t.shape[1])
    c = 1 if t.dim() == 2 else int(t.shape[2])
    return Tile(width=w, height=h, channels=c, bits=bits, levels=levels, qstep_log2=tuple(qstep_log2), x0=x0, y0=y0,
                pixels=t.data_ptr(), row_pitch_bytes=t.stride(0) * t.element_size(), keep=t, transform=transform)


def tile_from_array(a: np.ndarray, levels: int, bits: int, qstep_log2=(), x0: int = 0, y0: int = 0,
                    transform: int = CT_DEFAULT) -> Tile:
    """Tile over a host numpy view (for the *_host calls)."""
    h, w = a.shape[:2]
    c = 1 if a.ndim == 2 else a.shape[2]
    return Tile(width=w, height=h, channels=c, bits=bits, levels=levels, qstep_log2=tuple(qstep_log2), x0=x0, y0=y0,
                pixels=a.ctypes.data, row_pitch_bytes=a.strides[0], keep=a, transform=transform)
