"""CPU oracle of the codec — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  It wraps ``isx_oracle.cpp`` (plain,
slow, single-threaded per tile C++) through ctypes and shares no code with
the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isx_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcTile(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("bits", ctypes.c_int32), ("levels", ctypes.c_int32), ("x0", ctypes.c_int32),
                ("y0", ctypes.c_int32), ("qstep_log2", ctypes.c_uint8 * 16), ("transform", ctypes.c_int32)]


# colour transform selectors of a tile (orc_tile.transform): DEFAULT = RCT for three channels and none
# otherwise; RCT and YCOCG_R act on channels 0..2 of a tile of three or more channels
CT_DEFAULT, CT_NONE, CT_RCT, CT_YCOCG_R = 0, 1, 2, 3


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            sig = {
                "orc_rct_forward": ([vp, i64, vp], None),
                "orc_rct_inverse": ([vp, i64, vp], None),
                "orc_ycocg_forward": ([vp, i64, vp], None),
                "orc_ycocg_inverse": ([vp, i64, vp], None),
                "orc_lift53_forward": ([vp, i64, vp, vp], None),
                "orc_lift53_inverse": ([vp, vp, i64, vp], None),
                "orc_dwt2_forward": ([vp, i64, i64, i32], None),
                "orc_dwt2_inverse": ([vp, i64, i64, i32], None),
                "orc_quantise": ([i64, i64], i64),
                "orc_dequantise": ([i64, i64], i64),
                "orc_area_T": ([i64, i64, i64, vp], None),
                "orc_area_symbol": ([vp, i64, i64, i64, i64, i64], i32),
                "orc_huffman": ([vp, vp, vp, vp, i64], i64),
                "orc_tokens": ([vp, i64, i32, i32, vp, vp, i64], i64),
                "orc_encode_block": ([i32, i64, i64, vp, vp, i64, vp], i64),
                "orc_decode_block": ([i32, i64, i64, vp, i64, i32, vp], i32),
                "orc_tile_coefficients": ([vp, vp, i64, vp], i32),
                "orc_encode_tile": ([vp, vp, i64, vp, i64], i64),
                "orc_decode_tile": ([vp, i64, i32, i32, vp, i64], i32),
                "orc_encode_tiles_mt": ([i64, vp, vp, vp, vp, vp, vp, i32], None),
                "orc_decode_tiles_mt": ([i64, vp, vp, i32, vp, vp, vp, i32], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data


def tile_struct(width, height, channels, bits, levels, qstep_log2=(), x0=0, y0=0, transform=CT_DEFAULT) -> OrcTile:
    t = OrcTile()
    t.width, t.height, t.channels, t.bits, t.levels, t.x0, t.y0 = width, height, channels, bits, levels, x0, y0
    t.transform = transform
    q = list(qstep_log2) + [0] * (16 - len(qstep_log2))
    for i in range(16):
        t.qstep_log2[i] = q[i]
    return t


# ------------------------------------------------------------- step level
def rct_forward(rgb: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(rgb, dtype=np.int64).reshape(-1, 3)
    out = np.empty_like(a)
    _get().orc_rct_forward(_p(a), a.shape[0], _p(out))
    return out.reshape(np.shape(rgb))


def rct_inverse(ycc: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(ycc, dtype=np.int64).reshape(-1, 3)
    out = np.empty_like(a)
    _get().orc_rct_inverse(_p(a), a.shape[0], _p(out))
    return out.reshape(np.shape(ycc))


def ycocg_forward(rgb: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(rgb, dtype=np.int64).reshape(-1, 3)
    out = np.empty_like(a)
    _get().orc_ycocg_forward(_p(a), a.shape[0], _p(out))
    return out.reshape(np.shape(rgb))


def ycocg_inverse(ycc: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(ycc, dtype=np.int64).reshape(-1, 3)
    out = np.empty_like(a)
    _get().orc_ycocg_inverse(_p(a), a.shape[0], _p(out))
    return out.reshape(np.shape(ycc))


def lift53_forward(x):
    x = np.ascontiguousarray(x, dtype=np.int64)
    n = x.shape[0]
    lo = np.zeros((n + 1) // 2, np.int64)
    hi = np.zeros(n // 2, np.int64)
    _get().orc_lift53_forward(_p(x), n, _p(lo), _p(hi))
    return lo, hi


def lift53_inverse(lo, hi):
    lo = np.ascontiguousarray(lo, dtype=np.int64)
    hi = np.ascontiguousarray(hi, dtype=np.int64)
    n = lo.shape[0] + hi.shape[0]
    x = np.zeros(n, np.int64)
    _get().orc_lift53_inverse(_p(lo), _p(hi) if hi.size else None, n, _p(x))
    return x


def dwt2_forward(plane: np.ndarray, levels: int) -> np.ndarray:
    a = np.ascontiguousarray(plane, dtype=np.int64).copy()
    h, w = a.shape
    _get().orc_dwt2_forward(_p(a), w, h, levels)
    return a


def dwt2_inverse(plane: np.ndarray, levels: int) -> np.ndarray:
    a = np.ascontiguousarray(plane, dtype=np.int64).copy()
    h, w = a.shape
    _get().orc_dwt2_inverse(_p(a), w, h, levels)
    return a


def quantise(c: int, delta: int) -> int:
    return int(_get().orc_quantise(c, delta))


def dequantise(q: int, delta: int) -> int:
    return int(_get().orc_dequantise(q, delta))


def area_T(k: int, w: int, h: int):
    out = np.zeros(3, np.int64)
    _get().orc_area_T(k, w, h, _p(out))
    return int(out[0]), int(out[1]), int(out[2])


def area_symbol(coef: np.ndarray, i: int, j: int, p: int, d: int) -> int:
    a = np.ascontiguousarray(coef, dtype=np.int64)
    return int(_get().orc_area_symbol(_p(a), a.shape[1], i, j, p, d))


def huffman(freq):
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    assert f.shape == (256,)
    ln = np.zeros(256, np.int32)
    code = np.zeros(256, np.uint32)
    tree = np.zeros(1024, np.uint8)
    nbits = _get().orc_huffman(_p(f), _p(ln), _p(code), _p(tree), tree.size)
    return ln, code, tree[: (nbits + 7) // 8], int(nbits)


def tokens(seg, czr: int, w: int):
    s = np.ascontiguousarray(seg, dtype=np.int32)
    cap = max(16, 4 * s.size + 16)
    sym = np.zeros(cap, np.int32)
    run = np.zeros(cap, np.int64)
    n = _get().orc_tokens(_p(s), s.size, czr, w, _p(sym), _p(run), cap)
    return list(zip(sym[:n].tolist(), run[:n].tolist()))


def encode_block(coef: np.ndarray):
    """coef: (p, h, w) int64 padded block. Returns (bytes, stats dict)."""
    c = np.ascontiguousarray(coef, dtype=np.int64)
    p, h, w = c.shape
    cap = 64 + p * h * w * 8
    out = np.zeros(cap, np.uint8)
    st = np.zeros(8 + 256, np.int64)
    n = _get().orc_encode_block(p, w, h, _p(c), _p(out), cap, _p(st))
    assert n > 0
    keys = ["d", "czr", "w", "t", "b", "l_prov", "n_sym"]
    stats = dict(zip(keys, st[:7].tolist()))
    stats["prov_len"] = st[8:].tolist()   # provisional code lengths behind l (0 = absent)
    return out[:n].tobytes(), stats


def decode_block(data: bytes, p: int, w: int, h: int, drop: int = 0):
    buf = np.frombuffer(data, np.uint8).copy() if len(data) else np.zeros(1, np.uint8)
    out = np.zeros((p, h, w), np.int64)
    rc = _get().orc_decode_block(p, w, h, _p(buf), len(data), drop, _p(out))
    if rc != 0:
        raise ValueError("corrupt block")
    return out


# -------------------------------------------------------------- tile level
def _pixels(img: np.ndarray):
    a = np.ascontiguousarray(img)
    return a, a.strides[0]


def tile_coefficients(img: np.ndarray, levels: int, bits: int, qstep_log2=(), transform=CT_DEFAULT) -> np.ndarray:
    a, pitch = _pixels(img)
    h, w = a.shape[:2]
    C = 1 if a.ndim == 2 else a.shape[2]
    t = tile_struct(w, h, C, bits, levels, qstep_log2, transform=transform)
    out = np.zeros((C, h, w), np.int64)
    rc = _get().orc_tile_coefficients(ctypes.byref(t), _p(a), pitch, _p(out))
    if rc != 0:
        raise ValueError("bad tile")
    return out


def encode_tile(img: np.ndarray, levels: int, bits: int, qstep_log2=(), transform=CT_DEFAULT) -> bytes:
    a, pitch = _pixels(img)
    h, w = a.shape[:2]
    C = 1 if a.ndim == 2 else a.shape[2]
    t = tile_struct(w, h, C, bits, levels, qstep_log2, transform=transform)
    cap = 4096 + a.nbytes * 4
    while True:
        out = np.zeros(cap, np.uint8)
        n = _get().orc_encode_tile(ctypes.byref(t), _p(a), pitch, _p(out), cap)
        if n == 0:
            raise ValueError("bad tile")
        if n > 0:
            return out[:n].tobytes()
        cap = -n


def decode_tile(stream: bytes, level: int = 0, drop: int = 0) -> np.ndarray:
    s = np.frombuffer(stream, np.uint8)
    w = int(s[4]) | (int(s[5]) << 8)
    h = int(s[6]) | (int(s[7]) << 8)
    C, bits = int(s[8]), int(s[9])
    zw, zh = w, h
    for _ in range(level):
        zw, zh = (zw + 1) // 2, (zh + 1) // 2
    dt = np.uint8 if bits <= 8 else np.uint16
    out = np.zeros((zh, zw, C) if C > 1 else (zh, zw), dt)
    rc = _get().orc_decode_tile(_p(s), s.size, level, drop, _p(out), out.strides[0])
    if rc != 0:
        raise ValueError("corrupt tile stream")
    return out


def encode_tiles_mt(imgs, tiles, threads: int):
    """imgs: list of HWC arrays, tiles: list of OrcTile; returns list of bytes."""
    n = len(imgs)
    arrs = [np.ascontiguousarray(a) for a in imgs]
    caps = np.array([4096 + a.nbytes * 4 for a in arrs], np.int64)
    outs = [np.zeros(c, np.uint8) for c in caps]
    T = (OrcTile * n)(*tiles)
    px = (ctypes.c_void_p * n)(*[a.ctypes.data for a in arrs])
    pitch = np.array([a.strides[0] for a in arrs], np.int64)
    op = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    sizes = np.zeros(n, np.int64)
    _get().orc_encode_tiles_mt(n, ctypes.byref(T), px, _p(pitch), op, _p(caps), _p(sizes), threads)
    assert (sizes > 0).all()
    return [outs[i][: sizes[i]].tobytes() for i in range(n)]


def decode_tiles_mt(streams, level: int, outs, threads: int):
    n = len(streams)
    bufs = [np.frombuffer(s, np.uint8) for s in streams]
    sp = (ctypes.c_void_p * n)(*[b.ctypes.data for b in bufs])
    sizes = np.array([b.size for b in bufs], np.int64)
    op = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    pitch = np.array([o.strides[0] for o in outs], np.int64)
    rc = np.zeros(n, np.int32)
    _get().orc_decode_tiles_mt(n, sp, _p(sizes), level, op, _p(pitch), _p(rc), threads)
    assert (rc == 0).all()
