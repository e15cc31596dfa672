"""Seeded synthetic inputs shaped like the paper's workloads (no codec code).

The pixels come from ``synth.c`` (counter-based splitmix64, IEEE-exact
arithmetic), so the same seed gives the same bytes on every host.  Both the
CPU oracle and the GPU library are fed from here.

Workload recipes (stand-ins for the paper's datasets, which are not
available: TCIA CR/DX/MG radiographs and Philips 9-bit pathology scans):

* ``stain``   512 x 512 RGB8 tile, near-white base with smooth colour
  gradients, pink/purple stain hues, N(0, 8^2) noise.
* ``slide``   whole-slide-shaped RGB8 image (any crop of an unbounded
  plane): ~60% pale background 230..250 with N(0, 3^2) noise, tissue of
  pink stroma with dark purple nuclei (radius 3..8 px), N(0, 10^2).
* ``phantom`` 12-bit monochrome in uint16: 8..16 smooth elliptical
  phantoms summed and clamped to 4095, each value v replaced by a Poisson(v) sample.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libisx_synth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 20050813


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, i32, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.isx_gen_stain.argtypes = [u64, i64, i64, vp, i64, i32]
            lib.isx_gen_slide.argtypes = [u64, i64, i64, i64, i64, vp, i64, i32]
            lib.isx_gen_phantom.argtypes = [u64, i64, i64, i64, i64, i64, i64, vp, i64, i32]
            lib.isx_gen_mix64.argtypes = [u64]
            lib.isx_gen_mix64.restype = u64
            lib.isx_gen_normals.argtypes = [u64, i64, vp]
            lib.isx_gen_poissons.argtypes = [ctypes.c_double, u64, i64, vp]
            lib.isx_gen_series.argtypes = [vp, vp, vp, i64, vp, vp, vp]
            _lib = lib
    return _lib


def _threads(threads):
    return threads if threads else max(1, os.cpu_count() or 1)


def config_seed(config_id: int, seed: int = BASE_SEED) -> int:
    """Per-workload seed derived by hashing (seed, config id)."""
    return int(_get().isx_gen_mix64((seed * 1000003 + config_id) & 0xFFFFFFFFFFFFFFFF))


def mix64(x: int) -> int:
    return int(_get().isx_gen_mix64(x & 0xFFFFFFFFFFFFFFFF))


def normals(key0: int, n: int) -> np.ndarray:
    """n standard normal deviates of the generators' Box-Muller sampler (streams key0, key0 + 1, ...)."""
    out = np.empty(n, np.float64)
    _get().isx_gen_normals(key0 & 0xFFFFFFFFFFFFFFFF, n, out.ctypes.data)
    return out


def poissons(lam: float, key0: int, n: int) -> np.ndarray:
    """n Poisson(lam) samples of the generators' sampler (streams key0, key0 + 1, ...)."""
    out = np.empty(n, np.int64)
    _get().isx_gen_poissons(float(lam), key0 & 0xFFFFFFFFFFFFFFFF, n, out.ctypes.data)
    return out


def series(x, u, k):
    """The generators' own ln x, cos(2 pi u) and ln k! (series in +, -, *, /), elementwise."""
    x = np.ascontiguousarray(x, np.float64); u = np.ascontiguousarray(u, np.float64)
    k = np.ascontiguousarray(k, np.int64)
    n = len(x)
    assert len(u) == n and len(k) == n
    a, b, c = np.empty(n), np.empty(n), np.empty(n)
    _get().isx_gen_series(x.ctypes.data, u.ctypes.data, k.ctypes.data, n, a.ctypes.data, b.ctypes.data, c.ctypes.data)
    return a, b, c


def stain(seed: int, w: int = 512, h: int = 512, threads: int = 0) -> np.ndarray:
    out = np.empty((h, w, 3), np.uint8)
    _get().isx_gen_stain(seed, w, h, out.ctypes.data, out.strides[0], _threads(threads))
    return out


def slide(seed: int, x0: int, y0: int, w: int, h: int, out: np.ndarray | None = None, threads: int = 0) -> np.ndarray:
    if out is None:
        out = np.empty((h, w, 3), np.uint8)
    assert out.dtype == np.uint8 and out.shape[:2] == (h, w) and out.strides[1] == 3 and out.strides[2] == 1
    _get().isx_gen_slide(seed, x0, y0, w, h, out.ctypes.data, out.strides[0], _threads(threads))
    return out


def phantom(seed: int, W: int, H: int, x0: int = 0, y0: int = 0, w: int | None = None, h: int | None = None,
            threads: int = 0) -> np.ndarray:
    w = W if w is None else w
    h = H if h is None else h
    out = np.empty((h, w), np.uint16)
    _get().isx_gen_phantom(seed, W, H, x0, y0, w, h, out.ctypes.data, out.strides[0], _threads(threads))
    return out


def batch_specs(seed: int, n: int):
    """Tile recipe of the mixed batch workload: per tile, width and height
    uniform in 17..256, RGB8 (a crop of the slide generator) or 12-bit mono
    (a crop of the phantom generator) with equal odds, 2..6 wavelet levels,
    lossless or lossy (steps 8/4/2 on levels 1-3) with equal odds, and the
    crop position.  numpy's seeded generator draws the choices."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n):
        w, h = int(rng.integers(17, 257)), int(rng.integers(17, 257))
        levels = int(rng.integers(2, 7))
        rgb = bool(rng.random() < 0.5)
        if rgb:
            x0, y0 = int(rng.integers(0, 40000 - w)), int(rng.integers(0, 30000 - h))
        else:
            x0, y0 = int(rng.integers(0, 2048 - w)), int(rng.integers(0, 2048 - h))
        lossy = bool(rng.random() < 0.5)
        q = ([3, 2, 1] + [0] * 13)[:levels + 1] if lossy else [0] * (levels + 1)
        specs.append({"w": w, "h": h, "levels": levels, "rgb": rgb, "bits": 8 if rgb else 12, "x0": x0, "y0": y0, "q": q})
    return specs


def batch_image(spec, threads: int = 1) -> np.ndarray:
    """Pixels of one tile of batch_specs()."""
    if spec["rgb"]:
        return slide(config_seed(3), spec["x0"], spec["y0"], spec["w"], spec["h"], threads=threads)
    return phantom(config_seed(2), 2048, 2048, spec["x0"], spec["y0"], spec["w"], spec["h"], threads=threads)
