"""The encode's one-warp coarse levels (csrc/isx_warp_levels.cuh) run on the
host, lane by lane, against the oracle's 2-D 5/3 transform (Sec. 4).

The header is the device code itself, compiled for the host with three
macros (warp barrier, function qualifier, min); tests/warp_levels_host.cpp
runs its 32 lanes as threads.  The kernel's result is in the fused kernels'
in-place interleaved layout; the test rearranges it into the oracle's
Mallat layout (per level: LL, HL, LH, HH quadrants) and compares every
coefficient, for planes of up to 32 x 32 samples (the grids the warp path
takes) of every shape class: square, one row or column, odd sizes, and more
levels than the plane has halvings."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _ld(n, l):
    return -(-n // (1 << l))


def interleaved_to_mallat(I: np.ndarray, levels: int) -> np.ndarray:
    h, w = I.shape
    M = np.zeros_like(I)
    for l in range(levels):
        cw, ch = _ld(w, l), _ld(h, l)
        if cw <= 1 and ch <= 1:
            break
        s = 1 << l
        g = I[: (ch - 1) * s + 1: s, : (cw - 1) * s + 1: s]   # the level-l grid
        lw, lh = _ld(cw, 1), _ld(ch, 1)
        M[:lh, lw:cw] = g[0::2, 1::2]   # HL
        M[lh:ch, :lw] = g[1::2, 0::2]   # LH
        M[lh:ch, lw:cw] = g[1::2, 1::2]  # HH
    lvl = min(levels, max((max(w, h) - 1).bit_length(), 0))
    cw, ch = _ld(w, lvl), _ld(h, lvl)
    s = 1 << lvl
    M[:ch, :cw] = I[: (ch - 1) * s + 1: s, : (cw - 1) * s + 1: s]   # LL
    return M


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("wl") / "warp_levels_host")
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", os.path.join(HERE, "warp_levels_host.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("harness build failed:\n" + r.stderr[-2000:])
    return exe


def run(exe, plane: np.ndarray, levels: int) -> np.ndarray:
    h, w = plane.shape
    inp = f"{w} {h} {levels}\n" + "\n".join(" ".join(str(int(v)) for v in row) for row in plane) + "\n"
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return np.array([[int(v) for v in line.split()] for line in r.stdout.strip().splitlines()], dtype=np.int64)


@pytest.mark.parametrize("h,w,levels", [(32, 32, 5), (32, 32, 8), (1, 32, 5), (32, 1, 4), (25, 18, 3), (17, 31, 6),
                                        (2, 2, 1), (3, 5, 2), (1, 1, 3), (31, 32, 5), (9, 30, 15)])
def test_warp_levels_match_oracle(harness, orc, h, w, levels):
    rng = np.random.default_rng(h * 100 + w + levels)
    # level-0 samples of an RGB8 tile after the colour transform reach [-255, 255]
    plane = rng.integers(-255, 256, size=(h, w)).astype(np.int64)
    got = interleaved_to_mallat(run(harness, plane, levels), levels)
    ref = orc.dwt2_forward(plane, levels)
    assert np.array_equal(got, ref), f"{h}x{w} L={levels}: {np.argwhere(got != ref)[:5].tolist()}"
