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


SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    """The harness, built with the address and undefined-behaviour
    sanitizers where the compiler has them: then every plane and scratch
    access of the device code outside its buffer fails the run."""
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("wl") / "warp_levels_host")
    base = [cxx, "-std=c++20", "-O1", "-g", "-pthread", os.path.join(HERE, "warp_levels_host.cpp"), "-o", exe]
    r = subprocess.run(base[:1] + SANITIZE + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("harness build failed:\n" + r.stderr[-2000:])
    return exe


def run_many(exe, cases):
    """cases: [(plane, levels)] -> the harness's result plane of each."""
    inp = []
    for plane, levels in cases:
        h, w = plane.shape
        inp.append(f"{w} {h} {levels}\n" + "\n".join(" ".join(str(int(v)) for v in row) for row in plane) + "\n")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([exe], input="".join(inp), capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    out = r.stdout.split("--\n")
    assert len(out) == len(cases) + 1 and out[-1] == ""
    return [np.array([[int(v) for v in line.split()] for line in o.strip().splitlines()], dtype=np.int64) for o in out[:-1]]


def run(exe, plane: np.ndarray, levels: int) -> np.ndarray:
    return run_many(exe, [(plane, levels)])[0]


@pytest.mark.parametrize("h,w,levels", [(32, 32, 5), (32, 32, 8), (1, 32, 5), (32, 1, 4), (25, 18, 3), (17, 31, 6),
                                        (2, 2, 1), (3, 5, 2), (1, 1, 3), (31, 32, 5), (9, 30, 15)])
def test_warp_levels_match_oracle(harness, orc, h, w, levels):
    rng = np.random.default_rng(h * 100 + w + levels)
    # level-0 samples of an RGB8 tile after the colour transform reach [-255, 255]
    plane = rng.integers(-255, 256, size=(h, w)).astype(np.int64)
    got = interleaved_to_mallat(run(harness, plane, levels), levels)
    ref = orc.dwt2_forward(plane, levels)
    assert np.array_equal(got, ref), f"{h}x{w} L={levels}: {np.argwhere(got != ref)[:5].tolist()}"


def test_warp_levels_every_grid_shape(harness, orc):
    """Every grid of 1..32 x 1..32 samples at a random level count 1..7,
    in one run of the (sanitized) harness."""
    rng = np.random.default_rng(2024)
    cases = []
    for h in range(1, 33):
        for w in range(1, 33):
            cases.append((rng.integers(-255, 256, size=(h, w)).astype(np.int64), int(rng.integers(1, 8))))
    for (plane, levels), got in zip(cases, run_many(harness, cases)):
        ref = orc.dwt2_forward(plane, levels)
        assert np.array_equal(interleaved_to_mallat(got, levels), ref), (plane.shape, levels)
