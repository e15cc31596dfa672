"""Pins of the oracle's colour transform, 5/3 lifting, 2-D recursion and
quantiser against closed forms and invariants (Sec. 3, Sec. 4 of the paper).
"""
import itertools

import numpy as np
import pytest


# ---------------------------------------------------------------- RCT
def test_rct_exhaustive_roundtrip_and_ranges(orc):
    # all 2^24 RGB8 triples in chunks: exact inverse, Y in [0,255], chroma in [-255,255]
    for hi in range(0, 256, 16):
        r, g, b = np.meshgrid(np.arange(hi, hi + 16), np.arange(256), np.arange(256), indexing="ij")
        rgb = np.stack([r.ravel(), g.ravel(), b.ravel()], 1).astype(np.int64)
        ycc = orc.rct_forward(rgb)
        assert ycc[:, 0].min() >= 0 and ycc[:, 0].max() <= 255
        assert ycc[:, 1:].min() >= -255 and ycc[:, 1:].max() <= 255
        back = orc.rct_inverse(ycc)
        assert np.array_equal(back, rgb)


def test_rct_closed_forms(orc):
    # grey maps to (v, 0, 0); the chroma channels are the differences to green
    for v in (0, 1, 77, 128, 255):
        assert orc.rct_forward(np.array([[v, v, v]])).tolist() == [[v, 0, 0]]
    # pure primaries: luma is the weighted mean rounded down
    assert orc.rct_forward(np.array([[255, 0, 0]])).tolist() == [[63, 0, 255]]
    assert orc.rct_forward(np.array([[0, 255, 0]])).tolist() == [[127, -255, -255]]
    assert orc.rct_forward(np.array([[0, 0, 255]])).tolist() == [[63, 255, 0]]


# ------------------------------------------------------------ 5/3 lifting
def fir_53(x):
    """Linear 5/3 analysis filters with whole-sample symmetric extension,
    exact when every lifting division is exact (inputs in 8Z)."""
    n = len(x)
    if n == 1:
        return np.array(x[:1], float), np.zeros(0)
    def ext(i):
        period = 2 * (n - 1)
        i %= period
        return x[period - i if i >= n else i]
    lo = [(-ext(2 * k - 2) + 2 * ext(2 * k - 1) + 6 * ext(2 * k) + 2 * ext(2 * k + 1) - ext(2 * k + 2)) / 8
          for k in range((n + 1) // 2)]
    hi = [ext(2 * k + 1) - (ext(2 * k) + ext(2 * k + 2)) / 2 for k in range(n // 2)]
    return np.array(lo), np.array(hi)


def test_lift53_matches_fir_filters_when_exact(orc):
    rng = np.random.default_rng(1)
    for n in list(range(1, 20)) + [31, 64, 65]:
        for _ in range(20):
            x = rng.integers(-64, 64, n) * 8
            lo, hi = orc.lift53_forward(x)
            flo, fhi = fir_53(list(x))
            assert np.array_equal(lo, flo), (n, x)
            assert np.array_equal(hi, fhi), (n, x)


def test_lift53_perfect_reconstruction_exhaustive_small(orc):
    for n in range(1, 7):
        for x in itertools.product(range(-2, 3), repeat=n):
            lo, hi = orc.lift53_forward(np.array(x))
            assert len(lo) == (n + 1) // 2 and len(hi) == n // 2
            assert orc.lift53_inverse(lo, hi).tolist() == list(x)


def test_lift53_perfect_reconstruction_random(orc):
    rng = np.random.default_rng(2)
    for n in range(1, 130):
        x = rng.integers(-70000, 70000, n)
        lo, hi = orc.lift53_forward(x)
        assert np.array_equal(orc.lift53_inverse(lo, hi), x)


def test_lift53_constant_and_ramp(orc):
    for n in range(2, 40):
        lo, hi = orc.lift53_forward(np.full(n, 37))
        assert (hi == 0).all() and (lo == 37).all()
        ramp = np.arange(n) * 3 + 5
        lo, hi = orc.lift53_forward(ramp)
        # a linear ramp is predicted exactly away from the mirrored right edge
        interior = hi[: (n - 1) // 2] if n % 2 == 0 else hi
        assert (interior == 0).all()


def test_lift53_rounding_is_floor(orc):
    # x = [0, 1, 1]: d0 = 1 - floor(1/2) = 1; s0 = 0 + floor((1+1+2)/4) = 1;
    # s1 = 1 + floor((1+1+2)/4) = 2.  x = [0, -1, 0]: d0 = -1, s0 = floor(0/4) = 0
    lo, hi = orc.lift53_forward(np.array([0, 1, 1]))
    assert hi.tolist() == [1] and lo.tolist() == [1, 2]
    lo, hi = orc.lift53_forward(np.array([0, -3, 0]))
    assert hi.tolist() == [-3] and lo.tolist() == [-1, -1]  # floor(-4/4) = -1 each side


# ------------------------------------------------------------------- 2-D
def test_dwt2_perfect_reconstruction_all_small_sizes(orc):
    rng = np.random.default_rng(3)
    for h in range(1, 34):
        for w in range(1, 34, 3):
            for levels in range(0, 7):
                x = rng.integers(-300, 300, (h, w))
                y = orc.dwt2_forward(x, levels)
                assert np.array_equal(orc.dwt2_inverse(y, levels), x)


def test_dwt2_subband_orientation(orc):
    # an image that varies only along x has no vertical detail: LH = HH = 0
    w, h = 24, 16
    x = np.tile(np.array([(i * 37) % 11 for i in range(w)]), (h, 1))
    y = orc.dwt2_forward(x, 1)
    lw, lh = (w + 1) // 2, (h + 1) // 2
    assert (y[lh:, :] == 0).all()                    # LH and HH (bottom half)
    assert (y[:lh, lw:] != 0).any()                  # HL carries the horizontal detail
    # and the transpose: variation along y only -> HL = HH = 0
    y2 = orc.dwt2_forward(x.T.copy(), 1)
    lw2, lh2 = (h + 1) // 2, (w + 1) // 2
    assert (y2[:, lw2:] == 0).all()
    assert (y2[lh2:, :lw2] != 0).any()


def test_dwt2_level1_matches_separable_fir_when_exact(orc):
    rng = np.random.default_rng(4)
    for (h, w) in [(8, 8), (9, 12), (16, 5), (13, 13)]:
        x = rng.integers(-20, 20, (h, w)) * 64
        y = orc.dwt2_forward(x, 1)
        # columns then rows with the linear filters
        cols = np.zeros((h, w))
        for c in range(w):
            lo, hi = fir_53(list(x[:, c].astype(float)))
            cols[:, c] = np.concatenate([lo, hi])
        ref = np.zeros((h, w))
        for r in range(h):
            lo, hi = fir_53(list(cols[r, :]))
            ref[r, :] = np.concatenate([lo, hi])
        assert np.array_equal(y, ref)


def test_dwt2_recursion_is_on_ll(orc):
    rng = np.random.default_rng(5)
    x = rng.integers(0, 255, (37, 50))
    y3 = orc.dwt2_forward(x, 3)
    y1 = orc.dwt2_forward(x, 1)
    lw, lh = 25, 19
    y1[:lh, :lw] = orc.dwt2_forward(y1[:lh, :lw], 2)
    assert np.array_equal(y1, y3)


# ------------------------------------------------------------ quantiser
def test_quantiser_deadzone_and_midpoint(orc):
    for delta in (1, 2, 4, 8, 16):
        for c in range(-100, 101):
            q = orc.quantise(c, delta)
            assert q == int(np.sign(c)) * (abs(c) // delta)
            r = orc.dequantise(q, delta)
            if delta == 1:
                assert r == c
            elif abs(c) < delta:       # dead zone: twice as wide, reconstructed at 0
                assert q == 0 and r == 0
            else:                      # other bins: reconstructed at the midpoint
                assert abs(c - r) <= delta // 2
    # the reconstruction table for delta = 4: bins [4,8) -> 6, [8,12) -> 10
    assert [orc.dequantise(q, 4) for q in (-2, -1, 0, 1, 2)] == [-10, -6, 0, 6, 10]


def test_coefficient_range_bound_int16(orc, synth):
    """The GPU keeps coefficients of <= 12-bit input in int16: check the
    worst-case gain (L1 norms of the iterated 5/3 filters) leaves room."""
    h = np.array([-1, 2, 6, 2, -1]) / 8.0
    g = np.array([-1, 2, -1]) / 2.0
    cur = np.array([1.0])
    worst = 0.0
    for j in range(1, 16):
        up = np.zeros(2 ** (j - 1) * 4 + 1); up[:: 2 ** (j - 1)] = h
        upg = np.zeros(2 ** (j - 1) * 2 + 1); upg[:: 2 ** (j - 1)] = g
        lo, hi = np.convolve(cur, up), np.convolve(cur, upg)
        l1l, l1h = np.abs(lo).sum(), np.abs(hi).sum()
        # zero-sum filters on [0, M] reach M * L1 / 2; the low-pass pair reaches M * (L1 + 1) / 2
        worst = max(worst, (l1h * l1h) / 2, (l1h * l1l) / 2, (l1l * l1l + 1) / 2)
        cur = lo
    assert worst * 4095 + 4096 < 32767          # 12-bit mono
    assert worst * 510 + 4096 < 32767           # RCT chroma spans 510
    # and the oracle agrees on an adversarial 12-bit checkerboard
    x = (np.indices((64, 64)).sum(0) % 2) * 4095
    y = orc.dwt2_forward(x, 6)
    assert np.abs(y).max() < 32767
