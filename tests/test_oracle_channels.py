"""Pins of the oracle's colour transforms and channel counts (CPU).

Sec. 3 of the paper allows "an arbitrary number of channels and an arbitrary
bitdepth" and names the colour transform of Fig. 1 optional.  The oracle
offers no transform, the JPEG 2000 RCT and YCoCg-R (Malvar and Sullivan,
2003) on channels 0..2 of tiles of three or more channels; further channels
are coded as they are.  Pins: exhaustive round trips, the published linear
YCoCg matrix, the stored transform id, lossless identity at 1..16 channels
and 1..16 bits, and the resolution-progressive decode of a 4-channel
YCoCg-R tile equal to the inverse transform of the level-z LL bands."""
import numpy as np
import pytest


def _levels_dims(n, z):
    for _ in range(z):
        n = (n + 1) // 2
    return n


def test_ycocg_exhaustive_roundtrip_and_ranges(orc):
    # all 2^24 RGB8 triples in chunks: exact inverse, Y in [0, 255], Co and Cg in [-255, 255]
    for hi in range(0, 256, 16):
        r, g, b = np.meshgrid(np.arange(hi, hi + 16), np.arange(256), np.arange(256), indexing="ij")
        rgb = np.stack([r.ravel(), g.ravel(), b.ravel()], 1).astype(np.int64)
        ycc = orc.ycocg_forward(rgb)
        assert ycc[:, 0].min() >= 0 and ycc[:, 0].max() <= 255
        assert ycc[:, 1:].min() >= -255 and ycc[:, 1:].max() <= 255
        assert np.array_equal(orc.ycocg_inverse(ycc), rgb)


def test_ycocg_against_the_linear_ycocg_matrix(orc):
    """YCoCg-R is the lifting form of Y = R/4 + G/2 + B/4, Co = R/2 - B/2, Cg = -R/4 + G/2 - B/4 with both
    chroma channels doubled: Co is exact, Cg and Y are off by less than one from the rational values."""
    rng = np.random.default_rng(3)
    for bits in (8, 12, 16):
        rgb = rng.integers(0, 1 << bits, (200000, 3)).astype(np.int64)
        ycc = orc.ycocg_forward(rgb)
        R, G, B = (rgb[:, k].astype(float) for k in range(3))
        assert np.array_equal(ycc[:, 1], rgb[:, 0] - rgb[:, 2])
        dcg = ycc[:, 2] - 2 * (-R / 4 + G / 2 - B / 4)
        assert dcg.min() >= 0 and dcg.max() <= 0.5
        dy = ycc[:, 0] - (R / 4 + G / 2 + B / 4)
        assert dy.min() > -1 and dy.max() <= 0
        assert np.array_equal(orc.ycocg_inverse(ycc), rgb)
    for v in (0, 1, 77, 4095, 65535):   # grey maps to (v, 0, 0)
        assert orc.ycocg_forward(np.array([[v, v, v]])).tolist() == [[v, 0, 0]]


def test_ycocg_and_rct_differ(orc):
    # the two transforms are distinct readings of "colorspace transformation": same luma for grey only
    rgb = np.array([[255, 0, 0], [0, 255, 0], [10, 20, 30]], np.int64)
    assert not np.array_equal(orc.ycocg_forward(rgb), orc.rct_forward(rgb))


@pytest.mark.parametrize("transform,ct_id", [(0, 1), (1, 0), (2, 1), (3, 2)])
def test_stored_transform_id(orc, transform, ct_id):
    rng = np.random.default_rng(transform)
    img = rng.integers(0, 256, (20, 30, 3)).astype(np.uint8)
    s = orc.encode_tile(img, 2, 8, transform=transform)
    assert s[11] == ct_id and s[8] == 3
    assert np.array_equal(orc.decode_tile(s), img)


def test_transform_needs_three_channels(orc):
    img = np.zeros((8, 8, 2), np.uint8)
    with pytest.raises(ValueError):
        orc.encode_tile(img, 1, 8, transform=2)
    with pytest.raises(ValueError):
        orc.encode_tile(np.zeros((8, 8, 17), np.uint8), 1, 8)


@pytest.mark.parametrize("C", [2, 4, 5, 16])
@pytest.mark.parametrize("bits", [8, 12, 16])
def test_multichannel_lossless(orc, C, bits):
    rng = np.random.default_rng(C * 100 + bits)
    dt = np.uint8 if bits <= 8 else np.uint16
    img = rng.integers(0, 1 << bits, (23, 37, C)).astype(dt)
    for transform in ((1, 2, 3) if C >= 3 else (0, 1)):
        s = orc.encode_tile(img, 3, bits, transform=transform)
        assert s[8] == C
        assert np.array_equal(orc.decode_tile(s), img), (C, bits, transform)


@pytest.mark.parametrize("bits", [9, 11, 12, 16])
@pytest.mark.parametrize("transform", [2, 3])
def test_rgb_high_bit_depth_lossless_extremes(orc, bits, transform):
    hi = (1 << bits) - 1
    h, w = 33, 40
    yy, xx = np.indices((h, w))
    pats = [((yy + xx) % 2) * hi, (xx % 2) * hi, ((yy // 3) % 2) * hi]
    img = np.stack([pats[0], pats[1], hi - pats[2]], -1).astype(np.uint16)
    for L in (0, 2, 6):
        s = orc.encode_tile(img, L, bits, transform=transform)
        assert np.array_equal(orc.decode_tile(s), img)


def test_progressive_decode_of_a_four_channel_ycocg_tile(orc, synth):
    base = synth.slide(synth.config_seed(3), 5000, 7000, 120, 90).astype(np.int64)
    alpha = (np.indices((90, 120)).sum(0) * 3 % 256)[..., None]
    img = np.concatenate([base, alpha], -1).astype(np.uint8)
    L = 4
    s = orc.encode_tile(img, L, 8, transform=3)
    planes = np.concatenate([orc.ycocg_forward(base.reshape(-1, 3)).reshape(base.shape), alpha], -1)
    for z in range(L + 1):
        zh, zw = _levels_dims(90, z), _levels_dims(120, z)
        ll = np.stack([orc.dwt2_forward(planes[:, :, c], z)[:zh, :zw] for c in range(4)], -1)
        rgb = orc.ycocg_inverse(ll[..., :3].reshape(-1, 3)).reshape(zh, zw, 3)
        ref = np.clip(np.concatenate([rgb, ll[..., 3:]], -1), 0, 255).astype(np.uint8)
        assert np.array_equal(orc.decode_tile(s, z), ref), z
