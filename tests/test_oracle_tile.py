"""Pins of the oracle's tile codec: lossless identity (the premise of the
paper's lossless mode, Sec. 5), tiny images of every size and level count,
resolution-progressive decode (Sec. 4: discard the finer high-pass blocks)
and the lossy quantiser bound.
"""
import numpy as np
import pytest


def _levels_dims(n, z):
    for _ in range(z):
        n = (n + 1) // 2
    return n


def test_tiny_images_all_sizes_levels_lossless(orc):
    rng = np.random.default_rng(21)
    for h in range(1, 10):
        for w in range(1, 10):
            for L in range(0, 5):
                rgb = rng.integers(0, 256, (h, w, 3)).astype(np.uint8)
                s = orc.encode_tile(rgb, L, 8)
                assert np.array_equal(orc.decode_tile(s), rgb)
                mono = rng.integers(0, 4096, (h, w)).astype(np.uint16)
                s = orc.encode_tile(mono, L, 12)
                assert np.array_equal(orc.decode_tile(s), mono)


@pytest.mark.parametrize("bits", [1, 2, 7, 8, 9, 12, 16])
def test_extreme_values_every_bit_depth(orc, bits):
    hi = 2 ** bits - 1
    dt = np.uint8 if bits <= 8 else np.uint16
    for pat in ("zeros", "max", "checker", "stripes"):
        h, w = 21, 34
        if pat == "zeros":
            img = np.zeros((h, w), dt)
        elif pat == "max":
            img = np.full((h, w), hi, dt)
        elif pat == "checker":
            img = ((np.indices((h, w)).sum(0) % 2) * hi).astype(dt)
        else:
            img = ((np.arange(w)[None, :].repeat(h, 0) % 3 == 0) * hi).astype(dt)
        for L in (0, 1, 3, 6):
            s = orc.encode_tile(img, L, bits)
            assert np.array_equal(orc.decode_tile(s), img)


def test_config1_stain_tile_lossless(orc, synth):
    img = synth.stain(synth.config_seed(1))
    s = orc.encode_tile(img, 3, 8)
    assert np.array_equal(orc.decode_tile(s), img)
    assert len(s) < img.nbytes          # it compresses


def test_config2_phantom_crop_lossless(orc, synth):
    img = synth.phantom(synth.config_seed(2), 2048, 2048, 700, 900, 300, 260)
    assert img.max() <= 4095
    s = orc.encode_tile(img, 5, 12)
    assert np.array_equal(orc.decode_tile(s), img)


def test_resolution_progressive_decode_is_the_ll(orc, synth):
    img = synth.slide(synth.config_seed(3), 256 * 40, 256 * 30, 256, 200)
    L = 8
    s = orc.encode_tile(img, L, 8)
    ycc = orc.rct_forward(img.astype(np.int64).reshape(-1, 3)).reshape(img.shape)
    for z in range(0, L + 1):
        dec = orc.decode_tile(s, z)
        zh, zw = _levels_dims(200, z), _levels_dims(256, z)
        assert dec.shape == (zh, zw, 3)
        # LL_z of a z-level transform of each colour plane, back through the RCT
        ll = np.stack([orc.dwt2_forward(ycc[:, :, c], z)[:zh, :zw] for c in range(3)], -1)
        ref = np.clip(orc.rct_inverse(ll.reshape(-1, 3)).reshape(ll.shape), 0, 255)
        assert np.array_equal(dec, ref.astype(np.uint8)), z


def test_lossy_coefficients_within_quantiser_bound(orc, synth):
    img = synth.slide(synth.config_seed(3), 256 * 80, 256 * 60, 256, 256)
    q = [3, 2, 1, 0, 0, 0, 0, 0, 0]
    exact = orc.tile_coefficients(img, 8, 8)
    quant = orc.tile_coefficients(img, 8, 8, q)
    # level 1 (step 8) occupies the outer three quadrants
    hp1 = np.zeros((256, 256), bool)
    hp1[128:, :] = True
    hp1[:, 128:] = True
    assert np.array_equal(np.abs(quant[:, hp1]), np.abs(exact[:, hp1]) // 8)
    s = orc.encode_tile(img, 8, 8, q)
    dec = orc.decode_tile(s)
    err = np.abs(dec.astype(int) - img.astype(int))
    assert err.max() <= 40 and err.mean() < 4
    assert len(s) < len(orc.encode_tile(img, 8, 8))


def test_edge_tile_with_degenerate_levels(orc, synth):
    # 64 x 48 edge tile with 8 levels: levels 7-8 act on 1-pixel dimensions
    img = synth.slide(synth.config_seed(3), 39936, 29952, 64, 48)
    s = orc.encode_tile(img, 8, 8, [3, 2, 1, 0, 0, 0, 0, 0, 0])
    dec = orc.decode_tile(s, 8)
    assert dec.shape == (1, 1, 3)
    s = orc.encode_tile(img, 8, 8)
    assert np.array_equal(orc.decode_tile(s), img)


def test_multithreaded_encode_is_identical(orc, synth):
    imgs = [synth.slide(synth.config_seed(3), 256 * i, 256 * 7, 256, 256) for i in range(6)]
    tiles = [orc.tile_struct(256, 256, 3, 8, 8) for _ in imgs]
    mt = orc.encode_tiles_mt(imgs, tiles, 4)
    for a, s in zip(imgs, mt):
        assert s == orc.encode_tile(a, 8, 8)


def test_corrupt_tile_stream_is_an_error(orc, synth):
    img = synth.stain(synth.config_seed(1), 64, 64)
    s = bytearray(orc.encode_tile(img, 3, 8))
    with pytest.raises(ValueError):
        orc.decode_tile(bytes(s[: len(s) - 40]))
    bad = bytearray(s)
    bad[0] = ord("J")
    with pytest.raises(ValueError):
        orc.decode_tile(bytes(bad))


def _expected_bands(orc, img, levels, q):
    """Per channel, the quantised subbands of the tile built from the pinned steps: the colour transform,
    the 2-D transform in Mallat layout (LL top-left; per level HL top-right = high horizontally, LH
    bottom-left, HH bottom-right), then each band quantised with its own step: 2^q[l-1] for the bands
    of level l (l = 1 finest), 2^q[levels] for the LL band."""
    planes = orc.rct_forward(img.astype(np.int64)) if img.ndim == 3 else img.astype(np.int64)[..., None]
    h, w = img.shape[:2]
    quant = np.vectorize(orc.quantise)
    out = []
    for c in range(planes.shape[2]):
        M = orc.dwt2_forward(planes[..., c], levels)
        bands = {}
        for l in range(1, levels + 1):
            pw, ph = _levels_dims(w, l - 1), _levels_dims(h, l - 1)
            lw, lh = (pw + 1) // 2, (ph + 1) // 2
            delta = 1 << q[l - 1]
            bands[(l, 0)] = quant(M[:lh, lw:pw], delta)     # HL
            bands[(l, 1)] = quant(M[lh:ph, :lw], delta)     # LH
            bands[(l, 2)] = quant(M[lh:ph, lw:pw], delta)   # HH
        bands[(0, 0)] = quant(M[:_levels_dims(h, levels), :_levels_dims(w, levels)], 1 << q[levels])
        out.append(bands)
    return out


@pytest.mark.parametrize("shape,levels,bits,q", [((136, 200, 3), 3, 8, [1, 2, 3, 2]),
                                                 ((300, 260), 2, 12, [0, 1, 3]),
                                                 ((70, 45, 3), 4, 8, [0, 0, 0, 0, 0])])
def test_tile_stream_layout(orc, synth, shape, levels, bits, q):
    """The tile container as documented: header fields, then per channel the LL blocks and the high-pass
    blocks of levels L .. 1, each band cut into 128 x 128 cells in raster order; a high-pass block
    multiplexes HL, LH and HH (Fig. 3) in that order, each band quantised with its own level's step."""
    if len(shape) == 3:
        img = synth.slide(synth.config_seed(3), 7000, 9000, shape[1], shape[0])
    else:
        img = synth.phantom(synth.config_seed(2), 2048, 2048, 900, 700, shape[1], shape[0])
    h, w = img.shape[:2]
    C = 1 if img.ndim == 2 else 3
    s = orc.encode_tile(img, levels, bits, q)
    assert s[:4] == b"ISX1"
    hdr = np.frombuffer(s[4:12], np.uint8)
    assert int.from_bytes(s[4:6], "little") == w and int.from_bytes(s[6:8], "little") == h
    assert list(hdr[4:8]) == [C, bits, levels, 1 if C == 3 else 0]
    nb = int.from_bytes(s[12:16], "little")
    assert list(s[16:16 + levels + 1]) == list(q)
    ends = [int.from_bytes(s[32 + 4 * i:36 + 4 * i], "little") for i in range(nb)]
    data = s[32 + 4 * nb:]
    assert ends == sorted(ends) and ends[-1] == len(data)
    bands = _expected_bands(orc, img, levels, q)
    k = 0
    for c in range(C):
        for l in [0] + list(range(levels, 0, -1)):
            gw, gh = _levels_dims(w, levels if l == 0 else l), _levels_dims(h, levels if l == 0 else l)
            types = [(0, 0)] if l == 0 else [(l, 0), (l, 1), (l, 2)]
            for by in range(0, gh, 128):
                for bx in range(0, gw, 128):
                    bw, bh = -(-min(128, gw - bx) // 4) * 4, -(-min(128, gh - by) // 4) * 4
                    want = np.zeros((len(types), bh, bw), np.int64)
                    for t, key in enumerate(types):
                        part = bands[c][key][by:by + bh, bx:bx + bw]
                        want[t, :part.shape[0], :part.shape[1]] = part
                    blk = data[(ends[k - 1] if k else 0):ends[k]]
                    got = orc.decode_block(blk, len(types), bw, bh)
                    assert np.array_equal(got, want), (c, l, by, bx)
                    k += 1
    assert k == nb
