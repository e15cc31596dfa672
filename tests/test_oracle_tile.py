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
