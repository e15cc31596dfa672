"""GPU parity of the channel counts and colour transforms (Sec. 3: "an
arbitrary number of channels and an arbitrary bitdepth"; Fig. 1's optional
colour transform, here the RCT or YCoCg-R on channels 0..2) against the
oracle: RGB slide crops at 9..16 bits, 2-, 4- and 5-channel tiles, tiles of
different channel counts in one call, region decodes and the host-buffer
and no-allocation entry points.  Streams byte-identical, decodes
bit-exact; each test names the inverse path (fused int16 or global int32)
that its tiles take."""
import numpy as np
import pytest

from gpu_helpers import gpu_decode_tile, gpu_encode, to_device, torch_cuda
from test_gpu_parity import assert_streams_equal

pytestmark = pytest.mark.gpu

Q5 = (3, 2, 1, 0, 0, 0)


@pytest.fixture(scope="module")
def codec():
    torch_cuda()
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


def deep_slide(synth, x0, y0, w, h, bits, seed):
    """An RGB slide crop at `bits` bits: the 8-bit generator's samples shifted up, the new low bits
    filled from a seeded generator (texture finer than the 8-bit quantisation)."""
    img = synth.slide(synth.config_seed(3), x0, y0, w, h).astype(np.uint32)
    rng = np.random.default_rng(seed)
    low = rng.integers(0, 1 << (bits - 8), img.shape, dtype=np.uint32) if bits > 8 else 0
    return ((img << (bits - 8)) | low).astype(np.uint16 if bits > 8 else np.uint8)


def check(codec, orc, imgs, L, bits, q, transform, levels_to_check=(0, 2), drops=(0,)):
    from paper_2005_08713_gb300 import isx
    streams, tiles, out, offs = gpu_encode(codec, imgs, L, bits, list(q), transforms=transform)
    refs = [orc.encode_tile(a, L, bits, q, transform=transform) for a in imgs]
    assert_streams_equal(streams, refs, f"{imgs[0].shape} {bits}-bit transform {transform} q={q}")
    paths = set()
    for i, ref in enumerate(refs):
        for z in levels_to_check:
            for drop in drops:
                paths.add(isx.decode_path(tiles[i], z, drop)[0])
                dec = gpu_decode_tile(codec, out, offs, tiles, i, z, drop)
                assert np.array_equal(dec, orc.decode_tile(ref, z, drop)), (i, z, drop)
    return paths


@pytest.mark.parametrize("bits", [9, 10, 11, 12, 16])
@pytest.mark.parametrize("transform", [2, 3])
def test_rgb_above_8_bits_slide_crops(codec, orc, synth, bits, transform):
    """256 x 256 crops take the fused int16 path up to 11 bits (the colour transform doubles the chroma
    range) and the global int32 path from 12 bits; 600 x 300 crops the global path at level 0."""
    for q in ((), Q5):
        small = [deep_slide(synth, 4096 + 256 * k, 6144, 256, 256, bits, k) for k in range(3)]
        paths = check(codec, orc, small, 5, bits, q, transform)
        assert paths == ({1} if bits <= 11 else {0}), (bits, paths)
        big = [deep_slide(synth, 9000, 5000, 600, 300, bits, 7)]
        paths = check(codec, orc, big, 5, bits, q, transform, drops=(0, 2))
        assert 0 in paths and (bits >= 12) == (paths == {0}), (bits, paths)   # level 2 (150 x 75) fits the fused plane


@pytest.mark.parametrize("C,transform,bits", [(4, 3, 8), (4, 2, 8), (4, 1, 12), (2, 0, 8), (2, 0, 12), (5, 3, 11),
                                              (16, 1, 8)])
def test_multichannel_tiles(codec, orc, synth, C, transform, bits):
    rng = np.random.default_rng(C * 31 + bits)
    hi = (1 << bits) - 1
    dt = np.uint8 if bits <= 8 else np.uint16
    shapes = [(256, 256), (97, 130), (40, 700)] if C < 16 else [(64, 96)]
    for (h, w) in shapes:
        base = deep_slide(synth, 2048, 3072, w, h, max(bits, 8), C).astype(np.int64)
        chans = [base[..., k % 3] for k in range(min(C, 3))]
        yy, xx = np.indices((h, w))
        while len(chans) < C:   # extra channels: a gradient and a noisy mask, like alpha or label planes
            k = len(chans)
            chans.append(((xx * (k + 3) + yy * 7) % (hi + 1)) if k % 2 else rng.integers(0, hi + 1, (h, w)))
        img = np.clip(np.stack(chans, -1), 0, hi).astype(dt)
        for q in ((), Q5):
            check(codec, orc, [img], 5, bits, q, transform)


def test_mixed_channel_counts_in_one_call(codec, orc, synth):
    """One encode of tiles with 1..5 channels and every transform: the fused size classes launch as many
    CTAs per tile as their largest channel count."""
    rng = np.random.default_rng(9)
    imgs, levels, bits, qs, cts = [], [], [], [], []
    for k in range(40):
        C = [1, 2, 3, 4, 5][k % 5]
        b = [8, 12][k % 2] if C != 3 else [8, 9, 11][k % 3]
        ct = 0 if C < 3 else [1, 2, 3][k % 3]
        w, h = int(rng.integers(17, 257)), int(rng.integers(17, 257))
        img = rng.integers(0, 1 << b, (h, w, C) if C > 1 else (h, w)).astype(np.uint8 if b <= 8 else np.uint16)
        L = int(rng.integers(2, 7))
        q = list(Q5[:L]) + [0] if k % 3 else [0] * (L + 1)
        imgs.append(img); levels.append(L); bits.append(b); qs.append(q); cts.append(ct)
    streams, tiles, out, offs = gpu_encode(codec, imgs, levels, bits, qs, transforms=cts)
    refs = [orc.encode_tile(a, L, b, q, transform=ct) for a, L, b, q, ct in zip(imgs, levels, bits, qs, cts)]
    assert_streams_equal(streams, refs, "mixed channel counts")
    for i in range(0, 40, 3):
        z = i % (levels[i] + 1)
        assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, i, z), orc.decode_tile(refs[i], z)), (i, z)


def test_region_decode_of_a_four_channel_image(codec, orc, synth):
    torch = torch_cuda()
    rng = np.random.default_rng(12)
    H, W, T = 300, 520, 256
    img = np.concatenate([synth.slide(synth.config_seed(3), 1000, 2000, W, H),
                          rng.integers(0, 256, (H, W, 1)).astype(np.uint8)], -1)
    grid = [(x, y, min(T, W - x), min(T, H - y)) for y in range(0, H, T) for x in range(0, W, T)]
    imgs = [np.ascontiguousarray(img[y:y + h, x:x + w]) for (x, y, w, h) in grid]
    streams, tiles, out, offs = gpu_encode(codec, imgs, 4, 8, list(Q5[:4]) + [0], origins=[(x, y) for x, y, _, _ in grid],
                                           transforms=3)
    for z in (0, 1, 3):
        rx, ry, rw, rh = 37 >> z, 90 >> z, 400 >> z, 180 >> z
        res = torch.zeros((rh, rw, 4), dtype=torch.uint8, device="cuda")
        codec.decode_region(out, offs, tiles, z, (rx, ry, rw, rh), res)
        assert codec.sync_status() == 0
        ref = np.zeros((rh, rw, 4), np.uint8)
        for (x, y, w, h), s in zip(grid, streams):
            d = orc.decode_tile(s, z)
            tx, ty = x >> z, y >> z
            x0, y0 = max(tx, rx), max(ty, ry)
            x1, y1 = min(tx + d.shape[1], rx + rw), min(ty + d.shape[0], ry + rh)
            if x0 < x1 and y0 < y1:
                ref[y0 - ry:y1 - ry, x0 - rx:x1 - rx] = d[y0 - ty:y1 - ty, x0 - tx:x1 - tx]
        assert np.array_equal(res.cpu().numpy(), ref), z


def test_host_entry_points_and_static_encoder_with_channels(codec, orc, synth):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    img = deep_slide(synth, 3000, 3000, 200, 150, 12, 3)
    rgba = np.ascontiguousarray(np.concatenate([img, (img[..., :1] >> 1)], -1))
    ref = orc.encode_tile(rgba, 4, 12, Q5[:4] + (0,), transform=3)
    # host buffers in and out
    t = isx.tile_from_array(rgba, 4, 12, Q5[:4] + (0,), transform=3)
    h_out = np.zeros(rgba.nbytes * 2 + 4096, np.uint8)
    h_offs = np.zeros(2, np.uint64)
    codec.encode_tiles_host([t], h_out, h_offs)
    assert h_out[:int(h_offs[1])].tobytes() == ref
    dec = np.zeros_like(rgba)
    codec.decode_region_host(h_out, h_offs, [t], 0, (0, 0, 200, 150), dec)
    assert np.array_equal(dec, orc.decode_tile(ref, 0))
    # the no-allocation encoder gives the same bytes
    d = to_device(rgba)
    out = torch.zeros(rgba.nbytes * 2 + 4096, dtype=torch.uint8, device="cuda")
    n = isx.encode_tile_static(isx.tile_from_tensor(d, 4, 12, Q5[:4] + (0,), transform=3), out)
    assert out[:n].cpu().numpy().tobytes() == ref
