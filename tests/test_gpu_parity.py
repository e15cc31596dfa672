"""GPU parity: the CUDA library, called through the C ABI, against the CPU
oracle.  Integer codec: streams must be byte-identical and decodes
bit-exact (no tolerance)."""
import numpy as np
import pytest

from gpu_helpers import explain_mismatch, gpu_decode_tile, gpu_encode, to_device, torch_cuda

pytestmark = pytest.mark.gpu

CONFIG3_Q = [3, 2, 1, 0, 0, 0, 0, 0, 0]   # steps 8/4/2 on levels 1-3, 1 elsewhere


@pytest.fixture(scope="module")
def codec():
    torch_cuda()
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


def assert_streams_equal(gpu_streams, refs, what):
    bad = [i for i, (g, r) in enumerate(zip(gpu_streams, refs)) if g != r]
    if bad:
        i = bad[0]
        pytest.fail(f"{what}: {len(bad)} of {len(refs)} tile streams differ; first tile {i}: "
                    f"{explain_mismatch(gpu_streams[i], refs[i])}")


def test_forward_coefficients_match_oracle(codec, orc, synth):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    imgs = [synth.stain(synth.config_seed(1), 64, 48), synth.phantom(5, 512, 512, 10, 20, 37, 29),
            synth.slide(synth.config_seed(3), 2560, 1792, 256, 256)]
    params = [(3, 8, ()), (4, 12, ()), (8, 8, CONFIG3_Q)]
    tiles, keep = [], []
    for img, (L, B, q) in zip(imgs, params):
        d = to_device(img)
        keep.append(d)
        tiles.append(isx.tile_from_tensor(d, L, B, q))
    total = sum((3 if a.ndim == 3 else 1) * a.shape[0] * a.shape[1] for a in imgs)
    out = torch.zeros(total, dtype=torch.int32, device="cuda")
    codec.forward_coefficients(tiles, out)
    assert codec.sync_status() == 0
    got = out.cpu().numpy()
    off = 0
    for img, (L, B, q) in zip(imgs, params):
        ref = orc.tile_coefficients(img, L, B, q)
        n = ref.size
        assert np.array_equal(got[off:off + n].reshape(ref.shape), ref)
        off += n


def test_tiny_images_every_size_and_level(codec, orc):
    rng = np.random.default_rng(31)
    imgs, levels, bits, refs = [], [], [], []
    for h in range(1, 10):
        for w in range(1, 10):
            for L in range(0, 5):
                rgb = rng.integers(0, 256, (h, w, 3)).astype(np.uint8)
                imgs.append(rgb); levels.append(L); bits.append(8)
    streams, _, _, _ = gpu_encode(codec, imgs, levels, bits)
    refs = [orc.encode_tile(a, L, 8) for a, L in zip(imgs, levels)]
    assert_streams_equal(streams, refs, "tiny RGB")
    imgs, levels = [], []
    for h in range(1, 10):
        for w in range(1, 10):
            for L in range(0, 5):
                imgs.append(rng.integers(0, 4096, (h, w)).astype(np.uint16)); levels.append(L)
    streams, _, _, _ = gpu_encode(codec, imgs, levels, 12)
    refs = [orc.encode_tile(a, L, 12) for a, L in zip(imgs, levels)]
    assert_streams_equal(streams, refs, "tiny mono12")


@pytest.mark.parametrize("bits", [1, 8, 12, 16])
def test_extreme_patterns(codec, orc, bits):
    hi = 2 ** bits - 1
    dt = np.uint8 if bits <= 8 else np.uint16
    h, w = 37, 70
    pats = [np.zeros((h, w), dt), np.full((h, w), hi, dt), ((np.indices((h, w)).sum(0) % 2) * hi).astype(dt),
            ((np.arange(w)[None, :].repeat(h, 0) % 3 == 0) * hi).astype(dt)]
    imgs, levels = [], []
    for p in pats:
        for L in (0, 1, 3, 6):
            imgs.append(p); levels.append(L)
    streams, _, _, _ = gpu_encode(codec, imgs, levels, bits)
    refs = [orc.encode_tile(a, L, bits) for a, L in zip(imgs, levels)]
    assert_streams_equal(streams, refs, f"extreme patterns {bits}-bit")


def test_config1_stain_tile(codec, orc, synth):
    img = synth.stain(synth.config_seed(1))
    streams, tiles, out, offs = gpu_encode(codec, [img], 3, 8)
    ref = orc.encode_tile(img, 3, 8)
    assert_streams_equal(streams, [ref], "512x512 RGB, 3 levels")
    for z in range(4):
        dec = gpu_decode_tile(codec, out, offs, tiles, 0, z)
        assert np.array_equal(dec, orc.decode_tile(ref, z)), z
    assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, 0, 0), img)


def test_config2_phantom(codec, orc, synth):
    img = synth.phantom(synth.config_seed(2), 2048, 2048)
    streams, tiles, out, offs = gpu_encode(codec, [img], 5, 12)
    ref = orc.encode_tile(img, 5, 12)
    assert_streams_equal(streams, [ref], "2048x2048 mono12, 5 levels")
    assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, 0, 0), img)
    assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, 0, 3), orc.decode_tile(ref, 3))


def slide_tiles(synth, n, seed_offset=0):
    rng = np.random.default_rng(40 + seed_offset)
    imgs, origins = [], []
    for k in range(n):
        if k % 8 == 7:   # edge tiles of the 40000 x 30000 image: 64 wide / 48 tall
            x0, y0 = 156 * 256, int(rng.integers(0, 117)) * 256
            w, h = 64, 256
            if k % 16 == 15:
                x0, y0, w, h = 156 * 256, 117 * 256, 64, 48
        else:
            x0, y0 = int(rng.integers(0, 156)) * 256, int(rng.integers(0, 117)) * 256
            w, h = 256, 256
        imgs.append(synth.slide(synth.config_seed(3), x0, y0, w, h))
        origins.append((x0, y0))
    return imgs, origins


@pytest.mark.parametrize("lossy", [False, True])
def test_config3_slide_tiles(codec, orc, synth, lossy):
    imgs, origins = slide_tiles(synth, 48, int(lossy))
    q = CONFIG3_Q if lossy else ()
    streams, tiles, out, offs = gpu_encode(codec, imgs, 8, 8, q, origins=[(i * 256, 0) for i in range(len(imgs))])
    refs = orc.encode_tiles_mt(imgs, [orc.tile_struct(a.shape[1], a.shape[0], 3, 8, 8, q) for a in imgs], 8)
    assert_streams_equal(streams, refs, f"256x256 slide tiles, 8 levels, {'lossy' if lossy else 'lossless'}")
    for i in (0, 7, 15):
        for z in (0, 2, 8):
            dec = gpu_decode_tile(codec, out, offs, tiles, i, z)
            assert np.array_equal(dec, orc.decode_tile(refs[i], z)), (i, z)


def test_config4_mixed_batch(codec, orc, synth):
    rng = np.random.default_rng(44)
    imgs, levels, bits, qs = [], [], [], []
    for k in range(160):
        w, h = int(rng.integers(17, 257)), int(rng.integers(17, 257))
        L = int(rng.integers(2, 7))
        if rng.random() < 0.5:
            img = synth.slide(synth.config_seed(3), int(rng.integers(0, 39000)), int(rng.integers(0, 29000)), w, h)
            b = 8
        else:
            img = synth.phantom(synth.config_seed(2), 2048, 2048, int(rng.integers(0, 2048 - w)), int(rng.integers(0, 2048 - h)), w, h)
            b = 12
        q = [3, 2, 1] + [0] * 13 if rng.random() < 0.5 else [0] * 16
        imgs.append(img); levels.append(L); bits.append(b); qs.append(q[:L + 1])
    streams, tiles, out, offs = gpu_encode(codec, imgs, levels, bits, qs)
    refs = [orc.encode_tile(a, L, b, q) for a, L, b, q in zip(imgs, levels, bits, qs)]
    assert_streams_equal(streams, refs, "mixed batch")
    for i in range(0, 160, 9):
        z = i % (levels[i] + 1)
        assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, i, z), orc.decode_tile(refs[i], z)), (i, z)


def test_lsb_drop_decode(codec, orc, synth):
    img = synth.slide(synth.config_seed(3), 3000, 4000, 256, 256)
    streams, tiles, out, offs = gpu_encode(codec, [img], 8, 8)
    for drop in (1, 3, 7):
        for z in (0, 1):
            dec = gpu_decode_tile(codec, out, offs, tiles, 0, z, drop)
            assert np.array_equal(dec, orc.decode_tile(streams[0], z, drop)), (drop, z)


def test_region_decode_mosaic(codec, orc, synth):
    torch = torch_cuda()
    # a 3 x 2 grid of 256-px tiles (last column 100 wide) decoded as one region
    x0, y0 = 5120, 7680
    imgs, origins = [], []
    for ty in range(2):
        for tx in range(3):
            w = 256 if tx < 2 else 100
            imgs.append(synth.slide(synth.config_seed(3), x0 + 256 * tx, y0 + 256 * ty, w, 256))
            origins.append((x0 + 256 * tx, y0 + 256 * ty))
    streams, tiles, out, offs = gpu_encode(codec, imgs, 8, 8, CONFIG3_Q, origins=origins)
    full = np.zeros((512, 612, 3), np.uint8)
    for k, (ox, oy) in enumerate(origins):
        d = orc.decode_tile(streams[k], 0)
        full[oy - y0:oy - y0 + d.shape[0], ox - x0:ox - x0 + d.shape[1]] = d
    rect = (x0 + 100, y0 + 50, 400, 300)
    res = torch.zeros((300, 400, 3), dtype=torch.uint8, device="cuda")
    codec.decode_region(out, offs, tiles, 0, rect, res)
    assert codec.sync_status() == 0
    assert np.array_equal(res.cpu().numpy(), full[50:350, 100:500])
    # level 1: each tile's level-1 image lands at origin >> 1
    z = 1
    full1 = np.zeros((256, 306, 3), np.uint8)
    for k, (ox, oy) in enumerate(origins):
        d = orc.decode_tile(streams[k], z)
        full1[(oy - y0) >> 1:((oy - y0) >> 1) + d.shape[0], (ox - x0) >> 1:((ox - x0) >> 1) + d.shape[1]] = d
    res1 = torch.zeros((256, 306, 3), dtype=torch.uint8, device="cuda")
    codec.decode_region(out, offs, tiles, z, (x0 >> 1, y0 >> 1, 306, 256), res1)
    assert codec.sync_status() == 0
    assert np.array_equal(res1.cpu().numpy(), full1)


def test_capacity_error_reports_required_size(codec, orc, synth):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    img = synth.stain(synth.config_seed(1), 128, 128)
    d = to_device(img)
    tiles = [isx.tile_from_tensor(d, 3, 8)]
    out = torch.zeros(100, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    codec.encode_tiles(tiles, out, offs)
    assert codec.sync_status() == isx.ISX_ERR_CAPACITY
    need = int(offs[1].item())
    assert need >= len(orc.encode_tile(img, 3, 8))
    out2 = torch.zeros(need, dtype=torch.uint8, device="cuda")
    codec.encode_tiles(tiles, out2, offs)
    assert codec.sync_status() == 0
    assert out2[: int(offs[1].item())].cpu().numpy().tobytes() == orc.encode_tile(img, 3, 8)


@pytest.mark.parametrize("shape,bits,dtype", [((96, 80, 3), 4, np.uint8), ((64, 64), 6, np.uint8),
                                               ((128, 96), 12, np.uint16), ((1100, 40), 10, np.uint16)])
def test_samples_above_bit_depth_are_reported(codec, orc, synth, shape, bits, dtype):
    """Samples at or above 2^bits are an input error: the encode reports it (and stays within its
    buffers) on the fused shared-memory path and on the global path (the 1100-wide tile)."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    rng = np.random.default_rng(5)
    img = rng.integers(0, np.iinfo(dtype).max, size=shape, endpoint=True).astype(dtype)
    d = to_device(img)
    tiles = [isx.tile_from_tensor(d, 3, bits)]
    out = torch.zeros(img.nbytes * 4 + 4096, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    codec.encode_tiles(tiles, out, offs)
    assert codec.sync_status() == isx.ISX_ERR_ARG
    # the same tile within range encodes exactly afterwards
    ok = (img >> (img.dtype.itemsize * 8 - bits)).astype(dtype)
    d2 = to_device(ok)
    codec.encode_tiles([isx.tile_from_tensor(d2, 3, bits)], out, offs)
    assert codec.sync_status() == 0
    assert out[: int(offs[1].item())].cpu().numpy().tobytes() == orc.encode_tile(ok, 3, bits)


def test_channel_and_transform_argument_errors(codec):
    """Descriptors outside the documented ranges (more than 16 channels, a colour transform on fewer
    than 3 channels, an unknown transform) are refused before anything is enqueued, by encode and decode."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    out = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(2, dtype=torch.int64, device="cuda")
    for C, ct, msg in ((17, isx.CT_DEFAULT, "channels"), (2, isx.CT_RCT, "3 or more"), (1, isx.CT_YCOCG_R, "3 or more"),
                       (3, 4, "transform")):
        d = torch.zeros((16, 24, C), dtype=torch.uint8, device="cuda")
        t = isx.tile_from_tensor(d, 2, 8, transform=ct)
        with pytest.raises(isx.IsxError) as ei:
            codec.encode_tiles([t], out, offs)
        assert ei.value.status == isx.ISX_ERR_ARG and msg in str(ei.value)
        with pytest.raises(isx.IsxError) as ei:
            codec.decode_region(out, offs, [t], 0, (0, 0, 24, 16), d)
        assert ei.value.status == isx.ISX_ERR_ARG and msg in str(ei.value)
    assert codec.sync_status() == 0


def test_corrupt_stream_is_reported(codec, synth):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    img = synth.stain(synth.config_seed(1), 128, 128)
    streams, tiles, out, offs = gpu_encode(codec, [img], 3, 8)
    n = int(offs[1].item())
    bad = out.clone()
    bad[40:n] = bad[40:n] ^ 0x5A                    # scramble block data
    res = torch.zeros((128, 128, 3), dtype=torch.uint8, device="cuda")
    codec.decode_region(bad, offs, tiles, 0, (0, 0, 128, 128), res)
    assert codec.sync_status() == isx.ISX_ERR_CORRUPT
    bad2 = out.clone()
    bad2[0] = ord("J")                              # broken magic
    codec.decode_region(bad2, offs, tiles, 0, (0, 0, 128, 128), res)
    assert codec.sync_status() == isx.ISX_ERR_CORRUPT
    # the context stays usable
    codec.decode_region(out, offs, tiles, 0, (0, 0, 128, 128), res)
    assert codec.sync_status() == 0
    assert np.array_equal(res.cpu().numpy(), img)


def test_host_buffer_entry_points(codec, orc, synth):
    from paper_2005_08713_gb300 import isx
    img = np.ascontiguousarray(synth.slide(synth.config_seed(3), 0, 0, 700, 520))
    tiles = []
    for ty in range(0, 520, 256):
        for tx in range(0, 700, 256):
            v = img[ty:ty + 256, tx:tx + 256]
            tiles.append(isx.tile_from_array(v, 8, 8, CONFIG3_Q, tx, ty))
    out = np.zeros(img.nbytes * 2, np.uint8)
    offs = np.zeros(len(tiles) + 1, np.uint64)
    codec.encode_tiles_host(tiles, out, offs)
    for k, t in enumerate(tiles):
        v = img[t.y0:t.y0 + t.height, t.x0:t.x0 + t.width]
        assert out[offs[k]:offs[k + 1]].tobytes() == orc.encode_tile(v, 8, 8, CONFIG3_Q), k
    res = np.zeros((520, 700, 3), np.uint8)
    codec.decode_region_host(out, offs, tiles, 0, (0, 0, 700, 520), res)
    ref = np.zeros_like(res)
    for k, t in enumerate(tiles):
        d = orc.decode_tile(out[offs[k]:offs[k + 1]].tobytes(), 0)
        ref[t.y0:t.y0 + d.shape[0], t.x0:t.x0 + d.shape[1]] = d
    assert np.array_equal(res, ref)


def test_repeated_encodes_are_identical(codec, orc, synth):
    """Intermittent races show up as run-to-run differences: encode one batch
    several times and require the oracle's bytes every time."""
    imgs, origins = slide_tiles(synth, 40, 5)
    refs = orc.encode_tiles_mt(imgs, [orc.tile_struct(a.shape[1], a.shape[0], 3, 8, 8, CONFIG3_Q) for a in imgs], 8)
    for rep in range(6):
        streams, _, _, _ = gpu_encode(codec, imgs, 8, 8, CONFIG3_Q, origins=[(i * 256, 0) for i in range(len(imgs))])
        assert_streams_equal(streams, refs, f"repeat {rep}")


def _longest_code_bits(stream: bytes, w: int, h: int, channels: int, levels: int) -> int:
    """Longest Huffman code of any block of a tile stream, read with the independent block parser
    (block order: per channel the LL band, then levels L .. 1, 128 x 128 cells in raster order)."""
    from blockparse import parse_block
    from gpu_helpers import split_blocks

    def ld(n, l):
        return -(-n // (1 << l))

    _, blocks = split_blocks(stream)
    geo = []
    for _c in range(channels):
        for p, l in [(1, levels)] + [(3, l) for l in range(levels, 0, -1)]:
            gw, gh = ld(w, l), ld(h, l)
            for cy in range(0, gh, 128):
                for cx in range(0, gw, 128):
                    geo.append((p, -(-min(128, gw - cx) // 4) * 4, -(-min(128, gh - cy) // 4) * 4))
    assert len(geo) == len(blocks)
    best = 0
    for data, (p, bw, bh) in zip(blocks, geo):
        pb = parse_block(data, p, bw, bh)
        if pb.get("codes"):
            best = max(best, max(len(k) for k in pb["codes"]))
    return best


def test_codes_longer_than_the_lookup_table(codec, orc):
    # 12-bit samples with a geometric value distribution: skewed symbol counts
    # give some blocks codes of 10-11 bits, which the segment decoder resolves
    # by walking the tree past its 9-bit lookup table
    rng = np.random.default_rng(2024)
    imgs = []
    for k in range(3):
        g = rng.geometric(0.35, size=(128, 128)) - 1
        imgs.append(np.minimum(g * (1 + k), 4095).astype(np.uint16))
    refs = [orc.encode_tile(a, 1, 12) for a in imgs]
    assert max(_longest_code_bits(r, 128, 128, 1, 1) for r in refs) > 9, "inputs no longer produce long codes"
    streams, tiles, out, offs = gpu_encode(codec, imgs, 1, 12)
    assert_streams_equal(streams, refs, "long-code tiles")
    for i, a in enumerate(imgs):
        assert np.array_equal(gpu_decode_tile(codec, out, offs, tiles, i), a), i
