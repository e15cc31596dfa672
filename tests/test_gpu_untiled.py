"""Untiled images (whole-image transform) and windowed region decode, on the GPU
against the oracle.

The paper's product codes a whole slide with one wavelet transform, its
blocks partitioned in 128 x 128 cells of each band (Sec. 4), and decodes any
region at any level by reading only what the region depends on.  Here the
whole image is one tile (the int32 global path encodes it) and a region
decode of part of it runs windowed: only the blocks whose cells meet the
dependency windows of the 5/3 synthesis are decoded, and each inverse level
runs on a window with the halo its outputs need.  Streams must equal the
oracle's whole-image encode byte for byte; every windowed decode must equal
the matching crop of the oracle's whole-image decode at that level."""
import numpy as np
import pytest

from gpu_helpers import gpu_encode, torch_cuda
from test_gpu_parity import assert_streams_equal

pytestmark = pytest.mark.gpu

Q = (3, 2, 1, 0, 0, 0, 0, 0, 0)


@pytest.fixture(scope="module")
def codec():
    torch_cuda()
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


def windowed_decode(codec, out, offs, tiles, z, rect, drop=0):
    """Region decode of `rect` (level-z pixels) with stage timing on; returns (pixels, windowed path taken)."""
    torch = torch_cuda()
    t = tiles[0]
    rx, ry, rw, rh = rect
    dt = torch.uint8 if t.bits <= 8 else torch.int16
    res = torch.zeros((rh, rw, t.channels) if t.channels > 1 else (rh, rw), dtype=dt, device="cuda")
    codec.set_timing(True)
    try:
        codec.decode_region(out, offs, tiles, z, rect, res, drop)
        assert codec.sync_status() == 0
        stages = codec.stage_times()
    finally:
        codec.set_timing(False)
    a = res.cpu().numpy()
    return (a.view(np.uint16) if t.bits > 8 else a), "decode.inverse_window" in stages


def rects_for(zw, zh, rng, n):
    out = [(0, 0, min(zw, 37), min(zh, 23)), (zw - 1, zh - 1, 1, 1), (max(zw - 300, 0), 0, min(300, zw), min(77, zh)),
           (0, max(zh - 129, 0), min(zw, 129), min(zh, 129)), (zw // 3, zh // 3, max(1, zw // 3), max(1, zh // 4))]
    for _ in range(n):
        rw, rh = int(rng.integers(1, min(zw, 700) + 1)), int(rng.integers(1, min(zh, 500) + 1))
        out.append((int(rng.integers(0, zw - rw + 1)), int(rng.integers(0, zh - rh + 1)), rw, rh))
    return out


@pytest.mark.parametrize("lossy", [False, True])
def test_untiled_slide_crop_4096(codec, orc, synth, lossy):
    """A 4096 x 4096 RGB slide crop coded as one image with 8 levels: the stream equals the oracle's, and
    region decodes at levels 0, 1, 3 and 8 equal crops of the oracle's whole-image decode."""
    img = synth.slide(synth.config_seed(3), 12000, 9000, 4096, 4096)
    q = Q if lossy else ()
    streams, tiles, out, offs = gpu_encode(codec, [img], 8, 8, list(q))
    ref = orc.encode_tile(img, 8, 8, q)
    assert_streams_equal(streams, [ref], f"untiled 4096x4096 {'lossy' if lossy else 'lossless'}")
    rng = np.random.default_rng(8 + int(lossy))
    for z in (0, 1, 3, 8):
        full = orc.decode_tile(ref, z)
        zh, zw = full.shape[:2]
        for rect in rects_for(zw, zh, rng, 4):
            rx, ry, rw, rh = rect
            got, windowed = windowed_decode(codec, out, offs, tiles, z, rect)
            assert windowed == (rw < zw or rh < zh) or z == 8, (z, rect)
            assert np.array_equal(got, full[ry:ry + rh, rx:rx + rw]), (z, rect)


@pytest.mark.parametrize("bits,channels,transform", [(12, 1, 0), (8, 3, 3), (11, 4, 2)])
def test_untiled_odd_sizes_every_level(codec, orc, synth, bits, channels, transform):
    """Odd-sized untiled images (1500 x 1103) at every level, random windows, lossless and lossy, with
    dropped planes: the windows' halos and the symmetric extension at the image's edges."""
    rng = np.random.default_rng(bits * 10 + channels)
    h, w, L = 1103, 1500, 6
    if channels == 1:
        img = synth.phantom(synth.config_seed(2), 2048, 2048, 200, 300, w, h)
    else:
        base = synth.slide(synth.config_seed(3), 20000, 15000, w, h).astype(np.uint32)
        base = (base << (bits - 8)) | rng.integers(0, 1 << (bits - 8), base.shape, dtype=np.uint32) if bits > 8 else base
        extra = [((np.indices((h, w)).sum(0) * 7) % (1 << bits))[..., None]] * (channels - 3)
        img = np.concatenate([base] + extra, -1) if extra else base
        img = img.astype(np.uint8 if bits <= 8 else np.uint16)
    for q in ((), Q[:L] + (0,)):
        streams, tiles, out, offs = gpu_encode(codec, [img], L, bits, list(q), transforms=transform)
        ref = orc.encode_tile(img, L, bits, q, transform=transform)
        assert_streams_equal(streams, [ref], f"untiled {w}x{h} {bits}-bit C={channels}")
        for z in range(L + 1):
            for drop in ((0, 2) if z in (0, 2) else (0,)):
                full = orc.decode_tile(ref, z, drop)
                zh, zw = full.shape[:2]
                for rect in rects_for(zw, zh, rng, 3):
                    rx, ry, rw, rh = rect
                    got, _ = windowed_decode(codec, out, offs, tiles, z, rect, drop)
                    assert np.array_equal(got, full[ry:ry + rh, rx:rx + rw]), (q, z, drop, rect)


def test_windowed_and_whole_tiles_in_one_call(codec, orc, synth):
    """decode_jobs mixing a windowed job of a large image and whole-tile jobs of small tiles."""
    torch = torch_cuda()
    big = synth.slide(synth.config_seed(3), 3000, 3000, 2000, 1300)
    small = [synth.slide(synth.config_seed(3), 100 * k, 7000, 200, 150) for k in range(3)]
    imgs = [big] + small
    streams, tiles, out, offs = gpu_encode(codec, imgs, 5, 8, list(Q[:5]) + [0])
    refs = [orc.encode_tile(a, 5, 8, Q[:5] + (0,)) for a in imgs]
    assert_streams_equal(streams, refs, "mixed windowed batch")
    z = 1
    win = (317, 211, 400, 250)
    dst_big = torch.zeros((250, 400, 3), dtype=torch.uint8, device="cuda")
    dst_small = [torch.zeros((75, 100, 3), dtype=torch.uint8, device="cuda") for _ in small]
    jobs = [(0, (tiles[0].x0 // 2 + win[0], win[1], win[2], win[3]), dst_big)]
    jobs += [(i + 1, (tiles[i + 1].x0 // 2, 0, 100, 75), d) for i, d in enumerate(dst_small)]
    codec.decode_jobs(out, offs, tiles, jobs, z)
    assert codec.sync_status() == 0
    full = orc.decode_tile(refs[0], z)
    assert np.array_equal(dst_big.cpu().numpy(), full[win[1]:win[1] + win[3], win[0]:win[0] + win[2]])
    for i, d in enumerate(dst_small):
        assert np.array_equal(d.cpu().numpy(), orc.decode_tile(refs[i + 1], z))
