"""GPU parity of lossy coding on both inverse transforms, against the oracle.

Quantisation (Sec. 3, the dead-zone quantiser of JPEG 2000, reconstructed
at the bin midpoint) runs in four places: the fused shared-memory forward
and inverse transforms (int16 planes) and the global transform path (int32
planes in HBM: planes over 160 KB, a side over 1024 or more than 12 bits).
These tests encode lossy tiles that take each path and compare the streams
byte for byte and the decodes (levels 0 and z > 0, with and without dropped
planes) pixel for pixel with the oracle.  The extreme-pattern test drives
the fused inverse with the largest steps its int16 bound admits
(isx_decode_path) and the global inverse with larger ones."""
import numpy as np
import pytest

from gpu_helpers import gpu_decode_tile, gpu_encode, to_device, torch_cuda
from test_gpu_parity import assert_streams_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    torch_cuda()
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


def decode_uses_global_inverse(codec, out, offs, tiles, index, level, drop=0):
    """Decode tile `index` with stage timing on; returns (pixels, whether the global inverse ran)."""
    codec.set_timing(True)
    try:
        dec = gpu_decode_tile(codec, out, offs, tiles, index, level, drop)
        stages = codec.stage_times()
    finally:
        codec.set_timing(False)
    return dec, "decode.inverse_global" in stages


def check_tile(codec, orc, img, L, bits, q, levels_to_check, drops=(0,)):
    from paper_2005_08713_gb300 import isx
    streams, tiles, out, offs = gpu_encode(codec, [img], L, bits, qsteps=list(q))
    ref = orc.encode_tile(img, L, bits, q)
    assert_streams_equal(streams, [ref], f"{img.shape} {bits}-bit L={L} q={q}")
    paths = set()
    for z in levels_to_check:
        for drop in drops:
            dec, glob = decode_uses_global_inverse(codec, out, offs, tiles, 0, z, drop)
            want = isx.decode_path(tiles[0], z, drop)[0]
            assert glob == (want == 0), (z, drop, want)
            paths.add(want)
            assert np.array_equal(dec, orc.decode_tile(ref, z, drop)), (img.shape, bits, q, z, drop)
    return paths


def test_config1_stain_lossy_global_path(codec, orc, synth):
    """512 x 512 RGB8 (plane over 160 KB): the global forward and inverse at level 0, fused at z >= 1."""
    img = synth.stain(synth.config_seed(1))
    paths = check_tile(codec, orc, img, 3, 8, (3, 2, 1, 0), (0, 1, 2), drops=(0, 2))
    assert paths == {0, 1}


def test_config2_phantom_lossy_global_path(codec, orc, synth):
    """2048 x 2048 mono12 (sides over 1024), 5 levels, steps 8/4/2 on levels 1-3."""
    img = synth.phantom(synth.config_seed(2), 2048, 2048)
    paths = check_tile(codec, orc, img, 5, 12, (3, 2, 1, 0, 0, 0), (0, 3))
    assert 0 in paths


@pytest.mark.parametrize("shape,channels,bits,L,q", [
    ((40, 1100), 3, 8, 3, (2, 1, 0, 0)),            # a side over 1024, RGB
    ((90, 1500), 1, 12, 4, (4, 3, 2, 1, 0)),        # a side over 1024, mono12
    ((200, 300), 1, 14, 4, (4, 3, 2, 1, 0)),        # 13-16 bits: int32 coefficients
    ((96, 128), 1, 16, 3, (6, 5, 4, 2)),
    ((77, 61), 1, 13, 5, (3, 3, 3, 3, 3, 3)),
])
def test_lossy_global_path_shapes(codec, orc, shape, channels, bits, L, q):
    rng = np.random.default_rng(sum(shape) + bits)
    hi = 2 ** bits
    h, w = shape
    yy, xx = np.indices((h, w))
    base = (np.sin(xx / 17.0) + np.cos(yy / 11.0) + 2) / 4 * (hi - 1)
    if channels == 3:
        img = np.stack([base, base[::-1], base[:, ::-1]], -1)
        img = img + rng.normal(0, hi / 40, img.shape)
    else:
        img = base + rng.normal(0, hi / 40, base.shape)
    img = np.clip(np.rint(img), 0, hi - 1).astype(np.uint8 if bits <= 8 else np.uint16)
    check_tile(codec, orc, img, L, bits, q, (0, 1, L), drops=(0, 3))


def test_lossy_forward_coefficients_global_path(codec, orc, synth):
    """isx_forward_coefficients quantises the global path's int32 planes (Sec. 3): equal to the oracle."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    imgs = [synth.stain(synth.config_seed(1)), synth.phantom(7, 2048, 2048, 10, 20, 1200, 300)]
    params = [(3, 8, (3, 2, 1, 0)), (4, 12, (5, 4, 3, 2, 1))]
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
        assert np.array_equal(got[off:off + ref.size].reshape(ref.shape), ref)
        off += ref.size


def extreme_12bit(h, w, seed):
    yy, xx = np.indices((h, w))
    rng = np.random.default_rng(seed)
    return [((yy + xx) % 2) * 4095, (xx % 2) * 4095, ((yy // 2) % 2) * 4095, ((xx // 5) % 2) * 4095,
            rng.integers(0, 2, (h, w)) * 4095, rng.integers(0, 4096, (h, w))]


@pytest.mark.parametrize("qlog", [6, 8, 9, 10, 12, 15])
def test_lossy_extremes_fused_and_global_inverse(codec, orc, qlog):
    """12-bit checkerboards, stripes and 0/4095 noise with the same step 2^qlog on every level: the
    fused int16 inverse takes every case its bound admits, the global int32 inverse the rest; both
    bit-exact against the oracle's int64 decode."""
    paths = set()
    for (h, w), L in (((256, 256), 6), ((136, 200), 5)):
        pats = extreme_12bit(h, w, qlog)
        imgs = [p.astype(np.uint16) for p in pats]
        q = (qlog,) * (L + 1)
        streams, tiles, out, offs = gpu_encode(codec, imgs, L, 12, qsteps=list(q))
        refs = [orc.encode_tile(a, L, 12, q) for a in imgs]
        assert_streams_equal(streams, refs, f"12-bit extremes, step 2^{qlog}")
        from paper_2005_08713_gb300 import isx
        for i, ref in enumerate(refs):
            for z in (0, 2):
                for drop in (0, 3):
                    dec, glob = decode_uses_global_inverse(codec, out, offs, tiles, i, z, drop)
                    want = isx.decode_path(tiles[i], z, drop)[0]
                    assert glob == (want == 0)
                    paths.add(want)
                    assert np.array_equal(dec, orc.decode_tile(ref, z, drop)), (qlog, i, z, drop)
    if qlog <= 6:
        assert paths == {1}
    elif qlog >= 12:
        assert paths == {0}
    else:
        assert paths == {0, 1}
