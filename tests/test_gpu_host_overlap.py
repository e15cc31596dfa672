"""The host-buffer entry points on inputs large enough for the decode's
overlapped form (the inverse transform in chunks, each chunk's rows copied
back on their own stream while the next is inverted): the results must
equal, byte for byte, those of the device-buffer entry points on the same
tiles, which the other GPU tests hold against the oracle."""
import numpy as np
import pytest

from gpu_helpers import to_device, torch_cuda

pytestmark = pytest.mark.gpu

Q = [3, 2, 1, 0, 0, 0, 0, 0, 0]
W, H, T = 5000, 5000, 256   # 75 MB of RGB8: 400 tiles, the last column 136 px wide, the last row 136 px high


@pytest.fixture(scope="module")
def codec():
    torch_cuda()
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def case(synth):
    from paper_2005_08713_gb300 import isx
    img = np.ascontiguousarray(synth.slide(synth.config_seed(3), 3000, 2000, W, H))
    grid = [(x, y, min(T, W - x), min(T, H - y)) for y in range(0, H, T) for x in range(0, W, T)]
    h_tiles = [isx.tile_from_array(img[y:y + h, x:x + w], 8, 8, Q, x, y) for (x, y, w, h) in grid]
    d_img = to_device(img)
    d_tiles = [isx.tile_from_tensor(d_img[y:y + h, x:x + w], 8, 8, Q, x, y) for (x, y, w, h) in grid]
    return img, grid, h_tiles, d_img, d_tiles


def _device_encode(codec, d_tiles, cap):
    torch = torch_cuda()
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(len(d_tiles) + 1, dtype=torch.int64, device="cuda")
    codec.encode_tiles(d_tiles, out, offs)
    assert codec.sync_status() == 0
    o = offs.cpu().numpy().astype(np.uint64)
    return out[: int(o[-1])].cpu().numpy(), o, out, offs


def test_host_calls_equal_the_device_calls(codec, case, orc):
    torch = torch_cuda()
    img, grid, h_tiles, d_img, d_tiles = case
    ref_bytes, ref_offs, d_out, d_offs = _device_encode(codec, d_tiles, img.nbytes + (1 << 20))
    for rep in range(2):   # twice: the second call reuses the context's staging
        out = np.zeros(img.nbytes + (1 << 20), np.uint8)
        offs = np.zeros(len(h_tiles) + 1, np.uint64)
        codec.encode_tiles_host(h_tiles, out, offs)
        assert np.array_equal(offs, ref_offs), rep
        assert np.array_equal(out[: int(offs[-1])], ref_bytes), rep
    # two tiles against the oracle as well
    for k in (0, len(grid) - 1):
        x, y, w, h = grid[k]
        assert out[offs[k]:offs[k + 1]].tobytes() == orc.encode_tile(img[y:y + h, x:x + w], 8, 8, Q), k
    # the whole image, and a rectangle that cuts tiles on every side
    for rect in ((0, 0, W, H), (101, 77, 4800, 4600)):
        rx, ry, rw, rh = rect
        res = np.full((rh, rw, 3), 0x5A, np.uint8)
        codec.decode_region_host(out, offs, h_tiles, 0, rect, res)
        dev = torch.zeros((rh, rw, 3), dtype=torch.uint8, device="cuda")
        codec.decode_region(d_out, d_offs, d_tiles, 0, rect, dev)
        assert codec.sync_status() == 0
        assert np.array_equal(res, dev.cpu().numpy()), rect


def test_overlapped_decode_leaves_uncovered_rows_zero(codec, case):
    """A rectangle larger than the tiles: rows and columns no tile covers come back as 0."""
    img, grid, h_tiles, d_img, d_tiles = case
    out = np.zeros(img.nbytes + (1 << 20), np.uint8)
    offs = np.zeros(len(h_tiles) + 1, np.uint64)
    codec.encode_tiles_host(h_tiles, out, offs)
    sub = [t for t in h_tiles if t.y0 >= 1024]   # the tiles of rows 1024.. only
    first = len(h_tiles) - len(sub)
    sub_offs = offs[first:].copy()
    res = np.full((H, W, 3), 0x5A, np.uint8)
    codec.decode_region_host(out, sub_offs, sub, 0, (0, 0, W, H), res)
    assert not res[:1024].any()
    full = np.zeros((H, W, 3), np.uint8)
    codec.decode_region_host(out, offs, h_tiles, 0, (0, 0, W, H), full)
    assert np.array_equal(res[1024:], full[1024:])


def test_host_encode_reports_the_capacity_it_needs(codec, case):
    from paper_2005_08713_gb300 import isx
    img, grid, h_tiles, d_img, d_tiles = case
    out = np.zeros(img.nbytes + (1 << 20), np.uint8)
    offs = np.zeros(len(h_tiles) + 1, np.uint64)
    codec.encode_tiles_host(h_tiles, out, offs)
    total = int(offs[-1])
    small = np.zeros(total // 2, np.uint8)
    offs2 = np.zeros(len(h_tiles) + 1, np.uint64)
    with pytest.raises(isx.IsxError) as ei:
        codec.encode_tiles_host(h_tiles, small, offs2)
    assert ei.value.status == isx.ISX_ERR_CAPACITY
    assert int(offs2[-1]) >= total
    big = np.zeros(int(offs2[-1]), np.uint8)
    codec.encode_tiles_host(h_tiles, big, offs2)   # the reported size suffices
    assert np.array_equal(offs2, offs) and np.array_equal(big[:total], out[:total])
