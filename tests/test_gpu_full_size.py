"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: the 40000 x 30000 slide (18 526 tiles in one call, lossy
and lossless) checked on sampled tiles against the oracle plus the lossless
identity over the whole image, and the 4096-tile mixed batch checked tile by
tile in full."""
import os

import numpy as np
import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

W, H, T, L = 40000, 30000, 256, 8
LOSSY_Q = [3, 2, 1, 0, 0, 0, 0, 0, 0]


@pytest.fixture(scope="module")
def slide(synth):
    torch = torch_cuda()
    h = torch.empty((H, W, 3), dtype=torch.uint8, pin_memory=True)
    synth.slide(synth.config_seed(3), 0, 0, W, H, out=h.numpy())
    d = h.to("cuda")
    yield h.numpy(), d
    del d


@pytest.mark.parametrize("lossless", [False, True])
def test_whole_slide_sampled_tiles_and_lossless_identity(orc, slide, lossless):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    img, d_img = slide
    grid = [(x, y, min(T, W - x), min(T, H - y)) for y in range(0, H, T) for x in range(0, W, T)]
    q = [0] * 9 if lossless else LOSSY_Q
    tiles = isx.TileArray([isx.tile_from_tensor(d_img[y:y + h, x:x + w], L, 8, q, x, y) for (x, y, w, h) in grid])
    with isx.Codec(0) as codec:
        out = torch.empty(W * H * 3 + (1 << 24), dtype=torch.uint8, device="cuda")
        offs = torch.zeros(len(grid) + 1, dtype=torch.int64, device="cuda")
        dec = torch.empty_like(d_img)
        codec.encode_tiles(tiles, out, offs)
        assert codec.sync_status() == 0
        codec.decode_region(out, offs, tiles, 0, (0, 0, W, H), dec)
        assert codec.sync_status() == 0
        if lossless:
            assert torch.equal(dec, d_img), "lossless round trip of the whole slide"
        rng = np.random.default_rng(17 + lossless)
        gw, gh = -(-W // T), -(-H // T)
        sample = set(rng.choice(len(grid), 20, replace=False).tolist())
        sample |= {gw - 1, len(grid) - gw, len(grid) - 1}   # right edge, bottom edge, corner
        o = offs.cpu().numpy()
        for i in sorted(sample):
            x, y, w, h = grid[i]
            ref = orc.encode_tile(np.ascontiguousarray(img[y:y + h, x:x + w]), L, 8, q)
            got = out[int(o[i]):int(o[i + 1])].cpu().numpy().tobytes()
            assert got == ref, f"tile {i} ({x},{y},{w}x{h})"
            assert np.array_equal(dec[y:y + h, x:x + w].cpu().numpy(), orc.decode_tile(ref, 0)), i
            z = 1 + i % L
            reg = torch.zeros((-(-h // (1 << z)), -(-w // (1 << z)), 3), dtype=torch.uint8, device="cuda")
            codec.decode_region(out, offs, tiles, z, (x >> z, y >> z, reg.shape[1], reg.shape[0]), reg)
            assert codec.sync_status() == 0
            assert np.array_equal(reg.cpu().numpy(), orc.decode_tile(ref, z)), (i, z)


def test_mixed_batch_all_4096_tiles(orc, synth):
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    specs = synth.batch_specs(synth.config_seed(4), 4096)
    imgs = [synth.batch_image(sp) for sp in specs]
    dev = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda() for a in imgs]
    tiles = isx.TileArray([isx.tile_from_tensor(d, sp["levels"], sp["bits"], sp["q"], 512 * i, 0)
                           for i, (d, sp) in enumerate(zip(dev, specs))])
    cores = os.cpu_count() or 1
    ts = [orc.tile_struct(a.shape[1], a.shape[0], 3 if sp["rgb"] else 1, sp["bits"], sp["levels"], sp["q"])
          for a, sp in zip(imgs, specs)]
    refs = orc.encode_tiles_mt(imgs, ts, cores)
    with isx.Codec(0) as codec:
        cap = sum(a.nbytes for a in imgs) * 2 + 4096 * len(imgs)
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        offs = torch.zeros(len(imgs) + 1, dtype=torch.int64, device="cuda")
        codec.encode_tiles(tiles, out, offs)
        assert codec.sync_status() == 0
        o = offs.cpu().numpy()
        raw = out[:int(o[-1])].cpu().numpy().tobytes()
        bad = [i for i in range(len(imgs)) if raw[o[i]:o[i + 1]] != refs[i]]
        assert not bad, f"{len(bad)} of {len(imgs)} streams differ (first {bad[0]})"
        outs = [torch.zeros(d.shape, dtype=d.dtype, device="cuda") for d in dev]
        jobs = [(i, (t.x0, t.y0, t.width, t.height), oo) for i, (t, oo) in enumerate(zip(tiles, outs))]
        codec.decode_jobs(out, offs, tiles, jobs)
        assert codec.sync_status() == 0
    ref_dec = [np.zeros_like(a) for a in imgs]
    orc.decode_tiles_mt(refs, 0, ref_dec, cores)
    for i, (oo, r) in enumerate(zip(outs, ref_dec)):
        got = oo.cpu().numpy()
        if r.dtype == np.uint16:
            got = got.view(np.uint16)
        assert np.array_equal(got, r), i
