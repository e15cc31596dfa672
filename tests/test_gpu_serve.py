"""The viewport server: requests served in the mix (continuous batching over
several streams) give exactly what each gives decoded alone, and what the
oracle gives."""
import numpy as np
import pytest

from gpu_helpers import gpu_encode, torch_cuda

pytestmark = pytest.mark.gpu


def _pyramid(codec, synth, lossy, W=3000, H=2000, T=256, L=8):
    from paper_2005_08713_gb300 import isx, serve
    img = synth.slide(synth.config_seed(3), 9000, 6000, W, H)
    grid = [(x, y, min(T, W - x), min(T, H - y)) for y in range(0, H, T) for x in range(0, W, T)]
    imgs = [np.ascontiguousarray(img[y:y + h, x:x + w]) for (x, y, w, h) in grid]
    q = [3, 2, 1] + [0] * (L - 2) if lossy else [0] * (L + 1)
    streams, tiles, out, offs = gpu_encode(codec, imgs, L, 8, [q] * len(imgs), origins=[(x, y) for (x, y, _, _) in grid])
    return serve.Pyramid(W, H, T, L, 3, 8, out, offs, isx.TileArray(tiles)), streams, grid


def test_served_mix_equals_each_request_alone_and_the_oracle(orc, synth):
    from paper_2005_08713_gb300 import isx, serve
    torch = torch_cuda()
    codec = isx.Codec(0)
    pyrs, meta = [], []
    for lossy in (True, False):
        p, streams, grid = _pyramid(codec, synth, lossy)
        pyrs.append(p)
        meta.append((streams, grid))
    reqs = serve.poisson_requests(20000.0, 160, pyrs, seed=5, view=(640, 360), zmax=7)
    srv = serve.Server(pyrs, slots=3, max_batch=8, scratch_budget=64 << 20, out_shape=(360, 640), keep_outputs=True)
    done = srv.run(reqs)
    srv.close()
    # the same requests again with levels 3.. kept decoded on the device
    reqs2 = serve.poisson_requests(20000.0, 160, pyrs, seed=5, view=(640, 360), zmax=7)
    srv2 = serve.Server(pyrs, slots=2, max_batch=16, scratch_budget=64 << 20, out_shape=(360, 640), keep_outputs=True,
                        resident_from=3)
    done2 = srv2.run(reqs2)
    srv2.close()
    by_id = {r.rid: r.result for r in done}
    for r in done2:
        assert np.array_equal(r.result, by_id[r.rid]), r.rid
    assert len(done) == len(reqs)
    assert max(srv.batch_sizes) > 1, "requests arriving together should share batches"
    for r in done:
        p = pyrs[r.pyramid]
        rx, ry, rw, rh = r.rect
        alone = torch.zeros((rh, rw, 3), dtype=torch.uint8, device="cuda")
        codec.decode_region(p.stream, p.offsets, p.tiles, r.z, r.rect, alone)
        assert codec.sync_status() == 0
        assert np.array_equal(r.result, alone.cpu().numpy()), r.rid
    # a few against the oracle's decode of the tiles
    for r in done[:12]:
        streams, grid = meta[r.pyramid]
        rx, ry, rw, rh = r.rect
        z = r.z
        ref = np.zeros((rh, rw, 3), np.uint8)
        for (x, y, w, h), s in zip(grid, streams):
            tx, ty = x >> z, y >> z
            d = orc.decode_tile(s, z)
            x0, y0 = max(tx, rx), max(ty, ry)
            x1, y1 = min(tx + d.shape[1], rx + rw), min(ty + d.shape[0], ry + rh)
            if x0 < x1 and y0 < y1:
                ref[y0 - ry:y1 - ry, x0 - rx:x1 - rx] = d[y0 - ty:y1 - ty, x0 - tx:x1 - tx]
        assert np.array_equal(r.result, ref), r.rid
    codec.close()


def test_small_tile_cache_evicts_and_stays_exact(synth):
    """A decoded-tile cache far smaller than the levels it serves: tiles are evicted and decoded again,
    and every served viewport still equals the same region decoded alone."""
    from paper_2005_08713_gb300 import isx, serve
    torch = torch_cuda()
    codec = isx.Codec(0)
    p, _, _ = _pyramid(codec, synth, True, W=3000, H=2000)
    reqs = serve.poisson_requests(20000.0, 200, [p], seed=11, view=(640, 360), zmax=2)
    srv = serve.Server([p], slots=3, max_batch=8, scratch_budget=64 << 20, out_shape=(360, 640), keep_outputs=True,
                       cache_bytes=4 << 20)
    done = srv.run(reqs)
    stats = srv.cache_stats()
    srv.close()
    assert len(done) == 200 and stats["tile_hits"] > 0 and stats["tile_misses"] > stats["cache_bytes"] // (256 * 256 * 3)
    for r in done:
        rx, ry, rw, rh = r.rect
        alone = torch.zeros((rh, rw, 3), dtype=torch.uint8, device="cuda")
        codec.decode_region(p.stream, p.offsets, p.tiles, r.z, r.rect, alone)
        assert codec.sync_status() == 0
        assert np.array_equal(r.result, alone.cpu().numpy()), r.rid
    codec.close()


def test_server_admission_refuses_a_request_beyond_the_slot_budget(synth):
    from paper_2005_08713_gb300 import isx, serve
    codec = isx.Codec(0)
    p, _, _ = _pyramid(codec, synth, True, W=1024, H=768)
    reqs = [serve.Request(0, 0.0, 0, 0, (0, 0, 640, 360))]
    srv = serve.Server([p], slots=1, max_batch=4, scratch_budget=1 << 16, out_shape=(360, 640))
    with pytest.raises(RuntimeError, match="slot budget"):
        srv.run(reqs)
    srv.close()
    codec.close()


def test_served_request_over_a_corrupt_tile_alone_reports_an_error(synth):
    """One tile's stream scrambled on the device: the requests that meet it report ISX_ERR_CORRUPT,
    every other request of the same batches still equals its decode alone."""
    from paper_2005_08713_gb300 import isx, serve
    torch = torch_cuda()
    codec = isx.Codec(0)
    p, streams, grid = _pyramid(codec, synth, True, W=2048, H=1024)
    offs = p.offsets.cpu().numpy()
    bad = 9                                                # grid 8 x 4: pixels (256..511, 256..511) at level 0
    ref_stream = p.stream.clone()
    p.stream[int(offs[bad]) + 40:int(offs[bad + 1])] ^= 0x5A
    rects = [(0, 0, 200, 150), (300, 300, 200, 150), (1200, 700, 200, 150), (600, 40, 200, 150),
             (250, 250, 20, 20), (1800, 800, 200, 150)]
    reqs = [serve.Request(i, 0.0, 0, 0, r) for i, r in enumerate(rects)]
    srv = serve.Server([p], slots=1, max_batch=8, scratch_budget=64 << 20, out_shape=(150, 200), keep_outputs=True)
    done = srv.run(reqs)
    srv.close()
    assert len(srv.batch_sizes) == 1
    for r in done:
        meets = bad in set(p.tiles_meeting(0, *r.rect).tolist())
        assert (r.error == "ISX_ERR_CORRUPT") == meets, (r.rid, r.error)
        if not meets:
            rx, ry, rw, rh = r.rect
            alone = torch.zeros((rh, rw, 3), dtype=torch.uint8, device="cuda")
            codec.decode_region(ref_stream, p.offsets, p.tiles, 0, r.rect, alone)
            assert codec.sync_status() == 0
            assert np.array_equal(r.result, alone.cpu().numpy()), r.rid
    assert sum(r.error is not None for r in done) == 2
    codec.close()


def test_copy_rects_any_offsets_and_sizes():
    """isx_copy_rects against plain tensor slicing: source and destination at every byte offset modulo 4
    and 16, row lengths of 0..800 bytes (heads and tails of 0-3 bytes, rows shorter than a word), row
    counts that span several 32-row pieces, pitches that are not multiples of 4; bytes outside the
    rectangles stay untouched."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    rng = np.random.default_rng(11)
    src = torch.from_numpy(rng.integers(0, 256, 1 << 22, dtype=np.uint8)).cuda()
    dst = torch.zeros(1 << 26, dtype=torch.uint8, device="cuda")
    specs, lo = [], 0
    for k in range(300):
        rb = int(rng.integers(0, 801)) if k % 7 else int(rng.integers(0, 5))
        rows = int(rng.integers(1, 130)) if k % 5 else int(rng.integers(0, 3))
        sp, dp = rb + int(rng.integers(0, 40)), rb + int(rng.integers(0, 40))
        so = int(rng.integers(0, src.numel() - max(rows, 1) * (sp + 1)))
        do = lo + int(rng.integers(0, 17))                   # destinations side by side, never overlapping
        lo = do + max(rows, 1) * (dp + 1)
        specs.append((so, sp, do, dp, rb, rows))
    assert lo <= dst.numel()
    c = np.zeros(len(specs), isx.COPY_DTYPE)
    for i, (so, sp, do, dp, rb, rows) in enumerate(specs):
        c[i] = (src.data_ptr() + so, sp, dst.data_ptr() + do, dp, rb, rows)
    with isx.Codec(0) as codec:
        codec.copy_rects(c)
        assert codec.sync_status() == 0
    got = dst.cpu().numpy()
    want = np.zeros_like(got)
    s = src.cpu().numpy()
    for so, sp, do, dp, rb, rows in specs:
        for r in range(rows):
            want[do + r * dp:do + r * dp + rb] = s[so + r * sp:so + r * sp + rb]
    assert np.array_equal(got, want)
