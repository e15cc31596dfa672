"""Batched and served forms through the C ABI: decode jobs (mixed tile
types, several requests in one call), the size-class schedule and its
autotuner, and capture-safe plans replayed from a CUDA graph.  Every result
is compared with the oracle."""
import numpy as np
import pytest

from gpu_helpers import gpu_encode, to_device, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    from paper_2005_08713_gb300 import isx
    c = isx.Codec(0)
    yield c
    c.close()


def _batch(synth, n, seed=41):
    specs = synth.batch_specs(seed, n)
    imgs = [synth.batch_image(s) for s in specs]
    return specs, imgs


def _out_for(torch, img):
    if img.dtype == np.uint16:
        return torch.zeros(img.shape, dtype=torch.int16, device="cuda")
    return torch.zeros(img.shape, dtype=torch.uint8, device="cuda")


def _host(t, like):
    a = t.cpu().numpy()
    return a.view(np.uint16) if like.dtype == np.uint16 else a


def test_decode_jobs_mixed_batch_each_tile_its_own_buffer(codec, orc, synth):
    torch = torch_cuda()
    specs, imgs = _batch(synth, 120)
    levels = [s["levels"] for s in specs]
    streams, tiles, out, offs = gpu_encode(codec, imgs, levels, [s["bits"] for s in specs], [s["q"] for s in specs])
    refs = [orc.encode_tile(a, s["levels"], s["bits"], s["q"]) for a, s in zip(imgs, specs)]
    assert streams == refs
    for z in (0, 2):
        outs, jobs = [], []
        for i, (t, img) in enumerate(zip(tiles, imgs)):
            zw, zh = -(-img.shape[1] // (1 << z)), -(-img.shape[0] // (1 << z))
            o = _out_for(torch, img[:zh, :zw])
            outs.append(o)
            jobs.append((i, (t.x0 >> z, t.y0 >> z, zw, zh), o))
        codec.decode_jobs(out, offs, tiles, jobs, level=z)
        assert codec.sync_status() == 0
        for i in range(len(imgs)):
            ref = orc.decode_tile(refs[i], z)
            assert np.array_equal(_host(outs[i], imgs[i]), ref), (i, z)


def test_decode_jobs_several_requests_in_one_call(codec, orc, synth):
    """Two overlapping viewports over a 4 x 3 tile mosaic, decoded in one call, equal the crops of the oracle image."""
    torch = torch_cuda()
    T = 96
    img = synth.slide(synth.config_seed(3), 12000, 9000, 4 * T - 17, 3 * T - 5)
    H, W = img.shape[:2]
    grid = [(x, y, min(T, W - x), min(T, H - y)) for y in range(0, H, T) for x in range(0, W, T)]
    imgs = [np.ascontiguousarray(img[y:y + h, x:x + w]) for (x, y, w, h) in grid]
    streams, tiles, out, offs = gpu_encode(codec, imgs, 3, 8, [[2, 1, 0, 0]] * len(imgs), origins=[(x, y) for (x, y, _, _) in grid])
    z = 1
    full = np.zeros((-(-H // 2), -(-W // 2), 3), np.uint8)
    for (x, y, w, h), s in zip(grid, streams):
        d = orc.decode_tile(s, z)
        full[y // 2:y // 2 + d.shape[0], x // 2:x // 2 + d.shape[1]] = d
    rects = [(10, 7, 120, 70), (60, 40, 100, 90)]
    outs, jobs = [], []
    for (rx, ry, rw, rh) in rects:
        o = torch.zeros((rh, rw, 3), dtype=torch.uint8, device="cuda")
        outs.append(o)
        for i, t in enumerate(tiles):
            jobs.append((i, (rx, ry, rw, rh), o))   # tiles outside a rectangle are skipped by the library
    codec.decode_jobs(out, offs, tiles, jobs, level=z)
    assert codec.sync_status() == 0
    for (rx, ry, rw, rh), o in zip(rects, outs):
        assert np.array_equal(o.cpu().numpy(), full[ry:ry + rh, rx:rx + rw])


def test_schedule_every_thread_count_gives_identical_results(codec, orc, synth):
    torch = torch_cuda()
    specs, imgs = _batch(synth, 48, seed=7)
    refs = [orc.encode_tile(a, s["levels"], s["bits"], s["q"]) for a, s in zip(imgs, specs)]
    saved = codec.get_schedule()
    try:
        for t in (256, 512, 1024):
            codec.set_schedule([t] * 5, [t] * 5)
            streams, tiles, out, offs = gpu_encode(codec, imgs, [s["levels"] for s in specs], [s["bits"] for s in specs],
                                                   [s["q"] for s in specs])
            assert streams == refs, t
            outs = [_out_for(torch, a) for a in imgs]
            jobs = [(i, (tl.x0, tl.y0, a.shape[1], a.shape[0]), o) for i, (tl, a, o) in enumerate(zip(tiles, imgs, outs))]
            codec.decode_jobs(out, offs, tiles, jobs)
            assert codec.sync_status() == 0
            for i in range(len(imgs)):
                assert np.array_equal(_host(outs[i], imgs[i]), orc.decode_tile(refs[i], 0)), (t, i)
    finally:
        codec.set_schedule(saved["forward_threads"], saved["inverse_threads"])
    from paper_2005_08713_gb300 import isx
    with pytest.raises(isx.IsxError):
        codec.set_schedule([128] * 5, [256] * 5)


def test_autotune_then_plans_replayed_from_a_cuda_graph(orc, synth):
    from paper_2005_08713_gb300 import isx
    torch = torch_cuda()
    specs, imgs = _batch(synth, 64, seed=9)
    refs = [orc.encode_tile(a, s["levels"], s["bits"], s["q"]) for a, s in zip(imgs, specs)]
    with isx.Codec(0) as c:
        dev = [to_device(a) for a in imgs]
        maxw = 512
        tiles = [isx.tile_from_tensor(d, s["levels"], s["bits"], s["q"], i * maxw, 0) for i, (d, s) in enumerate(zip(dev, specs))]
        sched = c.autotune(tiles, reps=2)
        assert all(t in (256, 512, 1024) for t in sched["forward_threads"] + sched["inverse_threads"])
        cap = sum(a.nbytes for a in imgs) * 3 + 4096 * len(imgs)
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        offs = torch.zeros(len(imgs) + 1, dtype=torch.int64, device="cuda")
        outs = [_out_for(torch, a) for a in imgs]
        jobs = [(i, (t.x0, t.y0, t.width, t.height), o) for i, (t, o) in enumerate(zip(tiles, outs))]
        penc = c.plan_encode(tiles)
        pdec = c.plan_decode(tiles, jobs)
        assert penc.device_bytes > 0 and pdec.device_bytes > 0
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            penc.launch_encode(out, offs, s)          # eager launch first (warms every kernel)
            pdec.launch_decode(out, offs, s)
        s.synchronize()
        assert penc.sync_status(s) == 0 and pdec.sync_status(s) == 0
        assert penc.launch_count > 0 and pdec.launch_count > 0
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            penc.launch_encode(out, offs, s)
            pdec.launch_decode(out, offs, s)
        for rep in range(2):
            out.zero_()
            for o in outs:
                o.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert penc.sync_status(s) == 0 and pdec.sync_status(s) == 0
            o_h = offs.cpu().numpy()
            raw = out[:int(o_h[-1])].cpu().numpy().tobytes()
            got = [raw[o_h[i]:o_h[i + 1]] for i in range(len(imgs))]
            assert got == refs, rep
            for i in range(len(imgs)):
                assert np.array_equal(_host(outs[i], imgs[i]), orc.decode_tile(refs[i], 0)), (rep, i)
        del g
        penc.close()
        pdec.close()


def test_tile_stamps_bracket_each_tiles_work(synth):
    """isx_set_tile_stamps: every encoded tile gets start <= end, a decode stamps only the tiles of its jobs
    (by stream index), and a plan made while stamps are set records them on each launch."""
    torch = torch_cuda()
    from paper_2005_08713_gb300 import isx
    imgs = [synth.slide(synth.config_seed(3), 256 * k, 512, 200 + 7 * k, 150) for k in range(6)]
    codec = isx.Codec(0)
    st = torch.zeros(4 * 8, dtype=torch.int64, device="cuda")
    codec.set_tile_stamps(st)
    streams, tiles, out, offs = gpu_encode(codec, imgs, 5, 8, [3, 2, 1, 0, 0, 0])
    dec = torch.zeros((150, 300, 3), dtype=torch.uint8, device="cuda")
    codec.decode_jobs(out, offs, tiles, [(i, (tiles[i].x0, 0, tiles[i].width, 150), dec) for i in (2, 4)])
    assert codec.sync_status() == 0
    s = st.cpu().numpy().view(np.uint64).reshape(4, 8)
    none = np.iinfo(np.uint64).max
    assert all(0 < s[0, i] <= s[1, i] for i in range(6))                   # every encoded tile
    assert list(s[0, 6:]) == [none, none] and list(s[1, 6:]) == [0, 0]     # slots past the call's tiles
    for i in range(6):
        if i in (2, 4):
            assert s[1, i] <= s[2, i] <= s[3, i]                             # decoded after its encode
        else:
            assert s[2, i] == none and s[3, i] == 0
    assert (s[1, :6] - s[0, :6]).max() < 10 ** 10                          # under 10 s
    # a plan replayed: fresh stamps per launch
    plan = codec.plan_encode(isx.TileArray(tiles))
    codec.set_tile_stamps(None)
    st.zero_()
    plan.launch_encode(out, offs)
    assert plan.sync_status() == 0
    s2 = st.cpu().numpy().view(np.uint64).reshape(4, 8)
    assert all(s[1, i] < s2[0, i] <= s2[1, i] for i in range(6))
    with pytest.raises(isx.IsxError):
        codec.set_tile_stamps(torch.zeros(4 * 2, dtype=torch.int64, device="cuda"))
        codec.encode_tiles(tiles, out, offs)                                 # more tiles than stamp entries
    codec.set_tile_stamps(None)
    plan.close()
    codec.close()
