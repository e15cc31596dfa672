"""Host-side planning of the viewport server (no GPU): which tiles a request
touches at a resolution level, and the synthetic Poisson request stream."""
import numpy as np
import pytest

from paper_2005_08713_gb300 import isx, serve


def _pyramid(width, height, tile, levels):
    return serve.Pyramid(width=width, height=height, tile=tile, levels=levels, channels=3, bits=8,
                         stream=None, offsets=None, tiles=None)


def _brute_force(p, z, rx, ry, rw, rh):
    """Tiles whose level-z footprint [x0 >> z, (x0 >> z) + level size) meets the rectangle, row-major."""
    out = []
    for gy in range(p.grid_h):
        for gx in range(p.grid_w):
            x0, y0 = gx * p.tile, gy * p.tile
            tw, th = min(p.tile, p.width - x0), min(p.tile, p.height - y0)
            fx, fy = x0 >> z, y0 >> z
            fw, fh = isx.level_dim(tw, z), isx.level_dim(th, z)
            if fx < rx + rw and rx < fx + fw and fy < ry + rh and ry < fy + fh:
                out.append(gy * p.grid_w + gx)
    return out


@pytest.mark.parametrize("width,height,tile,levels", [(1000, 700, 256, 4), (40000, 30000, 256, 8), (513, 257, 128, 3),
                                                      (256, 256, 256, 5)])
def test_tiles_meeting_cover_the_rectangle(width, height, tile, levels):
    p = _pyramid(width, height, tile, levels)
    rng = np.random.default_rng(width + height + tile)
    for _ in range(40):
        z = int(rng.integers(0, levels + 1))
        lw, lh = p.level_size(z)
        rw, rh = int(rng.integers(1, min(lw, 2000) + 1)), int(rng.integers(1, min(lh, 1200) + 1))
        rx, ry = int(rng.integers(0, lw - rw + 1)), int(rng.integers(0, lh - rh + 1))
        got = set(p.tiles_meeting(z, rx, ry, rw, rh).tolist())
        need = set(_brute_force(p, z, rx, ry, rw, rh)) if p.grid_w * p.grid_h <= 4096 else None
        if need is not None:
            # every tile the rectangle needs is listed; extra tiles are allowed (the library skips them)
            assert need <= got, (z, rx, ry, rw, rh, sorted(need - got)[:5])
        assert all(0 <= i < p.grid_w * p.grid_h for i in got)


def test_tiles_meeting_is_exact_when_the_tile_edge_divides():
    p = _pyramid(1024, 768, 256, 3)
    for z in range(4):
        lw, lh = p.level_size(z)
        for rx, ry, rw, rh in [(0, 0, lw, lh), (lw // 3, lh // 5, max(1, lw // 4), max(1, lh // 4)), (lw - 1, lh - 1, 1, 1)]:
            assert sorted(p.tiles_meeting(z, rx, ry, rw, rh).tolist()) == _brute_force(p, z, rx, ry, rw, rh)


def test_poisson_requests_stay_inside_their_level():
    pyrs = [_pyramid(40000, 30000, 256, 8), _pyramid(5000, 3000, 256, 6)]
    reqs = serve.poisson_requests(2000.0, 500, pyrs, seed=3, view=(1920, 1080), zmax=7)
    assert len(reqs) == 500
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    # mean inter-arrival close to 1 / rate
    assert abs(float(np.diff(t).mean()) - 1 / 2000.0) < 0.25 / 2000.0
    for r in reqs:
        p = pyrs[r.pyramid]
        assert 0 <= r.z <= min(7, p.levels)
        lw, lh = p.level_size(r.z)
        rx, ry, rw, rh = r.rect
        assert rw == min(1920, lw) and rh == min(1080, lh)
        assert 0 <= rx and rx + rw <= lw and 0 <= ry and ry + rh <= lh


def test_latency_stats():
    class R:
        def __init__(self, a, d):
            self.arrival, self.done = a, d
    st = serve.latency_stats([R(0.0, 0.001 * (i + 1)) for i in range(100)])
    assert st["p50_ms"] == pytest.approx(50.5, abs=0.01)
    assert st["max_ms"] == pytest.approx(100.0)
    assert serve.latency_stats([])["p50_ms"] is None


@pytest.mark.parametrize("width,height,tile,levels", [(1000, 700, 256, 4), (40000, 30000, 256, 8), (513, 257, 128, 3),
                                                      (3000, 2000, 96, 5)])
def test_cells_tile_each_level_and_meet_rectangles_exactly(width, height, tile, levels):
    """At every exact level: the cells partition the level; each cell's tiles have footprints that
    partition the cell; cell_pairs lists, rectangle by rectangle, exactly the cells meeting it."""
    p = _pyramid(width, height, tile, levels)
    rng = np.random.default_rng(tile + levels)
    for z in range(levels + 1):
        if not p.exact_at(z):
            continue
        lw, lh = p.level_size(z)
        cw, ch = p.cell_grid(z)
        cells = np.arange(cw * ch)
        cx, cy, cwid, chei = p.cell_rects(z, cells)
        assert int((cwid * chei).sum()) == lw * lh and cwid.min() > 0 and chei.min() > 0
        pos, tiles = p.cell_tiles(z, cells)
        assert sorted(tiles.tolist()) == list(range(p.grid_w * p.grid_h))     # every tile in one cell
        fx, fy, fw, fh = p.tile_rects(z, tiles)
        assert np.all(fx >= cx[pos]) and np.all(fx + fw <= cx[pos] + cwid[pos])
        assert np.all(fy >= cy[pos]) and np.all(fy + fh <= cy[pos] + chei[pos])
        assert np.array_equal(np.bincount(pos, weights=fw * fh, minlength=len(cells)), (cwid * chei).astype(float))
        rects = []
        for _ in range(20):
            rw, rh = int(rng.integers(1, min(lw, 2000) + 1)), int(rng.integers(1, min(lh, 1200) + 1))
            rects.append((int(rng.integers(0, lw - rw + 1)), int(rng.integers(0, lh - rh + 1)), rw, rh))
        req, got = p.cell_pairs(z, np.array(rects, dtype=np.int64))
        assert np.all(np.diff(req) >= 0)
        for i, (rx, ry, rw, rh) in enumerate(rects):
            meet = (cx < rx + rw) & (rx < cx + cwid) & (cy < ry + rh) & (ry < cy + chei)
            assert got[req == i].tolist() == np.flatnonzero(meet).tolist(), (z, rects[i])


# ---------------------------------------------------------------- the batching loop, with fakes
# Server._admit, _copies and run only plan and keep time; decoding and copying are the library's.  A fake
# codec reports scratch sizes and records calls, CPU tensors stand in for the output pool and the tile
# caches, and fake events complete each batch after a few polls, so the continuous-batching logic and
# the cache bookkeeping run on the CPU through the server's own _launch.

class _FakeCodec:
    def __init__(self, per_tile):
        self.per_tile = per_tile
        self.decoded = []          # (level, tiles) of each decode call
        self.copies = 0

    def decode_jobs_scratch(self, tiles, jobs, level=0, drop_lsb_planes=0):
        return self.per_tile * len(jobs)

    # the device status word: a decode touching a tile in `bad` reports ISX_ERR_CORRUPT
    bad = frozenset()
    pending = 0

    def decode_jobs_array(self, stream_buf, offsets, tiles, jobs, level=0, drop_lsb_planes=0, stream=None):
        self.decoded.append((level, [int(t) for t in jobs["tile"]]))
        if any(int(t) in self.bad for t in jobs["tile"]):
            self.pending = 3

    def copy_rects(self, copies, stream=None):
        self.copies += len(copies)

    def sync_status(self, stream=None):
        st, self.pending = self.pending, 0
        return st


class _FakeEvent:
    def __init__(self, polls):
        self.left = polls

    def query(self):
        self.left -= 1
        return self.left <= 0


def _fake_server(pyrs, slots=2, max_batch=4, budget=10_000, pool=8, per_tile=100, resident_from=None, polls=3,
                 cache_bytes=1 << 30):
    import collections
    import torch
    srv = serve.Server.__new__(serve.Server)
    srv.torch = torch
    srv.pyr = list(pyrs)
    srv.max_batch, srv.budget = max_batch, budget
    srv.slots = [serve._Slot(_FakeCodec(per_tile), None) for _ in range(slots)]
    srv.pool = collections.deque(torch.zeros((64, 96, 3), dtype=torch.uint8) for _ in range(pool))
    srv.out_shape = (64, 96, 3)
    srv.keep_outputs = False
    srv.resident_from = resident_from if resident_from is not None else max(p.levels for p in pyrs) + 1
    srv._init_state()
    srv.resident = {(pi, z): torch.zeros((pyrs[pi].level_size(z)[1], pyrs[pi].level_size(z)[0], 3), dtype=torch.uint8)
                    for pi, z in srv._levels()[1]}
    srv._make_caches(cache_bytes, "cpu", srv.slots[0].codec)
    srv.launched, srv.waits, srv.cell_tiles = [], [], 0
    real_launch = srv._launch

    def launch(slot, batch):
        srv.launched.append([r.rid for r in batch])
        srv.cell_tiles += sum(len(srv.pyr[pi].cell_tiles(z, cells)[1]) for (pi, z), (cells, _) in slot.misses.items())
        real_launch(slot, batch)
    srv._launch = launch
    srv._record = lambda stream: _FakeEvent(polls)
    srv._wait = lambda stream, ev: srv.waits.append(ev)
    return srv


def _req(rid, t, pi=0, z=0, rect=(0, 0, 96, 64)):
    return serve.Request(rid, t, pi, z, rect)


def _consistent(cache):
    """The cache's maps agree: slot_of and tile_of are inverse, holds and fillers are clear."""
    s = np.flatnonzero(cache.tile_of >= 0)
    assert np.array_equal(cache.slot_of[cache.tile_of[s]], s)
    assert np.count_nonzero(cache.slot_of >= 0) == len(s)


def test_admit_takes_requests_in_order_and_shares_missing_tiles():
    import collections
    srv = _fake_server([_pyramid(1000, 700, 256, 4)], max_batch=3)
    q = collections.deque(_req(i, 0.0) for i in range(5))
    slot = srv.slots[0]
    batch = srv._admit(q, slot)
    assert [r.rid for r in batch] == [0, 1, 2] and [r.rid for r in q] == [3, 4]
    assert len(srv.pool) == 8 - 3
    cache = srv.caches[(0, 0)]
    for r in batch:
        assert r.out.shape == (64, 96, 3) and r.out.data_ptr() == r.buf.data_ptr()
    ridx, cells, slots = slot.pairs[(0, 0)]
    assert ridx.tolist() == [0, 1, 2] and cells.tolist() == [0, 0, 0]   # the one cell meeting each viewport
    # cell 0 is decoded once for the batch, which holds its slot once
    new, vict = slot.misses[(0, 0)]
    assert new.tolist() == [0] and slots.tolist() == [vict[0]] * 3
    assert cache.holds[vict[0]] == 1 and cache.filler[vict[0]] == slot.bid
    assert cache.misses == 1 and cache.hits == 2
    _consistent(cache)


def test_admit_stops_at_the_scratch_budget_of_a_group():
    import collections
    p = _pyramid(4000, 700, 256, 4)
    # each request meets 4 cells no other request meets (a 300 x 300 viewport at level 0, cells = tiles);
    # 100 bytes of scratch a tile (120 with the margin), budget 1000: two requests fit, the third would not
    srv = _fake_server([p], max_batch=8, budget=1000)
    q = collections.deque(_req(i, 0.0, rect=(600 * i + 200, 200, 300, 300)) for i in range(4))
    batch = srv._admit(q, srv.slots[0])
    base, per = srv.scratch_fit[(0, 0)]
    assert [r.rid for r in batch] == [0, 1] and len(q) == 2
    assert len(srv.slots[0].misses[(0, 0)][0]) == 8 and base + per * 8 <= 1000
    assert len(srv.caches[(0, 0)].cached()) == 8          # only the admitted requests' cells took slots
    # a request whose own tiles cannot fit the budget is refused outright
    srv2 = _fake_server([p], budget=300)
    with pytest.raises(RuntimeError, match="more than the slot budget"):
        srv2._admit(collections.deque([_req(0, 0.0, rect=(200, 200, 300, 300))]), srv2.slots[0])


def test_admit_waits_while_batches_in_flight_hold_the_slots():
    """A cache of few slots: the second batch cannot take slots while the first holds them; it is
    admitted once the first is released."""
    import collections
    p = _pyramid(4000, 700, 256, 4)
    srv = _fake_server([p], slots=2, max_batch=1, budget=1 << 30, cache_bytes=0)
    cache = srv.caches[(0, 0)]
    need = cache.n_slots // 2 + 1
    # two requests, each more than half the slots, no tile in common
    w = 256 * need
    reqs = [_req(0, 0.0, rect=(0, 0, min(w, 4000), 256)), _req(1, 0.0, rect=(0, 256, min(w, 4000), 256))]
    n0 = len(p.tiles_meeting(0, *reqs[0].rect))
    if 2 * n0 <= cache.n_slots:
        pytest.skip("cache large enough for both")
    q = collections.deque(reqs)
    a, b = srv.slots
    assert [r.rid for r in srv._admit(q, a)] == [0]
    srv._launch(a, [reqs[0]])
    assert srv._admit(q, b) == [] and len(q) == 1          # waits: not refused, not admitted
    srv._release(a)
    a.busy = False
    assert [r.rid for r in srv._admit(q, b)] == [1]


def test_admission_counts_only_the_hits_of_the_admitted_prefix():
    """The slots a prefix of requests may evict are the unheld ones minus the cells that prefix itself
    hits.  A full cache whose cells later requests hit must not make the first request look as if it
    could never fit; the batch ends where the next request's hits would leave too few slots."""
    import collections
    p = _pyramid(4000, 700, 256, 4)                  # level 0: 16 x 3 cells of 256 x 256
    srv = _fake_server([p], slots=1, max_batch=8, budget=1 << 30, cache_bytes=0)
    cache = srv.caches[(0, 0)]
    n = cache.n_slots
    assert n == 8
    cache.assign(np.arange(8, 16), np.arange(8))     # cells 8..15 cached, cell 8 + k in slot k
    cache.stamp[:] = np.arange(8)
    reqs = [_req(0, 0.0, rect=(0, 0, 1024, 200))]    # cells 0..3: four misses
    reqs += [_req(k, 0.0, rect=(2048 + 256 * (k - 1), 0, 96, 64)) for k in range(1, 8)]   # hits cells 8..14
    slot = srv.slots[0]
    batch = srv._admit(collections.deque(reqs), slot)
    # request k >= 1 hits one more cached cell: 4 misses fit while 8 - k >= 4
    assert [r.rid for r in batch] == [0, 1, 2, 3, 4]
    got = cache.cached()
    assert all(c in got for c in range(0, 4)) and all(c in got for c in range(8, 12))
    assert not any(c in got for c in range(12, 16))   # the least recently used unhit cells were evicted
    _consistent(cache)


def test_resident_levels_need_no_tiles_and_copy_one_rectangle():
    import collections
    p = _pyramid(1000, 700, 256, 4)
    srv = _fake_server([p], resident_from=3)
    q = collections.deque([_req(1, 0.0, z=3, rect=(0, 0, 4, 4))])
    slot = srv.slots[0]
    batch = srv._admit(q, slot)
    assert [r.rid for r in batch] == [1] and slot.pairs == {} and slot.misses == {}
    c = srv._copies(batch, slot)
    assert len(c) == 1 and c["row_bytes"][0] == 12 and c["rows"][0] == 4


def test_levels_without_exact_footprints_are_resident():
    """Tile edge 96 is a multiple of 2^z only up to z = 5: finer levels are cached, z = 6 stays resident."""
    p = _pyramid(1000, 700, 96, 6)
    srv = _fake_server([p])
    cached, resident = srv._levels()
    assert cached == [(0, z) for z in range(6)] and resident == [(0, 6)]


def test_admit_stops_when_the_output_pool_is_empty():
    import collections
    srv = _fake_server([_pyramid(1000, 700, 256, 4)], max_batch=8, pool=2)
    q = collections.deque(_req(i, 0.0) for i in range(5))
    assert len(srv._admit(q, srv.slots[0])) == 2 and not srv.pool


def test_copies_assemble_each_viewport_exactly_once():
    """Simulated on the host: painting every cached tile with its own values and applying the copy
    rectangles gives the viewport of the whole level-z image."""
    import collections
    p = _pyramid(1000, 700, 128, 4)
    srv = _fake_server([p], max_batch=8, pool=8, budget=1 << 30, resident_from=3)
    rng = np.random.default_rng(2)
    reqs = []
    for i in range(8):
        z = int(rng.integers(0, 4))
        lw, lh = p.level_size(z)
        rw, rh = int(rng.integers(1, min(96, lw) + 1)), int(rng.integers(1, min(64, lh) + 1))
        reqs.append(_req(i, 0.0, z=z, rect=(int(rng.integers(0, lw - rw + 1)), int(rng.integers(0, lh - rh + 1)), rw, rh)))
    slot = srv.slots[0]
    batch = srv._admit(collections.deque(reqs), slot)
    assert len(batch) == 8
    lvl = {}
    for z in range(p.levels + 1):
        lw, lh = p.level_size(z)
        yy, xx = np.indices((lh, lw))
        lvl[z] = np.stack([(xx * 7 + yy * 3) % 251, (xx + yy * 11) % 253, (xx * yy) % 255], -1).astype(np.uint8)
    for (pi, z), img in srv.resident.items():
        img.copy_(torch_from(lvl[z]))
    # fill the caches' slots as the decode jobs would: each tile of the cell at its place in the slot
    for (pi, z), cache in srv.caches.items():
        got = cache.cached()
        if not got:
            continue
        cells, slots = np.array(list(got.keys())), np.array(list(got.values()))
        jobs = srv._cell_jobs(pi, z, cells, slots)
        for j in jobs:
            rx, ry, rw, rh = int(j["rx"]), int(j["ry"]), int(j["rw"]), int(j["rh"])
            dst = int(j["d_out"])
            for row in range(rh):
                src = np.ascontiguousarray(lvl[z][ry + row, rx:rx + rw])
                ctypes_move(dst + row * int(j["out_pitch_bytes"]), src.ctypes.data, src.nbytes)
    copies = srv._copies(batch, slot)
    for r in batch:
        r.buf.zero_()
    for c in copies:   # host replica of k_copy_rects on CPU tensors (byte addresses)
        src, dst = int(c["src"]), int(c["dst"])
        for row in range(int(c["rows"])):
            ctypes_move(dst + row * int(c["dst_pitch"]), src + row * int(c["src_pitch"]), int(c["row_bytes"]))
    for r in batch:
        rx, ry, rw, rh = r.rect
        assert np.array_equal(r.out.numpy(), lvl[r.z][ry:ry + rh, rx:rx + rw]), r.rid


def torch_from(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a))


def ctypes_move(dst, src, n):
    import ctypes
    ctypes.memmove(dst, src, n)


def test_cache_hits_after_a_batch_and_lru_eviction_respects_holds():
    p = _pyramid(1000, 700, 256, 4)
    srv = _fake_server([p], slots=1, max_batch=2, pool=4, budget=1 << 30, cache_bytes=0)
    cache = srv.caches[(0, 0)]
    n = cache.n_slots
    reqs = [_req(i, 0.0, rect=(0, 0, 96, 64)) for i in range(3)]
    done = srv.run(reqs)
    assert len(done) == 3
    assert cache.misses == 1 and cache.hits == 2          # tile 0 decoded once, then served from the cache
    assert not cache.holds.any() and np.all(cache.filler == -1) and not srv.inflight
    # victims: empty slots first, then the least recently used unheld tiles
    cache.drop(np.arange(n))
    tiles = np.arange(n, dtype=np.int64)
    cache.assign(tiles, np.arange(n))
    cache.stamp[:] = np.arange(100, 100 + n)              # slot 0 least recently used
    cache.holds[0] = 1                                    # held: not evictable
    v = cache.victims(2)
    assert sorted(v.tolist()) == [1, 2]
    cache.assign(np.array([n, n + 1]), v)
    assert cache.slot_of[1] == -1 and cache.slot_of[2] == -1 and cache.tile_of[0] == 0
    _consistent(cache)
    cache.holds[:] = 1
    assert cache.victims(1) is None                       # every slot held


def test_a_batch_reading_a_tile_another_batch_fills_waits_for_it():
    """Batch A (slot 0) decodes tile 0; batch B (slot 1), admitted while A is in flight, reads tile 0
    from the cache: B's stream waits for A's event, and B decodes nothing."""
    p = _pyramid(1000, 700, 256, 4)
    srv = _fake_server([p], slots=2, max_batch=1, budget=1 << 30, polls=50)
    done = srv.run([_req(0, 0.0), _req(1, 0.0)])
    assert len(done) == 2 and len(srv.launched) == 2
    a, b = srv.slots
    assert a.codec.decoded == [(0, [0])] and b.codec.decoded == []
    assert len(srv.waits) == 1


@pytest.mark.parametrize("slots,max_batch,pool", [(1, 1, 1), (2, 4, 8), (4, 32, 16)])
def test_run_serves_every_request_once(slots, max_batch, pool):
    pyrs = [_pyramid(5000, 3000, 256, 6), _pyramid(1000, 700, 256, 4)]
    reqs = serve.poisson_requests(20000.0, 120, pyrs, seed=7, view=(96, 64), zmax=4)
    srv = _fake_server(pyrs, slots=slots, max_batch=max_batch, pool=pool, budget=1 << 30, cache_bytes=0)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(120))
    assert all(r.done >= r.arrival for r in done)
    # every batch within the limits, every request in exactly one batch, pool buffers all returned
    assert all(1 <= len(b) <= max_batch for b in srv.launched)
    assert sorted(i for b in srv.launched for i in b) == list(range(120))
    assert len(srv.pool) == pool
    assert srv.n_batches == len(srv.launched) and sum(srv.batch_sizes) == 120
    # requests are admitted in arrival order; every hold released
    order = [i for b in srv.launched for i in b]
    arrival = {r.rid: r.arrival for r in reqs}
    assert all(arrival[a] <= arrival[b] for a, b in zip(order, order[1:]))
    for c in srv.caches.values():
        assert not c.holds.any() and np.all(c.filler == -1)
        _consistent(c)
    assert not srv.inflight
    # the tiles decoded are exactly those of the missing cells, each once per call
    assert srv.cell_tiles == sum(len(t) for s in srv.slots for _, t in s.codec.decoded)
    assert all(len(set(t)) == len(t) for s in srv.slots for _, t in s.codec.decoded)
    assert sum(c.misses for c in srv.caches.values()) <= srv.cell_tiles


def test_run_isolates_a_failed_request_in_its_batch():
    """A batch whose device status reports a data error: its decoded tiles leave the cache and only the
    request over the bad tile is marked."""
    pyrs = [_pyramid(2048, 1024, 256, 3)]
    srv = _fake_server(pyrs, slots=1, max_batch=8, budget=1 << 40, pool=16)
    bad_tile = 9            # grid 8 x 4: row 1, column 1 (pixels 256..511 at level 0)
    for s in srv.slots:
        s.codec.bad = frozenset([bad_tile])
    reqs = [_req(0, 0.0, rect=(0, 0, 96, 64)), _req(1, 0.0, rect=(300, 300, 96, 64)),
            _req(2, 0.0, rect=(1200, 700, 96, 64)), _req(3, 0.0, rect=(600, 40, 96, 64))]
    done = srv.run(reqs)
    assert len(srv.launched) == 1 and sorted(srv.launched[0]) == [0, 1, 2, 3]
    errs = {r.rid: r.error for r in done}
    assert errs == {0: None, 1: "ISX_ERR_CORRUPT", 2: None, 3: None}
    assert not srv.caches[(0, 0)].cached()                   # the failed batch's tiles were dropped


def test_a_batch_reading_tiles_of_a_failed_batch_is_checked_too():
    """Batch A (slot 0) decodes a bad tile; batch B (slot 1), admitted while A is in flight, reads it
    from the cache.  When A fails, B is marked, and on completion its request is decoded again alone
    and reports the error itself."""
    pyrs = [_pyramid(2048, 1024, 256, 3)]
    srv = _fake_server(pyrs, slots=2, max_batch=1, budget=1 << 40, pool=4, polls=5)
    for s in srv.slots:
        s.codec.bad = frozenset([0])
    done = srv.run([_req(0, 0.0), _req(1, 0.0)])
    errs = {r.rid: r.error for r in done}
    assert errs == {0: "ISX_ERR_CORRUPT", 1: "ISX_ERR_CORRUPT"}
    assert srv.slots[1].codec.decoded[-1] == (0, [0])        # B's request was decoded again alone
