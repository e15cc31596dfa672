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


# ---------------------------------------------------------------- the batching loop, with fakes
# Server._admit and Server.run only plan and keep time; the decode itself is the library's.  A fake codec
# reports scratch sizes, CPU tensors stand in for the output pool, and a fake launch completes each batch
# after a few polls, so the continuous-batching logic runs on the CPU.

class _FakeCodec:
    def __init__(self, per_tile):
        self.per_tile = per_tile
        self.calls = 0

    def decode_jobs_scratch(self, tiles, jobs, level=0, drop_lsb_planes=0):
        self.calls += 1
        return self.per_tile * len(jobs)

    # the device status word: a batch containing a job of a tile in `bad` reports ISX_ERR_CORRUPT
    bad = frozenset()
    pending = 0

    def decode_jobs_array(self, stream_buf, offsets, tiles, jobs, level=0, drop_lsb_planes=0, stream=None):
        if any(int(t) in self.bad for t in jobs["tile"]):
            self.pending = 3

    def sync_status(self, stream=None):
        st, self.pending = self.pending, 0
        return st


class _FakeEvent:
    def __init__(self, polls):
        self.left = polls

    def query(self):
        self.left -= 1
        return self.left <= 0


def _fake_server(pyrs, slots=2, max_batch=4, budget=10_000, pool=8, per_tile=100, resident=(), polls=3):
    import torch
    srv = serve.Server.__new__(serve.Server)
    srv.torch = torch
    srv.pyr = list(pyrs)
    srv.max_batch, srv.budget = max_batch, budget
    srv.slots = [serve._Slot(_FakeCodec(per_tile), None) for _ in range(slots)]
    srv.pool = __import__("collections").deque(torch.zeros((64, 96, 3), dtype=torch.uint8) for _ in range(pool))
    srv.out_shape = (64, 96, 3)
    srv.keep_outputs = False
    srv.resident = {k: torch.zeros((4, 4, 3), dtype=torch.uint8) for k in resident}
    srv.launched = []

    def launch(slot, batch):
        srv.launched.append([r.rid for r in batch])
        for r in batch:
            if r.jobs is not None and len(r.jobs):
                slot.codec.decode_jobs_array(None, None, None, r.jobs, r.z)
        slot.batch, slot.event, slot.busy = batch, _FakeEvent(polls), True
    srv._launch = launch
    return srv


def _req(rid, t, pi=0, z=0, rect=(0, 0, 96, 64)):
    return serve.Request(rid, t, pi, z, rect)


def test_admit_takes_requests_in_order_up_to_the_batch_size():
    import collections
    srv = _fake_server([_pyramid(1000, 700, 256, 4)], max_batch=3)
    q = collections.deque(_req(i, 0.0) for i in range(5))
    batch = srv._admit(q, srv.slots[0])
    assert [r.rid for r in batch] == [0, 1, 2] and [r.rid for r in q] == [3, 4]
    assert len(srv.pool) == 8 - 3
    for r in batch:
        assert r.out.shape == (64, 96, 3) and r.out.data_ptr() == r.buf.data_ptr()
        # the jobs are the tiles meeting the viewport, all writing into this request's buffer
        assert sorted(r.jobs["tile"].tolist()) == [0]
        assert set(r.jobs["d_out"].tolist()) == {r.out.data_ptr()}


def test_admit_stops_at_the_scratch_budget_of_a_group():
    import collections
    p = _pyramid(1000, 700, 256, 4)
    # each request meets 4 tiles (a 300 x 300 viewport at level 0): 400 bytes of scratch; budget 1000
    srv = _fake_server([p], max_batch=8, budget=1000)
    q = collections.deque(_req(i, 0.0, rect=(200, 200, 300, 300)) for i in range(4))
    batch = srv._admit(q, srv.slots[0])
    assert len(batch) == 2 and len(q) == 2
    # another (pyramid, level) group has a budget of its own
    q = collections.deque([_req(10, 0.0, z=0, rect=(200, 200, 300, 300)), _req(11, 0.0, z=1, rect=(0, 0, 90, 60)),
                           _req(12, 0.0, z=0, rect=(200, 200, 300, 300)), _req(13, 0.0, z=0, rect=(200, 200, 300, 300))])
    batch = srv._admit(q, srv.slots[1])
    assert [r.rid for r in batch] == [10, 11, 12] and [r.rid for r in q] == [13]


def test_admit_refuses_a_request_beyond_the_budget_and_skips_resident_levels():
    import collections
    p = _pyramid(1000, 700, 256, 4)
    srv = _fake_server([p], budget=300, resident=[(0, 3)])
    with pytest.raises(RuntimeError, match="more than the slot budget"):
        srv._admit(collections.deque([_req(0, 0.0, rect=(200, 200, 300, 300))]), srv.slots[0])
    # a request at a resident level needs no decode scratch and no jobs
    q = collections.deque([_req(1, 0.0, z=3, rect=(0, 0, 4, 4))])
    batch = srv._admit(q, srv.slots[0])
    assert [r.rid for r in batch] == [1] and batch[0].jobs is None


def test_admit_stops_when_the_output_pool_is_empty():
    import collections
    srv = _fake_server([_pyramid(1000, 700, 256, 4)], max_batch=8, pool=2)
    q = collections.deque(_req(i, 0.0) for i in range(5))
    assert len(srv._admit(q, srv.slots[0])) == 2 and not srv.pool


@pytest.mark.parametrize("slots,max_batch,pool", [(1, 1, 1), (2, 4, 8), (4, 32, 16)])
def test_run_serves_every_request_once(slots, max_batch, pool):
    pyrs = [_pyramid(5000, 3000, 256, 6), _pyramid(1000, 700, 256, 4)]
    reqs = serve.poisson_requests(20000.0, 120, pyrs, seed=7, view=(96, 64), zmax=4)
    srv = _fake_server(pyrs, slots=slots, max_batch=max_batch, pool=pool, budget=1 << 30)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(120))
    assert all(r.done >= r.arrival for r in done)
    # every batch within the limits, every request in exactly one batch, pool buffers all returned
    assert all(1 <= len(b) <= max_batch for b in srv.launched)
    assert sorted(i for b in srv.launched for i in b) == list(range(120))
    assert len(srv.pool) == pool
    assert srv.n_batches == len(srv.launched) and sum(srv.batch_sizes) == 120
    # requests are admitted in arrival order
    order = [i for b in srv.launched for i in b]
    arrival = {r.rid: r.arrival for r in reqs}
    assert all(arrival[a] <= arrival[b] for a, b in zip(order, order[1:]))


def test_run_isolates_a_failed_request_in_its_batch():
    """A batch whose device status reports a data error: only the request over the bad tile is marked."""
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
