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
