"""Viewport serving over a device-resident compressed pyramid.

A pyramid is one image encoded as tiles (the stream, its tile offsets and
the tile descriptors stay in device memory); a request asks for a viewport
(a rectangle of pixels at one resolution level z, Sec. 4: a decode at level
z reads only the LL band and the levels above z).  The server runs
continuous batching: requests that arrive while others are on the GPU are
queued, and whenever one of its slots (a CUDA stream with its own library
context) is free it takes the queued requests, as many as its memory
budgets admit, and serves them with a few launches:

- the coarse levels (z >= resident_from) of each pyramid are decoded once,
  whole, at start and kept in device memory (about 1/48 of the image);
- the finer levels are served from a cache of decoded cells (a cell is a
  tile-edge square of level-z pixels, assembled from the 2^z x 2^z tiles
  it covers, so that a viewport meets about as many cells at any level as
  it meets tiles at level 0; one buffer of fixed slots per pyramid and
  level, least recently used cells evicted): a batch decodes only its
  missing cells, each tile whole into its place in the cell's slot (one
  isx_decode_jobs call per pyramid and level);
- every viewport is then assembled from cached cells and resident levels
  by one isx_copy_rects launch for the whole batch.

A batch is admitted while its missing cells find free or evictable slots
and their decode scratch fits the slot's budget.  A cached cell that a
batch in flight on another stream is still filling makes the batch's
stream wait for that batch's event (after the batch's own decodes, which
write only slots no batch in flight touches).  Each request's latency runs
from its arrival to the moment the host sees its batch's completion event.

All decoding and copying happens in the library's kernels; this module
only plans batches (which cells meet which viewport, which are cached) and
keeps time.  The plan of a batch is vectorised over its requests: the
cache's maps are arrays, so that planning costs a few dozen array
operations a batch, not a Python step a tile.
"""
from __future__ import annotations

import collections
import itertools
import time
from dataclasses import dataclass, field

import numpy as np

from . import isx


@dataclass
class Pyramid:
    """A tiled, encoded image resident on the device."""
    width: int
    height: int
    tile: int                 # tile edge at level 0 (edge tiles are smaller)
    levels: int               # wavelet levels of every tile
    channels: int
    bits: int
    stream: object            # uint8 CUDA tensor
    offsets: object           # int64 CUDA tensor, n_tiles + 1
    tiles: isx.TileArray
    grid_w: int = 0
    grid_h: int = 0

    def __post_init__(self):
        self.grid_w = -(-self.width // self.tile)
        self.grid_h = -(-self.height // self.tile)

    def level_size(self, z: int):
        return isx.level_dim(self.width, z), isx.level_dim(self.height, z)

    def exact_at(self, z: int) -> bool:
        """Tile footprints at level z tile the level exactly (the tile edge is a multiple of 2^z)."""
        return (self.tile >> z) << z == self.tile

    def tiles_meeting(self, z: int, rx: int, ry: int, rw: int, rh: int) -> np.ndarray:
        """Indices of the tiles whose level-z footprint meets the rectangle (row-major grid)."""
        if self.exact_at(z):
            # tile (i, j) covers [j * s, (j + 1) * s) at level z when the tile edge is a multiple of 2^z
            s = self.tile >> z
            c0, c1 = max(0, rx // s), min(self.grid_w - 1, (rx + rw - 1) // s)
            r0, r1 = max(0, ry // s), min(self.grid_h - 1, (ry + rh - 1) // s)
        else:
            c0, c1, r0, r1 = 0, self.grid_w - 1, 0, self.grid_h - 1   # the library skips tiles outside the rectangle
        cols = np.arange(c0, c1 + 1, dtype=np.int32)
        rows = np.arange(r0, r1 + 1, dtype=np.int32)
        return (rows[:, None] * self.grid_w + cols[None, :]).reshape(-1)

    def tile_rects(self, z: int, idx: np.ndarray):
        """Level-z footprint (x, y, w, h) of tiles `idx` (row-major grid), as four int64 arrays."""
        idx = np.asarray(idx, dtype=np.int64)
        gx, gy = idx % self.grid_w, idx // self.grid_w
        x0, y0 = gx * self.tile, gy * self.tile
        tw, th = np.minimum(self.tile, self.width - x0), np.minimum(self.tile, self.height - y0)
        return x0 >> z, y0 >> z, ((tw - 1) >> z) + 1, ((th - 1) >> z) + 1

    # Cells: the unit of the decoded-tile cache.  At an exact level z a cell is a tile-edge square of
    # level-z pixels (cell (cx, cy) covers [cx * tile, (cx + 1) * tile) x [cy * tile, (cy + 1) * tile),
    # clipped to the level), assembled from the 2^z x 2^z tiles whose footprints it covers, so that a
    # viewport meets about as many cells at every level as it meets tiles at level 0.
    def cell_grid(self, z: int):
        lw, lh = self.level_size(z)
        return -(-lw // self.tile), -(-lh // self.tile)

    def cell_pairs(self, z: int, rects: np.ndarray):
        """(rect index, cell index) int64 arrays of every cell meeting each rectangle (rects (n, 4) int64 at
        level z), rectangle by rectangle, cells row-major within each."""
        cw, ch = self.cell_grid(z)
        s = self.tile
        rx, ry, rw, rh = (rects[:, k] for k in range(4))
        c0, c1 = np.maximum(rx // s, 0), np.minimum((rx + rw - 1) // s, cw - 1)
        r0, r1 = np.maximum(ry // s, 0), np.minimum((ry + rh - 1) // s, ch - 1)
        nc, nr = np.maximum(c1 - c0 + 1, 0), np.maximum(r1 - r0 + 1, 0)
        cnt = nc * nr
        req = np.repeat(np.arange(len(rects), dtype=np.int64), cnt)
        k = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        ncr = nc[req]
        return req, (r0[req] + k // ncr) * cw + c0[req] + k % ncr

    def cell_rects(self, z: int, cells: np.ndarray):
        """Level-z extent (x, y, w, h) of cells `cells`, as four int64 arrays."""
        cw, _ = self.cell_grid(z)
        lw, lh = self.level_size(z)
        cells = np.asarray(cells, dtype=np.int64)
        x0, y0 = (cells % cw) * self.tile, (cells // cw) * self.tile
        return x0, y0, np.minimum(self.tile, lw - x0), np.minimum(self.tile, lh - y0)

    def cell_tiles(self, z: int, cells: np.ndarray):
        """(cell position in `cells`, tile index) int64 arrays of the tiles each cell is assembled from."""
        cw, _ = self.cell_grid(z)
        cells = np.asarray(cells, dtype=np.int64)
        k = 1 << z
        gx0, gy0 = (cells % cw) * k, (cells // cw) * k
        nc, nr = np.minimum(k, self.grid_w - gx0), np.minimum(k, self.grid_h - gy0)
        cnt = nc * nr
        pos = np.repeat(np.arange(len(cells), dtype=np.int64), cnt)
        i = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        ncp = nc[pos]
        return pos, (gy0[pos] + i // ncp) * self.grid_w + gx0[pos] + i % ncp


@dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the run
    pyramid: int              # index into the server's pyramids
    z: int
    rect: tuple               # (rx, ry, rw, rh) at level z
    out: object = None        # CUDA tensor view (rh, rw, channels) once admitted
    done: float = float("nan")
    buf: object = None        # the pooled output buffer `out` views
    result: object = None     # host copy of the output (Server(keep_outputs=True))
    error: object = None      # status name when the decode of this request reported a data error


@dataclass
class _Slot:
    codec: isx.Codec
    stream: object
    busy: bool = False
    batch: list = field(default_factory=list)
    event: object = None
    bid: int = 0                                 # id of the batch in flight
    held: list = field(default_factory=list)     # (cache, slots) the batch reads, each slot once
    filled: list = field(default_factory=list)   # (cache, slots) the batch decodes into
    misses: dict = field(default_factory=dict)   # (pyramid, level) -> (cells, slots) the batch decodes
    pairs: dict = field(default_factory=dict)    # (pyramid, level) -> (request index, cell, slot) it copies
    tainted: bool = False                        # it read cells that a failed batch decoded


class TileCache:
    """Decoded cells of one pyramid at one level z (Pyramid.cell_grid): `n_slots` fixed slots of one
    device buffer (tile edge squared x channels bytes each), least recently used cells evicted.  The
    maps are arrays: slot_of (cell -> slot, -1 when not cached), tile_of (slot -> cell, -1 when empty),
    stamp (the last batch that used the slot, -1 when empty), holds (batches in flight that read or fill
    the slot) and filler (the batch in flight filling the slot, -1 when none)."""

    def __init__(self, torch, n_slots: int, edge: int, channels: int, n_tiles: int, device):
        self.edge, self.channels = edge, channels
        self.buf = torch.empty((max(n_slots, 1), edge, edge, channels), dtype=torch.uint8, device=device)
        self.n_slots = n_slots
        self.pitch = edge * channels
        self.slot_bytes = edge * edge * channels
        self.base = self.buf.data_ptr()
        self.slot_of = np.full(n_tiles, -1, np.int64)
        self.tile_of = np.full(n_slots, -1, np.int64)
        self.stamp = np.full(n_slots, -1, np.int64)
        self.holds = np.zeros(n_slots, np.int64)
        self.filler = np.full(n_slots, -1, np.int64)
        self.hits = self.misses = 0

    def cached(self) -> dict:
        """{cell: slot} of the cached cells."""
        s = np.flatnonzero(self.tile_of >= 0)
        return dict(zip(self.tile_of[s].tolist(), s.tolist()))

    def victims(self, k: int):
        """k slots for new tiles: empty slots first, then the least recently used cached tiles that no
        batch in flight holds; None when fewer than k are unheld."""
        cand = np.flatnonzero(self.holds == 0)
        if len(cand) < k:
            return None
        if 0 < k < len(cand):
            cand = cand[np.argpartition(self.stamp[cand], k - 1)[:k]]
        return cand[:k]

    def assign(self, tiles: np.ndarray, slots: np.ndarray):
        """Slots `slots` now hold `tiles` (not cached before); the tiles they held leave the cache."""
        old = self.tile_of[slots]
        self.slot_of[old[old >= 0]] = -1
        self.tile_of[slots] = tiles
        self.slot_of[tiles] = slots

    def drop(self, slots: np.ndarray):
        """Forget the tiles in `slots` (their decode failed)."""
        slots = np.asarray(slots, dtype=np.int64)
        t = self.tile_of[slots]
        mine = t >= 0
        self.slot_of[t[mine]] = -1
        self.tile_of[slots] = -1
        self.stamp[slots] = -1

    def ptr(self, s):
        return self.base + np.asarray(s, dtype=np.int64) * self.slot_bytes


class Server:
    """Continuous-batching viewport server.

    slots:            concurrent batches (each a CUDA stream and a library context)
    max_batch:        most requests in one batch
    scratch_budget:   device scratch per slot (bytes); a batch's missing tiles of one
                      (pyramid, level) are decoded by one call whose scratch must fit it,
                      and the slots' scratch is reserved up front, so serving allocates
                      no device memory
    resident_from:    levels z >= resident_from are decoded once, whole, at start (so is
                      every level whose tile footprints are not exact: tile edge not a
                      multiple of 2^z)
    cache_bytes:      device memory of the decoded caches of the finer levels (cells of
                      tile-edge squares of level-z pixels), split between pyramids and
                      levels by their decoded size
    """

    def __init__(self, pyramids, device=0, slots=4, max_batch=32, scratch_budget=1 << 30, out_shape=None, keep_outputs=False,
                 resident_from=None, cache_bytes=2 << 30):
        import torch
        self.torch = torch
        self.pyr = list(pyramids)
        if any(p.bits > 8 for p in self.pyr):
            raise ValueError("the server's output buffers hold 8-bit samples")
        self.max_batch = max_batch
        self.budget = scratch_budget
        self.slots = []
        for _ in range(slots):
            c = isx.Codec(device, hbm_budget_bytes=scratch_budget)
            c.reserve_scratch(scratch_budget)
            self.slots.append(_Slot(c, torch.cuda.Stream(device=device)))
        self.device = device
        # output buffers, one per request that can be in flight
        h, w = out_shape if out_shape else (1080, 1920)
        ch = max(p.channels for p in self.pyr)
        self.pool = collections.deque(torch.empty((h, w, ch), dtype=torch.uint8, device=f"cuda:{device}")
                                      for _ in range(slots * max_batch))
        self.out_shape = (h, w, ch)
        self.keep_outputs = keep_outputs   # copy each result before its buffer is reused (tests)
        self.resident_from = resident_from if resident_from is not None else max(p.levels for p in self.pyr) + 1
        self._init_state()
        # Decoded levels kept resident: each is decoded once, whole, here;
        # requests at those levels are crops of it.
        self.resident = {}
        with isx.Codec(device) as c:
            for pi, z in self._levels()[1]:
                p = self.pyr[pi]
                lw, lh = p.level_size(z)
                img = torch.empty((lh, lw, p.channels), dtype=torch.uint8, device=f"cuda:{device}")
                jobs = np.zeros(len(p.tiles), isx.JOB_DTYPE)
                jobs["tile"] = np.arange(len(p.tiles), dtype=np.int32)
                jobs["rw"], jobs["rh"] = lw, lh
                jobs["d_out"] = img.data_ptr()
                jobs["out_pitch_bytes"] = img.stride(0)
                c.decode_jobs_array(p.stream, p.offsets, p.tiles, jobs, z)
                if c.sync_status() != 0:
                    raise RuntimeError(f"decode of resident level {z} failed")
                self.resident[(pi, z)] = img
        self._make_caches(cache_bytes, f"cuda:{device}", self.slots[0].codec)

    def _init_state(self):
        self.inflight = {}                   # batch id -> completion event, while the batch is in flight
        self._ids = itertools.count(1)
        self.n_batches, self.batch_sizes, self.elapsed = 0, [], 0.0

    def _levels(self):
        """([(pyramid, z)] served from tile caches, [(pyramid, z)] kept resident)."""
        cached, resident = [], []
        for pi, p in enumerate(self.pyr):
            for z in range(p.levels + 1):
                (cached if z < self.resident_from and p.exact_at(z) else resident).append((pi, z))
        return cached, resident

    def _make_caches(self, cache_bytes, device, codec):
        """One TileCache per pyramid and cached level, and each one's decode-scratch estimate: a linear
        fit through the scratch of decoding 1 and 2 whole interior cells, with a fifth added."""
        self.caches, self.scratch_fit = {}, {}
        vw, vh = self.out_shape[1], self.out_shape[0]
        levels = self._levels()[0]
        sizes = {(pi, z): self.pyr[pi].level_size(z)[0] * self.pyr[pi].level_size(z)[1] * self.pyr[pi].channels
                 for pi, z in levels}
        total = max(sum(sizes.values()), 1)
        for pi, z in levels:
            p = self.pyr[pi]
            edge = p.tile
            slot_bytes = edge * edge * p.channels
            # at least every slot's worth of batches of the largest request, so admission always progresses
            per_req = (-(-vw // edge) + 1) * (-(-vh // edge) + 1)
            n = max(int(cache_bytes * sizes[(pi, z)] / total) // slot_bytes, per_req * max(len(self.slots), 1) + per_req)
            cw, ch = p.cell_grid(z)
            n = min(n, cw * ch)
            self.caches[(pi, z)] = TileCache(self.torch, n, edge, p.channels, cw * ch, device)
            ci = (ch // 2) * cw + max(cw // 2 - 1, 0)
            s1 = codec.decode_jobs_scratch(p.tiles, self._cell_jobs(pi, z, [ci], [0]), z)
            s2 = codec.decode_jobs_scratch(p.tiles, self._cell_jobs(pi, z, [ci, min(ci + 1, cw * ch - 1)], [0, 0]), z)
            per = max(s2 - s1, 1)
            self.scratch_fit[(pi, z)] = (max(s1 - per, 0) * 1.2, per * 1.2)

    def close(self):
        for s in self.slots:
            s.codec.close()
        self.slots, self.caches, self.resident, self.pool = [], {}, {}, collections.deque()

    # ------------------------------------------------------------ planning
    def _cell_jobs(self, pi, z, cells, slots) -> np.ndarray:
        """Decode jobs assembling cells `cells` at level z into cache slots `slots`: one job per tile of
        each cell, its whole level-z footprint written at its place in the slot (a placeholder pointer
        while the caches are being made: scratch estimates only)."""
        p = self.pyr[pi]
        cells = np.asarray(cells, dtype=np.int64)
        pos, tiles = p.cell_tiles(z, cells)
        fx, fy, fw, fh = p.tile_rects(z, tiles)
        cx, cy, _, _ = p.cell_rects(z, cells[pos])
        jobs = np.zeros(len(tiles), isx.JOB_DTYPE)
        jobs["tile"] = tiles
        jobs["rx"], jobs["ry"], jobs["rw"], jobs["rh"] = fx, fy, fw, fh
        cache = self.caches.get((pi, z))
        if cache is not None:
            slots = np.asarray(slots, dtype=np.int64)
            jobs["d_out"] = cache.ptr(slots[pos]) + (fy - cy) * cache.pitch + (fx - cx) * p.channels
            jobs["out_pitch_bytes"] = cache.pitch
        else:
            jobs["d_out"] = 1
            jobs["out_pitch_bytes"] = p.tile * p.channels
        return jobs

    def _admit(self, queue, slot: _Slot):
        """Takes the longest run of queued requests (in arrival order, at most max_batch, one output buffer
        each) whose distinct missing cells of every (pyramid, level) find unheld slots in that level's cache
        and whose decode scratch fits the slot's budget.  Returns the batch; its plan is left in slot.held,
        slot.filled, slot.misses and slot.pairs.  A request that could never be admitted raises."""
        slot.held, slot.filled, slot.misses, slot.pairs = [], [], {}, {}
        n = min(len(queue), self.max_batch, len(self.pool))
        if n == 0:
            return []
        cand = list(itertools.islice(queue, n))
        keyc = np.fromiter((r.pyramid * 64 + r.z for r in cand), np.int64, n)
        rects = np.array([r.rect for r in cand], dtype=np.int64).reshape(n, 4)
        limit, groups, blocked = n, [], []
        for kc in np.unique(keyc).tolist():
            key = (kc // 64, kc % 64)
            if key in self.resident:
                continue
            cache = self.caches[key]
            sel = np.flatnonzero(keyc == kc)
            ridx, tiles = self.pyr[key[0]].cell_pairs(key[1], rects[sel])
            ridx = sel[ridx]
            slots = cache.slot_of[tiles]
            miss = slots < 0
            _, first = np.unique(tiles[miss], return_index=True)
            need = np.cumsum(np.bincount(ridx[miss][first], minlength=n))   # distinct missing cells of requests 0..k
            # unheld slots the missing cells may take: every unheld slot but the cells requests 0..k hit
            hr, hs = ridx[~miss], slots[~miss]
            unheld = cache.holds[hs] == 0
            _, first = np.unique(hs[unheld], return_index=True)
            free = int(np.count_nonzero(cache.holds == 0)) - np.cumsum(np.bincount(hr[unheld][first], minlength=n))
            base, per = self.scratch_fit[key]
            fits = int((self.budget - base) // per) if self.budget >= base else -1
            over = np.flatnonzero((need > 0) & ((need > free) | (need > fits)))
            if len(over):
                limit = min(limit, int(over[0]))
                if over[0] == 0:
                    blocked.append((key, cache, int(np.count_nonzero(ridx == 0))))
            groups.append((key, cache, ridx, tiles, slots))
        if limit == 0:
            for key, cache, n_tiles in blocked:
                # nothing in flight holds this cache: the first request cannot fit even alone
                if not cache.holds.any():
                    raise RuntimeError(f"request {cand[0].rid} needs more than the slot budget {self.budget} or the cache "
                                       f"of level {key[1]} ({cache.n_slots} slots) for its {n_tiles} cells")
            return []
        bid = next(self._ids)
        slot.bid = bid
        for key, cache, ridx, tiles, slots in groups:
            keep = ridx < limit
            if not keep.any():
                continue
            ridx, tiles, slots = ridx[keep], tiles[keep], slots[keep]
            miss = slots < 0
            used = np.unique(slots[~miss])
            cache.holds[used] += 1
            new = np.unique(tiles[miss])
            if len(new):
                vict = cache.victims(len(new))
                if vict is None:        # the admission count above leaves enough unheld slots (exactly)
                    raise AssertionError("tile cache admission miscounted its free slots")
                cache.assign(new, vict)
                cache.holds[vict] += 1
                cache.filler[vict] = bid
                slots = cache.slot_of[tiles]
                slot.filled.append((cache, vict))
                slot.misses[key] = (new, vict)
                used = np.concatenate([used, vict])
            cache.stamp[used] = bid
            cache.hits += len(tiles) - len(new)
            cache.misses += len(new)
            slot.held.append((cache, used))
            slot.pairs[key] = (ridx, tiles, slots)
        batch = cand[:limit]
        for r in batch:
            queue.popleft()
            buf = self.pool.popleft()
            r.out, r.buf = buf[:r.rect[3], :r.rect[2], :self.pyr[r.pyramid].channels], buf
        return batch

    def _copies(self, batch, slot: _Slot) -> np.ndarray:
        """The batch's copy rectangles: each request's crop of a resident level, and its part of every
        cached tile it meets (the plan's pairs)."""
        n = len(batch)
        out_ptr = np.fromiter((r.buf.data_ptr() for r in batch), np.int64, n)
        out_pitch = np.fromiter((r.buf.stride(0) for r in batch), np.int64, n)
        rects = np.array([r.rect for r in batch], dtype=np.int64).reshape(n, 4)
        parts = []
        res = [(i, self.resident[(r.pyramid, r.z)], self.pyr[r.pyramid].channels) for i, r in enumerate(batch)
               if (r.pyramid, r.z) in self.resident]
        if res:
            i = np.array([k for k, _, _ in res], dtype=np.int64)
            src = np.array([img.data_ptr() for _, img, _ in res], dtype=np.int64)
            pitch = np.array([img.stride(0) for _, img, _ in res], dtype=np.int64)
            C = np.array([c for _, _, c in res], dtype=np.int64)
            rx, ry, rw, rh = (rects[i, k] for k in range(4))
            c = np.zeros(len(res), isx.COPY_DTYPE)
            c["src"] = src + ry * pitch + rx * C
            c["src_pitch"], c["dst"], c["dst_pitch"] = pitch, out_ptr[i], out_pitch[i]
            c["row_bytes"], c["rows"] = rw * C, rh
            parts.append(c)
        for (pi, z), (ridx, tiles, slots) in slot.pairs.items():
            p, cache = self.pyr[pi], self.caches[(pi, z)]
            C = p.channels
            fx, fy, fw, fh = p.cell_rects(z, tiles)
            rx, ry, rw, rh = (rects[ridx, k] for k in range(4))
            x0, x1 = np.maximum(fx, rx), np.minimum(fx + fw, rx + rw)
            y0, y1 = np.maximum(fy, ry), np.minimum(fy + fh, ry + rh)
            c = np.zeros(len(ridx), isx.COPY_DTYPE)
            c["src"] = cache.base + slots * cache.slot_bytes + (y0 - fy) * cache.pitch + (x0 - fx) * C
            c["src_pitch"] = cache.pitch
            c["dst"] = out_ptr[ridx] + (y0 - ry) * out_pitch[ridx] + (x0 - rx) * C
            c["dst_pitch"] = out_pitch[ridx]
            c["row_bytes"], c["rows"] = (x1 - x0) * C, y1 - y0
            parts.append(c)
        return np.concatenate(parts) if parts else np.zeros(0, isx.COPY_DTYPE)

    def _record(self, stream):
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return ev

    def _wait(self, stream, event):
        stream.wait_event(event)

    def _launch(self, slot: _Slot, batch):
        stream = slot.stream
        # the missing cells first: their slots are held by no batch in flight, so nothing to wait for
        for (pi, z), (cells, slots) in slot.misses.items():
            p = self.pyr[pi]
            slot.codec.decode_jobs_array(p.stream, p.offsets, p.tiles, self._cell_jobs(pi, z, cells, slots), z, 0, stream)
        # cached cells this batch reads that a batch in flight on another stream is still filling
        waits = set()
        for cache, used in slot.held:
            f = cache.filler[used]
            waits.update(np.unique(f[(f >= 0) & (f != slot.bid)]).tolist())
        for b in sorted(waits):
            self._wait(stream, self.inflight[b])
        copies = self._copies(batch, slot)
        if len(copies):
            slot.codec.copy_rects(copies, stream)
        ev = self._record(stream)
        self.inflight[slot.bid] = ev
        slot.batch, slot.event, slot.busy = batch, ev, True

    def _release(self, slot: _Slot):
        """The slot's batch is done: its filled slots are ready, its holds end."""
        for cache, used in slot.held:
            cache.holds[used] -= 1
        for cache, vict in slot.filled:
            cache.filler[vict[cache.filler[vict] == slot.bid]] = -1
        self.inflight.pop(slot.bid, None)
        slot.held, slot.filled, slot.misses, slot.pairs = [], [], {}, {}

    def _isolate_failures(self, slot: _Slot, batch):
        """A batch whose decode reported a data error (a corrupt stream, a capacity or consistency
        status), or that read tiles such a batch decoded: the tiles it decoded leave the caches (batches
        in flight that read them are marked to be checked the same way), and each of its requests is
        decoded again alone (a region decode into its buffer), so that only the requests whose own decode
        fails get `error` set; the others keep a correct result."""
        for cache, vict in slot.filled:
            cache.drop(vict)
            for other in self.slots:
                if other is not slot and other.busy and any(c is cache and np.isin(u, vict).any() for c, u in other.held):
                    other.tainted = True
        for r in batch:
            key = (r.pyramid, r.z)
            if key in self.resident:
                continue
            p = self.pyr[r.pyramid]
            rx, ry, rw, rh = r.rect
            idx = p.tiles_meeting(r.z, rx, ry, rw, rh)
            jobs = np.zeros(len(idx), isx.JOB_DTYPE)
            jobs["tile"] = idx
            jobs["rx"], jobs["ry"], jobs["rw"], jobs["rh"] = rx, ry, rw, rh
            jobs["d_out"] = r.buf.data_ptr()
            jobs["out_pitch_bytes"] = r.buf.stride(0)
            slot.codec.decode_jobs_array(p.stream, p.offsets, p.tiles, jobs, r.z, 0, slot.stream)
            st = slot.codec.sync_status(slot.stream)
            r.error = None if st == 0 else isx.STATUS_NAMES.get(st, st)

    # ------------------------------------------------------------ the loop
    def run(self, requests):
        """Serves requests (sorted by arrival, seconds from now); returns them with `done` set."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue = collections.deque()
        done = []
        t0 = time.perf_counter()
        n_batches, batch_sizes = 0, []
        while pending or queue or any(s.busy for s in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            progressed = False
            for s in self.slots:
                if s.busy and s.event.query():
                    # the stream is idle: reading the slot's device status word costs no wait
                    if s.codec.sync_status(s.stream) != 0 or s.tainted:
                        self._isolate_failures(s, s.batch)
                    self._release(s)
                    t = time.perf_counter() - t0
                    for r in s.batch:
                        r.done = t
                        if self.keep_outputs:
                            r.result = r.out.cpu().numpy()
                        done.append(r)
                        self.pool.append(r.buf)
                    s.busy, s.batch, s.event, s.tainted = False, [], None, False
                    progressed = True
            for s in self.slots:
                if not s.busy and queue and self.pool:
                    batch = self._admit(queue, s)
                    if batch:
                        self._launch(s, batch)
                        n_batches += 1
                        batch_sizes.append(len(batch))
                        progressed = True
            if not progressed:
                if pending and not queue and not any(s.busy for s in self.slots):
                    time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
        self.n_batches, self.batch_sizes = n_batches, batch_sizes
        self.elapsed = time.perf_counter() - t0
        return done

    def cache_stats(self) -> dict:
        hits = sum(c.hits for c in self.caches.values())
        misses = sum(c.misses for c in self.caches.values())
        return {"tile_hits": hits, "tile_misses": misses, "hit_rate": round(hits / max(hits + misses, 1), 4),
                "cache_bytes": sum(c.n_slots * c.slot_bytes for c in self.caches.values())}


def poisson_requests(rate: float, n: int, pyramids, seed: int, view=(1920, 1080), zmax=7, first_id=0):
    """n requests with exponential inter-arrival times (Poisson process of `rate` per second): each picks a
    pyramid, a level z uniform in 0..zmax and a viewport position uniform over the valid ones (the whole level
    when it is smaller than the viewport)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    vw, vh = view
    for k in range(n):
        pi = int(rng.integers(0, len(pyramids)))
        p = pyramids[pi]
        z = int(rng.integers(0, min(zmax, p.levels) + 1))
        lw, lh = p.level_size(z)
        rw, rh = min(vw, lw), min(vh, lh)
        rx = int(rng.integers(0, lw - rw + 1))
        ry = int(rng.integers(0, lh - rh + 1))
        out.append(Request(first_id + k, float(t[k]), pi, z, (rx, ry, rw, rh)))
    return out


def latency_stats(done):
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    if not len(lat):
        return {"p50_ms": None, "p99_ms": None}
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}
