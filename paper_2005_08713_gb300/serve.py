"""Viewport serving over a device-resident compressed pyramid.

A pyramid is one image encoded as tiles (the stream, its tile offsets and
the tile descriptors stay in device memory); a request asks for a viewport
(a rectangle of pixels at one resolution level z, Sec. 4: a decode at level
z reads only the LL band and the levels above z).  The server runs
continuous batching: requests that arrive while others are on the GPU are
queued, and whenever one of its slots (a CUDA stream with its own library
context) is free it takes the queued requests, as many as the slot's
scratch budget admits, and decodes them with one isx_decode_jobs call per
(pyramid, level) group.  Several slots run at once, so batches overlap on
the device.  Each request's latency runs from its arrival to the moment the
host sees its batch's completion event.

The coarse levels of each pyramid (z >= resident_from) can be kept decoded
in device memory (decoded once, whole, when the server starts: together
they are about 1/48 of the full-resolution image); requests at those levels
are then device copies of a crop, while requests at the finer levels are
decoded per batch.

All decoding happens in the library's kernels; this module only plans
batches (which tiles meet which viewport) and keeps time.
"""
from __future__ import annotations

import collections
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

    def tiles_meeting(self, z: int, rx: int, ry: int, rw: int, rh: int) -> np.ndarray:
        """Indices of the tiles whose level-z footprint meets the rectangle (row-major grid)."""
        s = self.tile >> z if (self.tile >> z) << z == self.tile else None
        if s:
            # tile (i, j) covers [j * s, (j + 1) * s) at level z when the tile edge is a multiple of 2^z
            c0, c1 = max(0, rx // s), min(self.grid_w - 1, (rx + rw - 1) // s)
            r0, r1 = max(0, ry // s), min(self.grid_h - 1, (ry + rh - 1) // s)
        else:
            c0, c1, r0, r1 = 0, self.grid_w - 1, 0, self.grid_h - 1   # the library skips tiles outside the rectangle
        cols = np.arange(c0, c1 + 1, dtype=np.int32)
        rows = np.arange(r0, r1 + 1, dtype=np.int32)
        return (rows[:, None] * self.grid_w + cols[None, :]).reshape(-1)


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
    jobs: object = None
    result: object = None     # host copy of the output (Server(keep_outputs=True))
    error: object = None      # status name when the decode of this request reported a data error


@dataclass
class _Slot:
    codec: isx.Codec
    stream: object
    busy: bool = False
    batch: list = field(default_factory=list)
    event: object = None


class Server:
    """Continuous-batching viewport server.

    slots:            concurrent batches (each a CUDA stream and a library context)
    max_batch:        most requests in one batch
    scratch_budget:   device scratch per slot (bytes); a batch takes queued
                      requests while its decode scratch stays within it, and
                      the slots' scratch is reserved up front, so serving
                      allocates no device memory
    """

    def __init__(self, pyramids, device=0, slots=4, max_batch=32, scratch_budget=1 << 30, out_shape=None, keep_outputs=False,
                 resident_from=None):
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
        # Decoded levels kept resident: every level z >= resident_from of every
        # pyramid is decoded once, whole, here; requests at those levels are
        # crops of it (a device copy), the others are decoded per batch.
        self.resident = {}
        if resident_from is not None:
            with isx.Codec(device) as c:
                for pi, p in enumerate(self.pyr):
                    for z in range(resident_from, p.levels + 1):
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

    def close(self):
        for s in self.slots:
            s.codec.close()
        self.slots = []

    # ------------------------------------------------------------ planning
    def _jobs(self, req: Request, out) -> np.ndarray:
        p = self.pyr[req.pyramid]
        rx, ry, rw, rh = req.rect
        idx = p.tiles_meeting(req.z, rx, ry, rw, rh)
        jobs = np.zeros(len(idx), isx.JOB_DTYPE)
        jobs["tile"] = idx
        jobs["rx"], jobs["ry"], jobs["rw"], jobs["rh"] = rx, ry, rw, rh
        jobs["d_out"] = out.data_ptr()
        jobs["out_pitch_bytes"] = out.stride(0) * out.element_size()
        return jobs

    def _launch(self, slot: _Slot, batch):
        groups = collections.defaultdict(list)
        for r in batch:
            lvl = self.resident.get((r.pyramid, r.z))
            if lvl is not None:
                rx, ry, rw, rh = r.rect
                with self.torch.cuda.stream(slot.stream):
                    r.out.copy_(lvl[ry:ry + rh, rx:rx + rw], non_blocking=True)
                continue
            groups[(r.pyramid, r.z)].append(r)
        for (pi, z), rs in groups.items():
            p = self.pyr[pi]
            jobs = np.concatenate([r.jobs for r in rs])
            slot.codec.decode_jobs_array(p.stream, p.offsets, p.tiles, jobs, z, 0, slot.stream)
        ev = self.torch.cuda.Event()
        ev.record(slot.stream)
        slot.batch, slot.event, slot.busy = batch, ev, True

    def _admit(self, queue, slot: _Slot):
        """Takes queued requests in arrival order while the batch's decode scratch fits the slot's budget."""
        # one decode call per (pyramid, level) group, one after another on the slot's
        # stream: each group's scratch (bounded by the sum of its requests') must fit
        batch, need_by_group = [], collections.defaultdict(int)
        while queue and len(batch) < self.max_batch and self.pool:
            r = queue[0]
            buf = self.pool[0]
            p = self.pyr[r.pyramid]
            rx, ry, rw, rh = r.rect
            view = buf[:rh, :rw, :p.channels]
            if (r.pyramid, r.z) in self.resident:
                r.jobs, need = None, 0
            else:
                r.jobs = self._jobs(r, view)
                need = slot.codec.decode_jobs_scratch(p.tiles, r.jobs, r.z) if len(r.jobs) else 0
            key = (r.pyramid, r.z)
            if need_by_group[key] + need > self.budget:
                if not batch:
                    raise RuntimeError(f"request {r.rid} needs {need} bytes of scratch, more than the slot budget {self.budget}")
                break
            need_by_group[key] += need
            queue.popleft()
            self.pool.popleft()
            r.out, r.buf = view, buf
            batch.append(r)
        return batch

    def _isolate_failures(self, slot: _Slot, batch):
        """A batch whose decode reported a data error (a corrupt stream, a capacity or consistency
        status): each of its decoded requests is decoded again alone on the slot, so that only the
        requests whose own decode fails get `error` set; the others keep a correct result."""
        for r in batch:
            if r.jobs is None or not len(r.jobs):
                continue
            p = self.pyr[r.pyramid]
            slot.codec.decode_jobs_array(p.stream, p.offsets, p.tiles, r.jobs, r.z, 0, slot.stream)
            st = slot.codec.sync_status(slot.stream)
            if st != 0:
                r.error = isx.STATUS_NAMES.get(st, st)

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
                    if s.codec.sync_status(s.stream) != 0:
                        self._isolate_failures(s, s.batch)
                    t = time.perf_counter() - t0
                    for r in s.batch:
                        r.done = t
                        if self.keep_outputs:
                            r.result = r.out.cpu().numpy()
                        done.append(r)
                        self.pool.append(r.buf)
                    s.busy, s.batch, s.event = False, [], None
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
