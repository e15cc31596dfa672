#!/usr/bin/env python3
"""Benchmark: encode + decode of a whole-slide-shaped image on one GB300.

Workload (synthetic stand-in for the paper's 100-megapixel 27-bit pathology
scans, which are not available): a 40000 x 30000 RGB8 slide from the seeded
generator, cut into 256 x 256 tiles (edge tiles 64 wide / 48 tall), 8 wavelet
levels, lossy with quantiser steps 8/4/2 on levels 1-3 (1 elsewhere); the
same image is also measured lossless.  One step = encode every tile into one
contiguous stream + decode the full image back (all stages of the codec).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode & decode megapixels/s on 1 GB300 (bit-exact vs oracle), % of HBM roofline; p99 tile latency"
IMG_W, IMG_H, TILE, LEVELS = 40000, 30000, 256, 8   # --size overrides IMG_W x IMG_H (profiling runs)
LOSSY_Q = [3, 2, 1, 0, 0, 0, 0, 0, 0]


def tile_grid(w=None, h=None, t=TILE):
    w = IMG_W if w is None else w
    h = IMG_H if h is None else h
    return [(x, y, min(t, w - x), min(t, h - y)) for y in range(0, h, t) for x in range(0, w, t)]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms from start()
    (before the warm-up, so that sampling runs by the time the timed region
    starts) to stop(); the summary keeps the samples whose nvidia-smi
    timestamp falls between mark_start() and mark_end()."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index: int, exe: str = "nvidia-smi"):
        self.dev = device_index
        self.exe = exe
        self.proc = None
        self.lines = []
        self.thread = None
        self.t_start = self.t_end = None

    def start(self):
        try:
            self.proc = subprocess.Popen([self.exe, "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def mark_start(self):
        self.t_start = time.time()

    def mark_end(self):
        self.t_end = time.time()

    @staticmethod
    def _stamp(text):
        """nvidia-smi's timestamp ("2026/12/04 03:02:11.123", local time) as epoch seconds, else None."""
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text.strip(), fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self, lines):
        rows = []
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            active = {nm for k, nm in enumerate(self.REASONS) if parts[6 + k].lower().startswith("active")}
            rows.append((self._stamp(parts[0]), sm, smax, active))
        if self.t_start is not None and self.t_end is not None:
            inside = [r for r in rows if r[0] is not None and self.t_start <= r[0] <= self.t_end]
        else:
            inside = []
        # a timed region shorter than the sampling period can fall between two samples: then take the
        # first sample after it started (the clock the region ran at, as near as nvidia-smi saw it)
        if not inside and self.t_start is not None:
            after = [r for r in rows if r[0] is not None and r[0] >= self.t_start]
            inside = after[:1]
        if not inside:
            inside = rows
        reasons = set()
        for r in inside:
            reasons |= r[3]
        return {"sm_mhz": statistics.median([r[1] for r in inside]) if inside else None,
                "sm_max_mhz": inside[-1][2] if inside else None, "reasons": sorted(reasons),
                "samples": len(inside), "samples_total": len(rows)}

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary(list(self.lines))


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per pixel of each stage's kernel, from the
# committed ncu captures of the 8192 x 8192 case of this workload (one kernel per capture), scaled to a full
# launch by pixels.  These are figures copied from those captures, not measured by this run.  Valid only while the code of the kernel's source files is the one
# captured (source_digest: comments and whitespace aside); otherwise the bench reports traffic as null.
NCU_TRAFFIC = {
    "encode.transform": ("k_fwd_tile_smem", ('isx_transform.cu', 'isx_fused.cuh', 'isx_warp_levels.cuh', 'isx_internal.cuh'), "61c333bc78afa0da", 8.170),
    "encode.symbols": ("k_enc_symbols", ('isx_encode.cu', 'isx_coder_enc.cuh', 'isx_internal.cuh'), "832d6c6f04cd9b3b", 7.440),
    "encode.huffman": ("k_block_huffman", ('isx_encode.cu', 'isx_coder_enc.cuh', 'isx_internal.cuh'), "832d6c6f04cd9b3b", 0.520),
    "encode.layout": ("k_enc_layout", ('isx_encode.cu', 'isx_coder_enc.cuh', 'isx_internal.cuh'), "832d6c6f04cd9b3b", 0.910),
    "encode.emit": ("k_enc_emit", ('isx_encode.cu', 'isx_coder_enc.cuh', 'isx_internal.cuh'), "832d6c6f04cd9b3b", 3.840),
    "decode.tables": ("k_dec_tables", ('isx_decode.cu', 'isx_coder_dec.cuh', 'isx_internal.cuh'), "626129d9031bf72a", 0.420),
    "decode.segments": ("k_dec_segments", ('isx_decode.cu', 'isx_coder_dec.cuh', 'isx_internal.cuh'), "626129d9031bf72a", 2.670),
    "decode.inverse_transform": ("k_inv_tile_smem", ('isx_transform.cu', 'isx_fused.cuh', 'isx_warp_levels.cuh', 'isx_internal.cuh'), "61c333bc78afa0da", 4.090),
}


# Warp instructions per pixel of each stage's kernel (smsp__inst_executed.sum of the same captures),
# for the issue-rate co-roofline: the codec is integer work, and its kernels are bound by latency and
# instruction issue long before DRAM bandwidth.
NCU_WARP_INST_PER_PX = {
    "encode.transform": 6.150, "encode.symbols": 5.020, "encode.huffman": 3.450, "encode.layout": 0.630, "encode.emit": 6.260,
    "decode.tables": 1.340, "decode.segments": 7.830, "decode.inverse_transform": 7.260,
}


def issue_roofline(stage, px, ms):
    """Achieved warp instructions per second (ncu count per pixel x pixels / event time) against the issue
    peak: SMs x 4 schedulers x 1 warp instruction per cycle x the SM clock seen during the run."""
    import torch
    per_px = NCU_WARP_INST_PER_PX.get(stage)
    if per_px is None or traffic_bytes(stage, px) is None:   # same validity rule as the traffic figures
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return per_px, sms


def stage_issue_frac(stage, px, ms, clk):
    """A stage kernel's warp-instruction rate over the SM issue peak (None without a valid capture or clock)."""
    iss = issue_roofline(stage, px, ms)
    if not iss or not clk.get("sm_mhz") or ms <= 0:
        return None
    per_px, sms = iss
    return round(per_px * px / (ms / 1e3) / (sms * 4 * clk["sm_mhz"] * 1e6), 4)


def source_digest(names):
    """First 16 hex digits of the sha256 of the code of the named csrc files, comments and whitespace removed
    (an edit of a comment does not change the kernels the counters were taken on)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2005_08713_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_bytes(stage, px):
    ent = NCU_TRAFFIC.get(stage)
    if not ent:
        return None
    names = ent[1] if isinstance(ent[1], tuple) else (ent[1],)
    try:
        digest = source_digest(names)
    except OSError:
        return None
    return int(ent[3] * px) if digest == ent[2] else None


def block_geometry(w, h, levels, channels):
    """(p, padded width, padded height) of every block of a tile, in stream order (Fig. 3)."""
    def ld(n, l):
        for _ in range(l):
            n = (n + 1) >> 1
        return n
    out = []
    for _c in range(channels):
        for lv in range(levels + 1):
            level = 0 if lv == 0 else levels + 1 - lv
            gw, gh = ld(w, levels if level == 0 else level), ld(h, levels if level == 0 else level)
            p = 1 if level == 0 else 3
            for by in range(-(-gh // 128)):
                for bx in range(-(-gw // 128)):
                    out.append((p, (min(128, gw - 128 * bx) + 3) // 4 * 4, (min(128, gh - 128 * by) + 3) // 4 * 4))
    return out


def kept_symbol_bytes(raw, offs, grid, levels, channels):
    """Number of blocks and total symbol bytes of their kept (plane, type) pairs, read from the block
    headers of an encoded stream: each block opens with d (5 bits) and p*d removed-plane flags."""
    starts, geo = [], []
    cache = {}
    for i, (x, y, w, h) in enumerate(grid):
        t0 = int(offs[i])
        nb = int(np.frombuffer(raw[t0 + 12:t0 + 16].tobytes(), "<u4")[0])
        ends = np.frombuffer(raw[t0 + 32:t0 + 32 + 4 * nb].tobytes(), "<u4").astype(np.int64)
        data = t0 + 32 + 4 * nb
        starts.append(data + np.concatenate(([0], ends[:-1])))
        key = (w, h)
        if key not in cache:
            cache[key] = np.array(block_geometry(w, h, levels, channels), np.int64)
        geo.append(cache[key])
    starts = np.concatenate(starts)
    geo = np.concatenate(geo)
    padded = np.concatenate([raw, np.zeros(16, np.uint8)])
    bits = np.unpackbits(padded[starts[:, None] + np.arange(16)[None, :]], axis=1).astype(np.int32)
    d = bits[:, :5] @ np.array([16, 8, 4, 2, 1])
    p, bw, bh = geo[:, 0], geo[:, 1], geo[:, 2]
    cs = np.cumsum(bits, axis=1)
    removed = cs[np.arange(len(d)), 4 + p * d] - cs[:, 4]
    kept = p * d - removed
    return len(d), int((kept * (bw * bh // 8)).sum())


def stamp_latency(st, n):
    """p50 / p99 / max of the per-tile encode and decode latencies (ms) from isx_set_tile_stamps arrays:
    end - start of each tile that both stamps saw."""
    out = {}
    for name, k in (("encode", 0), ("decode", 2)):
        s0, s1 = st[k * n:(k + 1) * n], st[(k + 1) * n:(k + 2) * n]
        ok = (s0 != np.iinfo(np.uint64).max) & (s1 != 0) & (s1 >= s0)
        d = np.sort((s1[ok] - s0[ok]).astype(np.float64) / 1e6)
        if not len(d):
            out[name] = None
            continue
        out[name] = {"p50": round(float(d[len(d) // 2]), 3), "p99": round(float(d[int(0.99 * (len(d) - 1))]), 3),
                     "max": round(float(d[-1]), 3), "tiles": int(len(d))}
    out["what"] = ("per tile, %globaltimer from its first kernel to its last step (tile header written / pixels stored), "
                   "every tile of one call")
    return out


def make_slide(seed):
    import torch
    from paper_2005_08713_gb300 import synth
    h_img = torch.empty((IMG_H, IMG_W, 3), dtype=torch.uint8, pin_memory=True)
    synth.slide(seed, 0, 0, IMG_W, IMG_H, out=h_img.numpy())
    return h_img


def soft(fn, *a, **kw):
    """Runs one of the optional measurements (CPU baseline, serving, mixed batch): a failure there is
    recorded in the JSON line as {"error": ...} instead of losing the line and its headline number."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - any failure of an optional part is reported, not raised
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def replica_seed(rank):
    """Each replica encodes its own slide: the workload's seed offset by the rank."""
    from paper_2005_08713_gb300 import synth
    return synth.config_seed(3) + rank


def max_over_ranks(ms, world, device):
    """The slowest replica's timed region (ms): a MAX reduction over the ranks."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(ms_total, steps, world, mp_per_replica):
    """(ms per step, whole-job MP/s): every replica's pixels over the slowest
    replica's time (weak scaling, one slide per GPU)."""
    ms_step = ms_total / steps
    return ms_step, world * mp_per_replica / (ms_step / 1e3)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2005_08713_gb300 import isx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    h_img = make_slide(replica_seed(rank))
    mp = IMG_W * IMG_H / 1e6
    d_img = h_img.to(dev, non_blocking=False)
    grid = tile_grid()
    codec = isx.Codec(local)
    q = LOSSY_Q if not args.lossless else [0] * 9

    def tiles_for(buf, qs):
        return isx.TileArray([isx.tile_from_tensor(buf[y:y + h, x:x + w], LEVELS, 8, qs, x, y) for (x, y, w, h) in grid])

    tiles = tiles_for(d_img, q)
    cap = IMG_W * IMG_H * 3 + (1 << 24)
    d_out = torch.empty(cap, dtype=torch.uint8, device=dev)
    d_offs = torch.empty(len(tiles) + 1, dtype=torch.int64, device=dev)
    d_dec = torch.empty_like(d_img)
    stream = torch.cuda.current_stream()

    def step():
        codec.encode_tiles(tiles, d_out, d_offs, stream)
        n_enc = codec.last_launch_count
        codec.decode_region(d_out, d_offs, tiles, 0, (0, 0, IMG_W, IMG_H), d_dec, 0, stream)
        return n_enc + codec.last_launch_count

    # correctness gate before timing: the full image round-trips and sampled tiles match the oracle
    step()
    st = codec.sync_status(stream)
    if st != 0:
        raise RuntimeError(f"device status {st}")
    total_bytes = int(d_offs[-1].item())

    # clocks are sampled from here on, so that nvidia-smi is running by the time the timed region starts
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # separate encode/decode timing (device events), then the full step timing
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    enc_ms, dec_ms = [], []
    for _ in range(2):
        ev[0].record(stream)
        codec.encode_tiles(tiles, d_out, d_offs, stream)
        ev[1].record(stream)
        codec.decode_region(d_out, d_offs, tiles, 0, (0, 0, IMG_W, IMG_H), d_dec, 0, stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        enc_ms.append(ev[0].elapsed_time(ev[1]))
        dec_ms.append(ev[1].elapsed_time(ev[2]))

    codec.set_timing(True)
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    clocks.mark_start()
    t0.record(stream)
    for _ in range(args.steps):
        launches += step()
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    stages = codec.stage_times()
    codec.set_timing(False)
    ms = max_over_ranks(ms, world, dev)
    ms_step, value = replica_throughput(ms, args.steps, world, mp)

    # exactness on the bench's own launch: decoded tiles equal the oracle's, sampled
    exact = None
    if rank == 0 and not args.no_check:
        import oracle
        rng = np.random.default_rng(7)
        o = d_offs.cpu().numpy()
        idx = rng.choice(len(grid), min(12, len(grid)), replace=False).tolist() + [len(grid) - 1]
        ok = True
        img_np = h_img.numpy()
        for i in idx:
            x, y, w, h = grid[i]
            ref = oracle.encode_tile(np.ascontiguousarray(img_np[y:y + h, x:x + w]), LEVELS, 8, q)
            got = d_out[int(o[i]):int(o[i + 1])].cpu().numpy().tobytes()
            dec_ok = np.array_equal(d_dec[y:y + h, x:x + w].cpu().numpy(), oracle.decode_tile(ref, 0))
            ok = ok and got == ref and dec_ok
        exact = {"sampled_tiles": len(idx), "bit_exact": bool(ok)}

    # roofline of the dominant single-kernel stage
    hbm, peak_kind = peaks()
    n_tiles = len(grid)
    coef_elems = 0
    for (x, y, w, h) in grid:
        lw, lh = w, h
        cnt = 0
        for _ in range(LEVELS):
            lw, lh = (lw + 1) // 2, (lh + 1) // 2
            cnt += 3 * ((lw + 3) // 4 * 4) * ((lh + 3) // 4 * 4)
        cnt += ((lw + 3) // 4 * 4) * ((lh + 3) // 4 * 4)
        coef_elems += 3 * cnt
    raw = d_out[:total_bytes].cpu().numpy()
    n_blocks, sym_bytes = kept_symbol_bytes(raw, d_offs.cpu().numpy(), grid, LEVELS, 3)
    px = IMG_W * IMG_H
    # bytes each kernel must read and write in this design, per call (units: one call over the whole image);
    # sym_bytes = symbols of every kept (plane, type) of every block, one byte each
    algo = {
        "encode.transform": 3 * px + 2 * coef_elems,                    # RGB8 in, int16 area-ordered blocks out
        # statistics per block: 1.1 KB of block totals, plus per kept plane 560 B (a plane of more than
        # 512 symbols: its histogram) or 48 B (a shorter one, whose symbols the layout pass reads instead);
        # about 2 KB per block on this workload
        "encode.symbols": 2 * coef_elems + sym_bytes + 3100 * n_blocks,  # blocks in, kept symbols + statistics out
        "encode.huffman": (1200 + 1700) * n_blocks,                      # block statistics in, code tables out
        "encode.layout": 2300 * n_blocks,                                # plane statistics + code lengths in, layout out
        "encode.emit": sym_bytes + 1700 * n_blocks + total_bytes,        # symbols + codes in, stream out
        "decode.tables": 600 * n_blocks,                                 # block headers in (<= 600 B), tables out
        "decode.segments": total_bytes + sym_bytes,                      # stream in, kept symbols out
        "decode.inverse_transform": sym_bytes + 3 * px,                  # symbols in, RGB8 pixels out (fused store)
    }
    single = {k: v for k, v in stages.items() if k in algo}
    dom = max(single, key=lambda k: single[k][0]) if single else None
    roof = None
    # algorithmic bytes of the path (one encode or one decode of the image): 3 B/px of pixels plus the
    # compressed stream; coefficients and symbols moved between kernels are not algorithmic
    path_bytes = 3 * px + total_bytes
    if dom:
        avg_ms = single[dom][0] / max(1, single[dom][1])
        ach = path_bytes / (avg_ms / 1e3) / 1e9
        iss = issue_roofline(dom, px, avg_ms)
        alu = None
        if iss and clk.get("sm_mhz"):
            per_px, sms = iss
            peak_wi = sms * 4 * clk["sm_mhz"] * 1e6
            got = per_px * px / (avg_ms / 1e3)
            alu = {"bound": "issue", "achieved": round(got / 1e9, 1), "peak": round(peak_wi / 1e9, 1), "unit": "G warp-inst/s",
                   "frac": round(got / peak_wi, 4), "warp_inst_per_px": per_px,
                   "peak_basis": f"{sms} SMs x 4 schedulers x 1 warp-inst/cycle x {clk['sm_mhz']:.0f} MHz (median under load)"}
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                "algorithmic_bytes": int(path_bytes),
                "algorithmic_basis": "3 B/px of pixels + the compressed stream, per launch (the kernel covers the whole image)",
                "issue_coroofline": alu,
                "traffic": traffic_bytes(dom, px), "peak_kind": peak_kind,
                "traffic_source": "committed ncu capture of the 8192x8192 case, scaled by pixels; null once the kernel's code "
                                  "differs from the captured code",
                "avg_launch_ms": round(avg_ms, 3),
                "kernel_io_bytes": int(algo[dom]),
                "stage_rooflines": {
                    k: {"ms": round(v[0] / max(1, v[1]), 3),
                        "path_frac": round(path_bytes / (v[0] / max(1, v[1]) / 1e3) / 1e9 / hbm, 4),
                        "kernel_io_GBps": round(algo[k] / (v[0] / max(1, v[1]) / 1e3) / 1e9, 1),
                        "kernel_io_frac": round(algo[k] / (v[0] / max(1, v[1]) / 1e3) / 1e9 / hbm, 4),
                        "issue_frac": stage_issue_frac(k, px, v[0] / max(1, v[1]), clk)} for k, v in single.items()},
                "stage_rooflines_basis": "path_frac: the path's algorithmic bytes over the stage's time; kernel_io: the bytes this "
                                         "design's kernel must read and write (intermediates included); issue_frac: the "
                                         "kernel's warp instructions (ncu count per pixel x pixels) per second over SMs x 4 "
                                         "x the SM clock, null where the captured code differs"}
        if alu:
            alu["source"] = "warp instructions per pixel from the committed ncu capture (not measured by this run)"
    path = {"encode_GBps": round(path_bytes / (statistics.median(enc_ms) / 1e3) / 1e9, 1),
            "decode_GBps": round(path_bytes / (statistics.median(dec_ms) / 1e3) / 1e9, 1),
            "algorithmic_bytes_per_px": round(path_bytes / (IMG_W * IMG_H), 3), "peak_GBps": hbm}
    path["encode_frac"] = round(path["encode_GBps"] / hbm, 4)
    path["decode_frac"] = round(path["decode_GBps"] / hbm, 4)

    # per-tile latency inside the full-image encode and decode: %globaltimer stamps of every tile's first
    # kernel and of its last step (its tile header, its stored pixels), one stamped step after the timed region
    stamps = torch.zeros(4 * len(grid), dtype=torch.int64, device=dev)
    codec.set_tile_stamps(stamps)
    step()
    torch.cuda.synchronize()
    codec.set_tile_stamps(None)
    tile_lat = stamp_latency(stamps.cpu().numpy().view(np.uint64), len(grid))

    # per-tile decode latency (single-tile region requests): device events, and the host time of the call
    lat = [float("nan")]
    host_ms = []
    rng = np.random.default_rng(3)
    tile_out = torch.empty((TILE, TILE, 3), dtype=torch.uint8, device=dev)
    for i in ([] if args.no_latency else rng.choice(n_tiles, min(64, n_tiles), replace=False).tolist()):
        x, y, w, h = grid[i]
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h0 = time.perf_counter()
        codec.decode_region(d_out, d_offs, tiles, 0, (x, y, w, h), tile_out, 0, stream)
        host_ms.append((time.perf_counter() - h0) * 1e3)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    lat = sorted(v for v in lat if v == v) or [float("nan")]
    host_ms = sorted(host_ms) or [float("nan")]

    # end to end through the host-buffer entry points (pinned host memory)
    h_np = h_img.numpy()
    h_tiles = isx.TileArray([isx.tile_from_array(h_np[y:y + h, x:x + w], LEVELS, 8, q, x, y) for (x, y, w, h) in grid])
    e2e = None
    if not args.no_e2e:
        import torch as _t
        h_out = _t.empty(cap, dtype=_t.uint8, pin_memory=True).numpy()
        h_offs = np.zeros(len(grid) + 1, np.uint64)
        h_dec = _t.empty((IMG_H, IMG_W, 3), dtype=_t.uint8, pin_memory=True).numpy()
        codec.encode_tiles_host(h_tiles, h_out, h_offs)
        e2e_steps = max(1, min(args.steps, 3))
        t_start = time.perf_counter()
        for _ in range(e2e_steps):
            codec.encode_tiles_host(h_tiles, h_out, h_offs)
            codec.decode_region_host(h_out, h_offs, h_tiles, 0, (0, 0, IMG_W, IMG_H), h_dec)
        e2e_s = (time.perf_counter() - t_start) / e2e_steps
        nbytes = int(h_offs[-1])
        e2e = {"value": round(world * mp / e2e_s, 1), "unit": "MP/s",
               "h2d_bytes_per_step": 3 * IMG_W * IMG_H + nbytes + 8 * (len(grid) + 1),
               "d2h_bytes_per_step": nbytes + 8 * (len(grid) + 1) + 3 * IMG_W * IMG_H}

    # the same slide lossless (BASELINE config 3's second run): encode + full decode, device events
    ll = {"tiles": None}

    def lossless_run():
        tiles_ll = tiles_for(d_img, [0] * 9)
        d_out2 = torch.empty(cap, dtype=torch.uint8, device=dev)
        d_offs2 = torch.empty(len(grid) + 1, dtype=torch.int64, device=dev)
        codec.encode_tiles(tiles_ll, d_out2, d_offs2, stream)
        if codec.sync_status(stream) != 0:
            raise RuntimeError("lossless encode failed")
        ll.update(tiles=tiles_ll, out=d_out2, offs=d_offs2)
        e_ms, d_ms = [], []
        for _ in range(max(3, min(args.steps, 6))):
            ev[0].record(stream)
            codec.encode_tiles(tiles_ll, d_out2, d_offs2, stream)
            ev[1].record(stream)
            codec.decode_region(d_out2, d_offs2, tiles_ll, 0, (0, 0, IMG_W, IMG_H), d_dec, 0, stream)
            ev[2].record(stream)
            torch.cuda.synchronize()
            e_ms.append(ev[0].elapsed_time(ev[1]))
            d_ms.append(ev[1].elapsed_time(ev[2]))
        if codec.sync_status(stream) != 0:
            raise RuntimeError("lossless round trip failed")
        nb = int(d_offs2[-1].item())
        pb = 3 * px + nb
        em, dm = statistics.median(e_ms), statistics.median(d_ms)
        return {"workload": f"slide_{IMG_W}x{IMG_H}_rgb8_tile{TILE}_L{LEVELS}_lossless",
                "encode_mps": round(mp / (em / 1e3), 1), "decode_mps": round(mp / (dm / 1e3), 1),
                "encode_ms": round(em, 3), "decode_ms": round(dm, 3),
                "compressed_bytes": nb, "bits_per_pixel": round(8 * nb / px, 3),
                "algorithmic_bytes_per_px": round(pb / px, 3),
                "encode_frac": round(pb / (em / 1e3) / 1e9 / hbm, 4), "decode_frac": round(pb / (dm / 1e3) / 1e9 / hbm, 4),
                "lossless_identity": bool(torch.equal(d_dec, d_img))}

    lossless = soft(lossless_run) if rank == 0 and not args.lossless and not args.no_lossless else None

    singles = soft(run_single_configs, dev, stream, max(5, args.steps)) if rank == 0 and not args.no_single else None

    untiled = soft(run_untiled, d_img, dev, stream) if rank == 0 and not args.no_untiled else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = soft(cpu_baseline, h_img.numpy(), grid, q, args.cpu_tiles)

    res = {"metric": METRIC, "value": round(value, 1), "unit": "MP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic",
           "config": {"workload": f"slide_{IMG_W}x{IMG_H}_rgb8_tile{TILE}_L{LEVELS}_" + ("lossless" if args.lossless else "lossy_q8421"),
                      "tiles": n_tiles, "megapixels_per_gpu": round(mp, 1), "l2": "inputs larger than L2 (3.6 GB per step)",
                      "parallelism": f"replicas x{world}"},
           "encode_mps": round(mp / (statistics.median(enc_ms) / 1e3), 1),
           "decode_mps": round(mp / (statistics.median(dec_ms) / 1e3), 1),
           "compressed_bytes": total_bytes, "bits_per_pixel": round(8 * total_bytes / (IMG_W * IMG_H), 3),
           "exact": exact, "roofline": roof, "path_roofline": path,
           "tile_decode_latency_ms": {"p50": round(lat[len(lat) // 2], 3), "p99": round(lat[int(0.99 * (len(lat) - 1))], 3),
                                      "host_call_p50": round(host_ms[len(host_ms) // 2], 3),
                                      "what": "one 256x256 tile decoded alone by isx_decode_region (device events around "
                                              "the call, host planning included)"},
           "tile_latency_in_step_ms": tile_lat,
           "stages_ms": {k: round(v[0] / max(1, v[1]), 3) for k, v in stages.items()},
           "e2e": e2e, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu,
           "lossless": lossless, "single_image_configs": singles, "untiled": untiled}
    def serving():
        # the slide's lossy pyramid is the stream above; encode the lossless one beside it
        from paper_2005_08713_gb300 import serve
        if ll["tiles"] is None:
            lossless_run()
        tiles_ll, d_out2, d_offs2 = ll["tiles"], ll["out"], ll["offs"]
        pyramids = [serve.Pyramid(IMG_W, IMG_H, TILE, LEVELS, 3, 8, d_out, d_offs, tiles),
                    serve.Pyramid(IMG_W, IMG_H, TILE, LEVELS, 3, 8, d_out2, d_offs2, tiles_ll)]
        return run_serve(args, dev, pyramids)

    if rank == 0 and not args.no_serve:
        res["serve"] = soft(serving)
    codec.close()
    if rank == 0 and not args.no_batch:
        res["batch"] = soft(run_batch, args, dev, args.batch_tiles)
    if world > 1:
        dist.destroy_process_group()
    return res if rank == 0 else None


def run_untiled(d_img, dev, stream, viewports=48):
    """The slide coded as ONE image (whole-image transform, the int32 global path), lossy: encode and full
    decode time, then 1920 x 1080 viewports at levels 0-3 decoded windowed (only the blocks and samples each
    depends on), device latency per viewport; each viewport checked against the same window of the full
    decode."""
    import torch
    from paper_2005_08713_gb300 import isx
    H, W = int(d_img.shape[0]), int(d_img.shape[1])
    mp = W * H / 1e6
    with isx.Codec(dev.index or 0) as codec:
        tiles = isx.TileArray([isx.tile_from_tensor(d_img, LEVELS, 8, LOSSY_Q)])
        cap = W * H * 3 + (1 << 24)
        d_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        d_offs = torch.empty(2, dtype=torch.int64, device=dev)
        d_dec = torch.empty_like(d_img)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e_ms, d_ms = [], []
        for k in range(3):
            ev[0].record(stream)
            codec.encode_tiles(tiles, d_out, d_offs, stream)
            ev[1].record(stream)
            codec.decode_region(d_out, d_offs, tiles, 0, (0, 0, W, H), d_dec, 0, stream)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if codec.sync_status(stream) != 0:
                raise RuntimeError("untiled round trip failed")
            if k:
                e_ms.append(ev[0].elapsed_time(ev[1]))
                d_ms.append(ev[1].elapsed_time(ev[2]))
        nbytes = int(d_offs[1].item())
        rng = np.random.default_rng(21)
        lat, ok = [], True
        vw, vh = 1920, 1080
        fulls = {}
        for k in range(viewports):
            z = k % 4
            zw, zh = isx.level_dim(W, z), isx.level_dim(H, z)
            rw, rh = min(vw, zw), min(vh, zh)
            rx, ry = int(rng.integers(0, zw - rw + 1)), int(rng.integers(0, zh - rh + 1))
            res = torch.empty((rh, rw, 3), dtype=torch.uint8, device=dev)
            ev[0].record(stream)
            codec.decode_region(d_out, d_offs, tiles, z, (rx, ry, rw, rh), res, 0, stream)
            ev[1].record(stream)
            ev[1].synchronize()
            lat.append(ev[0].elapsed_time(ev[1]))
            if k < 8:   # against the same window of a full decode at that level
                if z not in fulls:
                    f = torch.empty((zh, zw, 3), dtype=torch.uint8, device=dev)
                    codec.decode_region(d_out, d_offs, tiles, z, (0, 0, zw, zh), f, 0, stream)
                    fulls[z] = f
                ok = ok and bool(torch.equal(res, fulls[z][ry:ry + rh, rx:rx + rw]))
        if codec.sync_status(stream) != 0:
            raise RuntimeError("untiled viewport decode failed")
        lat = sorted(lat)
        em, dm = statistics.median(e_ms), statistics.median(d_ms)
        return {"workload": f"untiled_{W}x{H}_rgb8_L{LEVELS}_lossy_q8421 (one image, whole-image transform)",
                "encode_mps": round(mp / (em / 1e3), 1), "decode_mps": round(mp / (dm / 1e3), 1),
                "encode_ms": round(em, 3), "decode_ms": round(dm, 3), "compressed_bytes": nbytes,
                "viewport_1920x1080_z0to3_ms": {"p50": round(lat[len(lat) // 2], 3),
                                                 "p99": round(lat[int(0.99 * (len(lat) - 1))], 3), "n": len(lat)},
                "viewports_equal_full_decode": ok}


def run_single_configs(dev, stream, reps):
    """The two single-image workloads on the GPU: the 512 x 512 RGB8 stain tile (3 levels) and the
    2048 x 2048 12-bit phantom (5 levels), lossless; encode and decode MP/s (device events, median of
    `reps`), streams checked byte for byte and decodes pixel for pixel against the oracle."""
    import torch
    import oracle
    from paper_2005_08713_gb300 import isx, synth
    cases = {"stain_512x512_rgb8_L3_lossless": (synth.stain(synth.config_seed(1)), 3, 8),
             "phantom_2048x2048_u12_L5_lossless": (synth.phantom(synth.config_seed(2), 2048, 2048), 5, 12)}
    out = {}
    with isx.Codec(dev.index or 0) as codec:
        for name, (img, L, bits) in cases.items():
            a = np.ascontiguousarray(img)
            d = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).to(dev)
            tiles = isx.TileArray([isx.tile_from_tensor(d, L, bits)])
            cap = a.nbytes * 2 + (1 << 16)
            d_out = torch.empty(cap, dtype=torch.uint8, device=dev)
            d_offs = torch.empty(2, dtype=torch.int64, device=dev)
            d_dec = torch.empty_like(d)
            h, w = a.shape[:2]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e_ms, d_ms = [], []
            for k in range(reps + 2):
                ev[0].record(stream)
                codec.encode_tiles(tiles, d_out, d_offs, stream)
                ev[1].record(stream)
                codec.decode_region(d_out, d_offs, tiles, 0, (0, 0, w, h), d_dec, 0, stream)
                ev[2].record(stream)
                torch.cuda.synchronize()
                if k >= 2:
                    e_ms.append(ev[0].elapsed_time(ev[1]))
                    d_ms.append(ev[1].elapsed_time(ev[2]))
            if codec.sync_status(stream) != 0:
                raise RuntimeError(f"{name}: device status")
            n = int(d_offs[1].item())
            got = d_out[:n].cpu().numpy().tobytes()
            dec = d_dec.cpu().numpy()
            dec = dec.view(np.uint16) if a.dtype == np.uint16 else dec
            exact = got == oracle.encode_tile(a, L, bits) and np.array_equal(dec, a)
            em, dm = statistics.median(e_ms), statistics.median(d_ms)
            mpx = w * h / 1e6
            out[name] = {"encode_mps": round(mpx / (em / 1e3), 1), "decode_mps": round(mpx / (dm / 1e3), 1),
                         "encode_ms": round(em, 3), "decode_ms": round(dm, 3), "compressed_bytes": n,
                         "bit_exact": bool(exact)}
    return out


def run_batch(args, dev, n_tiles=4096):
    """Mixed batch: n_tiles tiles of 17-256 px per side, RGB8 and 12-bit mono, 2-6 levels, lossless and lossy,
    encoded and decoded (each tile into its own buffer) as one plan pair replayed from a CUDA graph,
    against the same work issued one tile per call."""
    import torch
    from paper_2005_08713_gb300 import isx, synth
    specs = synth.batch_specs(synth.config_seed(4), n_tiles)
    imgs = [synth.batch_image(sp) for sp in specs]
    # pixels packed into one device buffer, 16-byte aligned per tile
    offs, pos = [], 0
    for a in imgs:
        offs.append(pos)
        pos += (a.nbytes + 15) & ~15
    h_pix = torch.empty(pos, dtype=torch.uint8, pin_memory=True)
    hp = h_pix.numpy()
    for a, o in zip(imgs, offs):
        hp[o:o + a.nbytes] = a.reshape(-1).view(np.uint8)
    d_pix = h_pix.to(dev)
    base = d_pix.data_ptr()
    tiles = []
    for i, (a, sp, o) in enumerate(zip(imgs, specs, offs)):
        bpp = 3 if sp["rgb"] else 2
        tiles.append(isx.Tile(width=sp["w"], height=sp["h"], channels=3 if sp["rgb"] else 1, bits=sp["bits"], levels=sp["levels"],
                              qstep_log2=tuple(sp["q"]), x0=0, y0=0, pixels=base + o, row_pitch_bytes=sp["w"] * bpp, keep=d_pix))
    tarr = isx.TileArray(tiles)
    mp = sum(sp["w"] * sp["h"] for sp in specs) / 1e6
    cap = pos * 2 + 4096 * n_tiles
    d_out = torch.zeros(cap, dtype=torch.uint8, device=dev)
    d_offs = torch.zeros(n_tiles + 1, dtype=torch.int64, device=dev)
    d_dec = torch.zeros(pos, dtype=torch.uint8, device=dev)
    jobs = []
    for i, (sp, o) in enumerate(zip(specs, offs)):
        bpp = 3 if sp["rgb"] else 2
        view = d_dec[o:o + sp["w"] * sp["h"] * bpp].view(sp["h"], sp["w"] * bpp)
        jobs.append((i, (0, 0, sp["w"], sp["h"]), view))
    codec = isx.Codec(dev.index or 0)
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    sched = codec.autotune(tarr, reps=3, stream=stream)
    tune_s = time.perf_counter() - t0
    stamps = torch.zeros(4 * n_tiles, dtype=torch.int64, device=dev)
    codec.set_tile_stamps(stamps)   # the plans record per-tile stamps on every launch
    penc = codec.plan_encode(tarr)
    pdec = codec.plan_decode(tarr, jobs)
    codec.set_tile_stamps(None)
    with torch.cuda.stream(stream):
        penc.launch_encode(d_out, d_offs, stream)
        pdec.launch_decode(d_out, d_offs, stream)
    assert penc.sync_status(stream) == 0 and pdec.sync_status(stream) == 0
    launches = penc.launch_count + pdec.launch_count
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        penc.launch_encode(d_out, d_offs, stream)
        pdec.launch_decode(d_out, d_offs, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps):
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    with torch.cuda.stream(stream):   # replays run on the current stream, the one the events are recorded on
        for _ in range(args.warmup):
            g.replay()
        graph_ms = timed(g.replay, max(3, args.steps))
    tile_lat = stamp_latency(stamps.cpu().numpy().view(np.uint64), n_tiles)

    def eager():
        penc.launch_encode(d_out, d_offs, stream)
        pdec.launch_decode(d_out, d_offs, stream)

    with torch.cuda.stream(stream):
        eager_ms = timed(eager, max(3, args.steps))
    assert penc.sync_status(stream) == 0 and pdec.sync_status(stream) == 0
    # exactness on sampled tiles of the graph's output
    import oracle
    rng = np.random.default_rng(4)
    o_h = d_offs.cpu().numpy()
    ok = True
    sample = rng.choice(n_tiles, 16, replace=False).tolist()
    dec_h = d_dec.cpu().numpy()
    for i in sample:
        sp = specs[i]
        ref = oracle.encode_tile(imgs[i], sp["levels"], sp["bits"], sp["q"])
        got = d_out[int(o_h[i]):int(o_h[i + 1])].cpu().numpy().tobytes()
        bpp = 3 if sp["rgb"] else 2
        dec = dec_h[offs[i]:offs[i] + sp["w"] * sp["h"] * bpp]
        dec = dec.view(np.uint16).reshape(sp["h"], sp["w"]) if not sp["rgb"] else dec.reshape(sp["h"], sp["w"], 3)
        ok = ok and got == ref and np.array_equal(dec, oracle.decode_tile(ref, 0))
    # the same work one tile per call (each call plans, uploads and launches its own kernels)
    per_tile = None
    if not args.no_per_tile:
        one = [isx.TileArray([t]) for t in tiles]

        def per_tile_pass():
            for i in range(n_tiles):
                codec.encode_tiles(one[i], d_out, d_offs, stream)
                codec.decode_jobs(d_out, d_offs, one[i], [(0, jobs[i][1], jobs[i][2])], 0, 0, stream)

        per_tile_pass()
        codec.sync_status(stream)
        t0 = time.perf_counter()
        pt_ms = timed(per_tile_pass, 1)
        pt_wall = time.perf_counter() - t0
        assert codec.sync_status(stream) == 0
        per_tile = {"ms": round(pt_ms, 2), "MP_per_s": round(mp / (pt_ms / 1e3), 1), "wall_s": round(pt_wall, 2),
                    "calls": 2 * n_tiles}
    out = {"workload": f"batch_{n_tiles}_mixed_17to256px_rgb8_mono12_L2to6_lossless_lossy", "tiles": n_tiles,
           "megapixels": round(mp, 2), "unit": "MP/s (encode + decode round trip)",
           "graph": {"ms": round(graph_ms, 3), "MP_per_s": round(mp / (graph_ms / 1e3), 1), "kernels": launches},
           "tile_latency_ms": tile_lat,
           "eager_plans": {"ms": round(eager_ms, 3), "MP_per_s": round(mp / (eager_ms / 1e3), 1)},
           "per_tile_calls": per_tile, "schedule": sched, "autotune_s": round(tune_s, 2),
           "exact": {"sampled_tiles": len(sample), "bit_exact": bool(ok)}}
    if per_tile:
        out["speedup_vs_per_tile"] = round(per_tile["ms"] / graph_ms, 1)
    del g
    penc.close()
    pdec.close()
    codec.close()
    return out


def run_serve(args, dev, pyramids):
    """Viewport serving: Poisson arrivals of 1920x1080 viewport requests at random zoom levels 0-7 and pan
    positions over the slide's lossy and lossless pyramids (device resident), continuous batching over
    several streams, scratch admitted by a per-slot HBM budget."""
    from paper_2005_08713_gb300 import serve
    rates = [float(r) for r in args.serve_rates.split(",")]
    out = {"workload": "serve_viewport_1920x1080_z0to7_slide_lossy_lossless", "unit": "MP/s delivered", "rates": []}
    t0 = time.perf_counter()
    srv = serve.Server(pyramids, device=dev.index or 0, slots=args.serve_slots, max_batch=args.serve_batch,
                       scratch_budget=args.serve_budget_mb << 20,
                       resident_from=None if args.serve_resident_from < 0 else args.serve_resident_from,
                       cache_bytes=args.serve_cache_mb << 20)
    out["resident_levels_from"] = args.serve_resident_from
    out["startup_s"] = round(time.perf_counter() - t0, 2)
    srv.run(serve.poisson_requests(1000.0, 64, pyramids, seed=1))   # warm-up
    for k, rate in enumerate(rates):
        n = int(min(rate * args.serve_seconds, args.serve_cap))
        reqs = serve.poisson_requests(rate, n, pyramids, seed=100 + k)
        done = srv.run(reqs)
        px = sum(r.rect[2] * r.rect[3] for r in done)
        row = {"rate_per_s": rate, "requests": len(done), "elapsed_s": round(srv.elapsed, 3),
               "achieved_per_s": round(len(done) / srv.elapsed, 1), "MP_per_s": round(px / 1e6 / srv.elapsed, 1),
               "batches": srv.n_batches, "mean_batch": round(float(np.mean(srv.batch_sizes)), 2)}
        row.update(serve.latency_stats(done))
        row["cache"] = srv.cache_stats()
        out["rates"].append(row)
    srv.close()
    # the same kind of load served one request per launch on one stream
    one = serve.Server(pyramids, device=dev.index or 0, slots=1, max_batch=1, scratch_budget=args.serve_budget_mb << 20,
                       resident_from=None if args.serve_resident_from < 0 else args.serve_resident_from,
                       cache_bytes=args.serve_cache_mb << 20)
    n = int(min(rates[-1] * args.serve_seconds, args.serve_cap, 4000))
    reqs = serve.poisson_requests(rates[-1], n, pyramids, seed=999)
    done = one.run(reqs)
    px = sum(r.rect[2] * r.rect[3] for r in done)
    out["one_request_per_launch"] = {"rate_per_s": rates[-1], "requests": len(done), "elapsed_s": round(one.elapsed, 3),
                                     "MP_per_s": round(px / 1e6 / one.elapsed, 1), **serve.latency_stats(done)}
    one.close()
    out["slots"], out["max_batch"], out["scratch_budget_mb_per_slot"] = args.serve_slots, args.serve_batch, args.serve_budget_mb
    out["tile_cache_mb"] = args.serve_cache_mb
    return out


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or the machine type."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_single_core():
    """One host core running the oracle on the two single-image workloads:
    the 512 x 512 RGB8 stain tile (3 levels, lossless) and the 2048 x 2048
    12-bit phantom (5 levels, lossless); encode and decode ms, best of 3."""
    import oracle
    from paper_2005_08713_gb300 import synth
    cases = {"stain_512x512_rgb8_L3_lossless": (synth.stain(synth.config_seed(1)), 3, 8),
             "phantom_2048x2048_u12_L5_lossless": (synth.phantom(synth.config_seed(2), 2048, 2048), 5, 12)}
    out = {}
    for name, (img, levels, bits) in cases.items():
        enc, dec = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            s = oracle.encode_tile(img, levels, bits, [0] * (levels + 1))
            t1 = time.perf_counter()
            back = oracle.decode_tile(s)
            t2 = time.perf_counter()
            enc.append(t1 - t0)
            dec.append(t2 - t1)
        if not np.array_equal(back, img):
            raise RuntimeError(f"oracle round trip of {name} is not lossless")
        out[name] = {"encode_ms": round(min(enc) * 1e3, 1), "decode_ms": round(min(dec) * 1e3, 1),
                     "mp": round(img.shape[0] * img.shape[1] / 1e6, 3), "bytes": len(s)}
    return out


def cpu_baseline(img, grid, q, n_tiles):
    """The oracle as it stands, all host cores, on a bounded sample of the workload's tiles."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    idx = rng.choice(len(grid), min(n_tiles, len(grid)), replace=False)
    imgs = [np.ascontiguousarray(img[grid[i][1]:grid[i][1] + grid[i][3], grid[i][0]:grid[i][0] + grid[i][2]]) for i in idx]
    ts = [oracle.tile_struct(a.shape[1], a.shape[0], 3, 8, LEVELS, q) for a in imgs]
    mp = sum(a.shape[0] * a.shape[1] for a in imgs) / 1e6
    t0 = time.perf_counter()
    streams = oracle.encode_tiles_mt(imgs, ts, cores)
    t1 = time.perf_counter()
    outs = [np.zeros_like(a) for a in imgs]
    oracle.decode_tiles_mt(streams, 0, outs, cores)
    t2 = time.perf_counter()
    return {"value": round(mp / (t2 - t0), 2), "unit": "MP/s", "cores": cores, "kind": "oracle",
            "encode_mps": round(mp / (t1 - t0), 2), "decode_mps": round(mp / (t2 - t1), 2),
            "sample": f"{len(imgs)} random 256x256 tiles of the same slide ({mp:.1f} MP), encode+decode, thread pool over tiles",
            "cpu_model": host_cpu_model(), "single_core": oracle_single_core()}


def run_reference(args):
    """The CPU oracle timed on the machine's host cores (reference arm)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from paper_2005_08713_gb300 import synth
    import oracle
    grid = tile_grid()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(5)
    n = args.cpu_tiles
    idx = rng.choice(len(grid), n, replace=False)
    q = LOSSY_Q if not args.lossless else [0] * 9
    seed = synth.config_seed(3)
    imgs = [synth.slide(seed, grid[i][0], grid[i][1], grid[i][2], grid[i][3]) for i in idx]
    ts = [oracle.tile_struct(a.shape[1], a.shape[0], 3, 8, LEVELS, q) for a in imgs]
    mp = sum(a.shape[0] * a.shape[1] for a in imgs) / 1e6
    outs = [np.zeros_like(a) for a in imgs]

    def one():
        s = oracle.encode_tiles_mt(imgs, ts, cores)
        oracle.decode_tiles_mt(s, 0, outs, cores)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    value = mp / dt
    return {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "MP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"slide_{IMG_W}x{IMG_H}_rgb8_tile{TILE}_L{LEVELS}_" + ("lossless" if args.lossless else "lossy_q8421"),
                       "sample_tiles": n},
            "cpu_baseline": {"value": round(value, 2), "unit": "MP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} random tiles of the slide per step ({mp:.1f} MP), encode+decode",
                             "cpu_model": host_cpu_model()},
            "e2e": {"value": round(value, 2), "unit": "MP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lossless", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--cpu-tiles", type=int, default=256)
    ap.add_argument("--size", default=None, help="WxH of the slide instead of 40000x30000 (small cases for profiling)")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-single", action="store_true", help="skip the single-image workloads (512x512 stain, 2048x2048 phantom)")
    ap.add_argument("--no-untiled", action="store_true", help="skip the slide coded as one untiled image")
    ap.add_argument("--no-lossless", action="store_true", help="skip the lossless run of the slide beside the lossy one")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-batch measurement")
    ap.add_argument("--no-per-tile", action="store_true", help="skip the one-tile-per-call comparison of the batch")
    ap.add_argument("--batch-tiles", type=int, default=4096)
    ap.add_argument("--no-serve", action="store_true", help="skip the viewport-serving measurement")
    ap.add_argument("--serve-rates", default="1000,5000,10000,20000,50000")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="arrivals per rate: seconds of Poisson arrivals ...")
    ap.add_argument("--serve-cap", type=int, default=60000, help="... but at most this many requests")
    ap.add_argument("--serve-cache-mb", type=int, default=4096, help="decoded-cell caches of the levels below resident")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-batch", type=int, default=32)
    ap.add_argument("--serve-budget-mb", type=int, default=1024)
    ap.add_argument("--serve-resident-from", type=int, default=3, help="keep levels >= this decoded on the device (-1: none)")
    args = ap.parse_args()
    if args.size:
        global IMG_W, IMG_H
        IMG_W, IMG_H = (int(v) for v in args.size.lower().split("x"))
    if args.impl == "reference":
        res = run_reference(args)
    else:
        res = run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
