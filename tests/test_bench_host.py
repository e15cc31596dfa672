"""Host-side parts of the benchmark's CPU baseline (no GPU): the oracle's
single-core timings of the two single-image workloads, and the CPU model
recorded beside them."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_single_core_workloads():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_single_core()   # raises if a round trip is not lossless
    stain, phantom = r["stain_512x512_rgb8_L3_lossless"], r["phantom_2048x2048_u12_L5_lossless"]
    assert stain["mp"] == 0.262 and phantom["mp"] == 4.194
    # the oracle stays usable as a checker: the 512 x 512 tile in under a second, both directions
    assert stain["encode_ms"] + stain["decode_ms"] < 1000.0
    # lossless streams of real content are smaller than the samples they code
    assert 0 < stain["bytes"] < 512 * 512 * 3
    assert 0 < phantom["bytes"] < 2048 * 2048 * 2


def test_host_cpu_model_is_named():
    sys.path.insert(0, ROOT)
    import bench
    m = bench.host_cpu_model()
    assert isinstance(m, str) and m.strip()


def test_cpu_baseline_on_a_small_slide():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2005_08713_gb300 import synth
    img = synth.slide(bench.replica_seed(0), 0, 0, 600, 300)
    grid = bench.tile_grid(600, 300)
    assert len(grid) == 3 * 2 and grid[-1] == (512, 256, 88, 44)
    r = bench.cpu_baseline(img, grid, bench.LOSSY_Q, 4)
    assert r["kind"] == "oracle" and r["unit"] == "MP/s" and r["cores"] >= 1
    assert r["value"] > 0 and r["encode_mps"] > 0 and r["decode_mps"] > 0
    assert r["cpu_model"] and set(r["single_core"]) == {"stain_512x512_rgb8_L3_lossless",
                                                         "phantom_2048x2048_u12_L5_lossless"}


def _smi_line(t, sm, reasons=()):
    import datetime
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if nm in reasons else "Not Active" for nm in ("hw_slowdown", "hw_thermal_slowdown",
                                                                     "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join([stamp, "0", str(sm), "2070", "900.5", "0x0"] + flags)


def test_clock_summary_keeps_the_timed_region():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.t_start, c.t_end = 1_700_000_010.0, 1_700_000_011.0
    lines = [_smi_line(1_700_000_009.5, 1200),                              # warm-up, before the region
             _smi_line(1_700_000_010.2, 2070), _smi_line(1_700_000_010.4, 2055, {"sw_power_cap"}),
             _smi_line(1_700_000_010.6, 2070),
             _smi_line(1_700_000_011.3, 900, {"hw_slowdown"}),               # after the region
             "garbage line", ""]
    r = c.summary(lines)
    assert r["samples"] == 3 and r["samples_total"] == 5
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_summary_of_a_region_between_two_samples():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.t_start, c.t_end = 1_700_000_010.00, 1_700_000_010.05
    r = c.summary([_smi_line(1_700_000_009.9, 1500), _smi_line(1_700_000_010.1, 2070, {"sw_thermal_slowdown"})])
    # the first sample after the region started stands for it
    assert r["samples"] == 1 and r["sm_mhz"] == 2070 and r["reasons"] == ["sw_thermal_slowdown"]
    # unparseable timestamps: every sample counts
    c2 = bench.ClockSampler(0)
    c2.t_start, c2.t_end = 1.0, 2.0
    r2 = c2.summary(["??, 0, 1980, 2070, 800, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert r2["samples"] == 1 and r2["sm_mhz"] == 1980 and r2["reasons"] == []


def test_clock_sampler_runs_a_sampling_process(tmp_path):
    """start/mark/stop around a fake nvidia-smi that prints a sample every 50 ms."""
    import time
    fake = tmp_path / "fake-smi"
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import datetime, sys, time\n"
        "assert sys.argv[1:3] == ['-i', '0'] and sys.argv[3].startswith('--query-gpu=timestamp,')\n"
        "while True:\n"
        "    s = datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]\n"
        "    print(s + ', 0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
        "    time.sleep(0.05)\n")
    fake.chmod(0o755)
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0, exe=str(fake))
    c.start()
    time.sleep(0.5)
    c.mark_start()
    time.sleep(0.6)
    c.mark_end()
    r = c.stop()
    assert r["sm_mhz"] == 2070 and r["reasons"] == []
    assert 5 <= r["samples"] <= r["samples_total"], r
    assert c.proc.poll() is not None   # the sampler is gone


def test_clock_sampler_without_nvidia_smi():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0, exe="/nonexistent/nvidia-smi")
    c.start()
    c.mark_start()
    c.mark_end()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _blocks_of_tile(w, h, levels, channels):
    """(p, padded w, padded h) of each block in stream order, from the container's documented order: per
    channel the LL band, then the high-pass bands of levels L .. 1, each cut into 128 x 128 cells in raster
    order; a level-l band is ceil(w / 2^l) x ceil(h / 2^l); blocks are padded to multiples of 4."""
    out = []
    for _ in range(channels):
        bands = [(1, levels)] + [(3, l) for l in range(levels, 0, -1)]
        for p, l in bands:
            bw, bh = ((w - 1) >> l) + 1, ((h - 1) >> l) + 1
            for cy in range(0, bh, 128):
                for cx in range(0, bw, 128):
                    cw, chh = min(128, bw - cx), min(128, bh - cy)
                    out.append((p, -(-cw // 4) * 4, -(-chh // 4) * 4))
    return out


def _kept_bytes_by_parsing(streams, geoms):
    import numpy as np
    from blockparse import Bits
    n, total = 0, 0
    for s, geo in zip(streams, geoms):
        assert s[:4] == b"ISX1"
        nb = int(np.frombuffer(s[12:16], "<u4")[0])
        assert nb == len(geo)
        ends = np.frombuffer(s[32:32 + 4 * nb], "<u4")
        data = 32 + 4 * nb
        begin = 0
        for (p, bw, bh), end in zip(geo, ends):
            b = Bits(s, 8 * (data + begin))
            d = b.get(5)
            removed = sum(b.get(1) for _ in range(p * d))
            total += (p * d - removed) * (bw * bh // 8)
            n += 1
            begin = int(end)
    return n, total


def _check_kept_symbol_bytes(orc, imgs, grid, levels, channels, bits, q):
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    streams = [orc.encode_tile(a, levels, bits, q) for a in imgs]
    offs = np.concatenate(([0], np.cumsum([len(s) for s in streams]))).astype(np.int64)
    raw = np.frombuffer(b"".join(streams), np.uint8)
    geoms = [_blocks_of_tile(w, h, levels, channels) for (_, _, w, h) in grid]
    for (_, _, w, h), g in zip(grid, geoms):
        assert [tuple(int(v) for v in b) for b in bench.block_geometry(w, h, levels, channels)] == g
    got = bench.kept_symbol_bytes(raw, offs, grid, levels, channels)
    assert got == _kept_bytes_by_parsing(streams, geoms)
    return got


def test_kept_symbol_bytes_of_slide_tiles(orc, synth):
    """The benchmark's algorithmic bytes come from the block headers of its own stream; count them again with
    the independent block reader on oracle streams (edge tiles included, lossy and lossless)."""
    sys.path.insert(0, ROOT)
    import bench
    W, H = 600, 300
    img = synth.slide(bench.replica_seed(0), 0, 0, W, H)
    grid = bench.tile_grid(W, H)
    tiles = [img[y:y + h, x:x + w] for (x, y, w, h) in grid]
    for q in (bench.LOSSY_Q, [0] * 9):
        nb, kept = _check_kept_symbol_bytes(orc, tiles, grid, 8, 3, 8, q)
        assert nb > 0 and kept > 0


def test_kept_symbol_bytes_of_a_12_bit_mono_tile(orc, synth):
    a = synth.phantom(synth.config_seed(2), 2048, 2048, 300, 500, 200, 130)
    _check_kept_symbol_bytes(orc, [a], [(0, 0, 200, 130)], 5, 1, 12, [0] * 6)


def test_traffic_figures_follow_the_source_digest(tmp_path, monkeypatch):
    """ncu traffic is reported only for the kernel code it was captured on: comments and whitespace may
    change, code may not."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    for stage, ent in bench.NCU_TRAFFIC.items():
        valid = bench.source_digest(ent[1]) == ent[2]
        t = bench.traffic_bytes(stage, 1_000_000)
        assert (t == int(ent[3] * 1_000_000)) if valid else (t is None), stage
    assert bench.traffic_bytes("no.such.stage", 10) is None
    # a copy of the sources: comment and whitespace edits keep the digest, a code edit changes it
    csrc = tmp_path / "paper_2005_08713_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2005_08713_gb300", "csrc"), csrc)
    names = ("isx_decode.cu", "isx_internal.cuh")
    before = bench.source_digest(names)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.source_digest(names) == before
    p = csrc / "isx_decode.cu"
    src = p.read_text()
    p.write_text("// a new comment\n/* and a\n   block comment */\n" + src.replace("\n", "\n\n", 3) + "   \n")
    assert bench.source_digest(names) == before
    p.write_text(src + "\nstatic int isx_extra_symbol = 1;\n")
    assert bench.source_digest(names) != before
    # a missing file makes the figure unavailable, not an error
    p.unlink()
    assert bench.traffic_bytes("decode.segments", 10) is None


def test_optional_measurements_fail_soft():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.soft(lambda a, b=0: a + b, 2, b=3) == 5

    def broken():
        raise RuntimeError("device status 3")
    r = bench.soft(broken)
    assert r == {"error": "RuntimeError: device status 3"}
    assert len(bench.soft(lambda: (_ for _ in ()).throw(ValueError("x" * 1000)))["error"]) == 400


def test_slide_workload_geometry():
    """40000 x 30000 pixels in 256 x 256 tiles: 157 x 118 = 18 526 tiles, the right column 64 wide, the
    bottom row 48 tall; the tiles cover the image exactly once."""
    sys.path.insert(0, ROOT)
    import bench
    grid = bench.tile_grid(40000, 30000)
    assert len(grid) == 157 * 118 == 18526
    assert {w for (x, _, w, _) in grid if x == 156 * 256} == {64}
    assert {h for (_, y, _, h) in grid if y == 117 * 256} == {48}
    assert sum(w * h for (_, _, w, h) in grid) == 40000 * 30000
    assert grid[0] == (0, 0, 256, 256) and grid[-1] == (156 * 256, 117 * 256, 64, 48)
    # row-major order: the offsets index of tile (row r, column c) is r * 157 + c
    assert grid[157] == (0, 256, 256, 256)
    assert bench.LEVELS == 8 and bench.LOSSY_Q[:4] == [3, 2, 1, 0]


def test_stage_issue_fraction(monkeypatch):
    """A stage's issue fraction: its captured warp instructions per pixel x pixels over its event time,
    against SMs x 4 schedulers x the SM clock; None without a valid capture or a clock."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "issue_roofline", lambda stage, px, ms: (7.26, 152) if stage == "decode.inverse_transform" else None)
    px = 40000 * 30000
    f = bench.stage_issue_frac("decode.inverse_transform", px, 13.809, {"sm_mhz": 2070.0})
    assert abs(f - 7.26 * px / 13.809e-3 / (152 * 4 * 2070e6)) < 1e-4 and 0.49 < f < 0.51
    assert bench.stage_issue_frac("encode.emit", px, 6.7, {"sm_mhz": 2070.0}) is None
    assert bench.stage_issue_frac("decode.inverse_transform", px, 13.809, {}) is None
    # every stage with captured instructions also has captured traffic (the same validity rule applies to both)
    assert set(bench.NCU_WARP_INST_PER_PX) == set(bench.NCU_TRAFFIC)
