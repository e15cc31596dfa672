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
