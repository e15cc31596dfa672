"""The seeded generators: determinism across hosts and workload shape."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_generator_bytes_match_stored_hashes(synth):
    import sys
    sys.path.insert(0, GOLDEN)
    from make_synth_hashes import digests
    stored = {}
    with open(os.path.join(GOLDEN, "synth_hashes.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                stored[k] = v
    assert digests() == stored


def test_crops_are_position_pure(synth):
    s = synth.config_seed(3)
    big = synth.slide(s, 1000, 2000, 300, 200)
    small = synth.slide(s, 1100, 2050, 64, 48, threads=1)
    assert np.array_equal(big[50:98, 100:164], small)
    ph = synth.phantom(7, 512, 512)
    assert np.array_equal(ph[100:120, 30:70], synth.phantom(7, 512, 512, 30, 100, 40, 20))


def test_slide_background_fraction_and_ranges(synth):
    s = synth.config_seed(3)
    rng = np.random.default_rng(0)
    fr = []
    for _ in range(120):
        x, y = int(rng.integers(0, 40000 - 64)), int(rng.integers(0, 30000 - 64))
        c = synth.slide(s, x, y, 64, 64, threads=1)
        fr.append((c.min(axis=2) >= 215).mean())
    assert 0.5 < np.mean(fr) < 0.7


def test_phantom_is_12_bit(synth):
    ph = synth.phantom(synth.config_seed(2), 2048, 2048, 0, 0, 2048, 256)
    assert ph.dtype == np.uint16 and ph.max() <= 4095 and ph.max() > 1000


def test_mixed_batch_recipe(synth):
    """4096 tiles: sides uniform in 17..256, RGB8 slide crops or 12-bit phantom crops with equal odds,
    2..6 levels, lossless or lossy with equal odds; every crop inside its generator's image."""
    import numpy as np
    specs = synth.batch_specs(synth.config_seed(4), 4096)
    assert specs == synth.batch_specs(synth.config_seed(4), 4096)           # seeded
    w = np.array([s["w"] for s in specs]); h = np.array([s["h"] for s in specs])
    assert w.min() >= 17 and w.max() <= 256 and h.min() >= 17 and h.max() <= 256
    assert abs(w.mean() - 136.5) < 3 and abs(h.mean() - 136.5) < 3
    lv = np.array([s["levels"] for s in specs])
    assert set(lv.tolist()) == {2, 3, 4, 5, 6}
    rgb = np.array([s["rgb"] for s in specs])
    assert 0.45 < rgb.mean() < 0.55
    lossy = np.array([any(s["q"]) for s in specs])
    assert 0.45 < lossy.mean() < 0.55
    for s in specs:
        assert len(s["q"]) == s["levels"] + 1
        assert s["bits"] == (8 if s["rgb"] else 12)
        W, H = (40000, 30000) if s["rgb"] else (2048, 2048)
        assert 0 <= s["x0"] and s["x0"] + s["w"] <= W and 0 <= s["y0"] and s["y0"] + s["h"] <= H
    img = synth.batch_image(specs[0])
    assert img.shape[:2] == (specs[0]["h"], specs[0]["w"])
