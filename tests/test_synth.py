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


def test_series_match_the_library_functions(synth):
    """The generators' own ln x, cos(2 pi u) and ln k! (series in +, -, *, / only, for identical bytes on
    every host) agree with libm / the Gamma function to about double precision."""
    import math
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.random(3000) + 1e-300, np.exp(rng.uniform(-700, 700, 3000)), [1.0, 0.5, 2.0, 2.0 ** -1074]])
    u = np.concatenate([rng.random(len(x) - 6), [0.0, 0.125, 0.25, 0.5, 0.75, 0.999999]])
    k = rng.integers(0, 5000, len(x))
    ln_x, cos_u, ln_k = synth.series(x, u, k)
    assert np.allclose(ln_x, np.log(x), rtol=4e-16, atol=4e-16 * 745)
    assert np.max(np.abs(cos_u - np.cos(2 * np.pi * u))) < 2e-15
    ref = np.array([math.lgamma(int(v) + 1) for v in k])
    assert np.allclose(ln_k, ref, rtol=1e-13, atol=1e-13)


def test_normal_sampler_is_standard_normal(synth):
    """Box-Muller deviates: mean 0, variance 1, normal tails, and a Kolmogorov-Smirnov distance within
    what 400 000 draws from N(0, 1) give."""
    z = synth.normals(12345, 400_000)
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n) and abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(np.abs(z) > 3) - 0.0026998) < 0.0005   # Irwin-Hall sums would cut the tails
    from math import erf, sqrt
    zs = np.sort(z)
    cdf = 0.5 * (1 + np.vectorize(erf)(zs / sqrt(2)))
    ks = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n))
    assert ks < 1.95 / np.sqrt(n)   # the 0.1 % point of the KS statistic is about 1.95 / sqrt(n)


def test_poisson_sampler_has_the_poisson_law(synth):
    """Small means (inter-arrival counting) and large ones (transformed rejection): sample mean and
    variance near lam, and a chi-square fit of the probabilities on the central values."""
    from math import exp, lgamma, log
    for lam in (0.3, 3.5, 9.9, 10.0, 60.0, 517.25, 4095.0):
        s = synth.poissons(lam, 777 + int(lam * 8), 200_000)
        n = len(s)
        assert s.min() >= 0
        assert abs(s.mean() - lam) < 5 * np.sqrt(lam / n), lam
        assert abs(s.var() / lam - 1) < 5 * np.sqrt(2 / n) + 1e-3, lam
        # chi-square over the values with expected counts >= 50, the rest pooled at both ends
        lo, hi = int(s.min()), int(s.max())
        ks = np.arange(lo, hi + 1)
        p = np.array([exp(-lam + k * log(lam) - lgamma(k + 1)) if lam > 0 else 0.0 for k in ks])
        obs = np.bincount(s - lo, minlength=len(ks)).astype(float)
        keep = p * n >= 50
        exp_in = p[keep] * n
        chi = np.sum((obs[keep] - exp_in) ** 2 / exp_in)
        dof = int(keep.sum()) - 1
        assert chi < dof + 5 * np.sqrt(2 * dof) + 10, (lam, chi, dof)


def test_phantom_noise_is_poisson_about_the_smooth_value(synth):
    """On a flat patch of the phantom (the ellipse field nearly constant there) the pixel values scatter
    like Poisson samples about it: the variance is close to the mean."""
    ph = synth.phantom(synth.config_seed(2), 2048, 2048, 0, 0, 64, 64).astype(float)
    # the corner lies outside every ellipse: the field is the constant 60
    assert abs(ph.mean() - 60) < 1.0 and abs(ph.var() / 60 - 1) < 0.15
