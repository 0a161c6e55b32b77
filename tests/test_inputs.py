"""The seeded input recipe: what the synthetic stand-ins for the paper's images, filters and workloads are."""
import math

import numpy as np

from paper_1609_05722_gb300 import synth


def test_clean_images_are_normalised_and_seeded():
    a = synth.clean_image(64, 96, 5)
    assert a.shape == (64, 96) and a.min() == 0.0 and a.max() == 1.0
    assert np.array_equal(a, synth.clean_image(64, 96, 5))
    assert not np.array_equal(a, synth.clean_image(64, 96, 6))
    # piecewise-constant shapes on a gradient plus a weak texture: most of the image is smooth
    assert np.median(np.abs(np.diff(a, axis=1))) < 0.05


def test_poisson_observation_is_counts_with_the_peak_as_mean_scale():
    clean = synth.clean_image(256, 256, 9)
    for peak in (1.0, 4.0, 30.0):
        y = synth.poisson_observation(clean, peak, 10)
        assert np.all(y >= 0) and np.array_equal(y, np.round(y))
        m = (peak * clean).mean()
        # the mean of 65536 Poisson draws is within 4 standard errors of its expectation
        assert abs(y.mean() - m) <= 4.0 * math.sqrt(m / y.size)


def test_filter_bank_is_an_orthonormal_zero_mean_family():
    k, a = synth.filter_bank()
    assert k.shape == (48, 7, 7) and a.shape == (48,)
    f = k.reshape(48, 49)
    assert np.abs(f.sum(axis=1)).max() < 1e-12                      # zero mean: constants give no response
    np.testing.assert_allclose(f @ f.T, np.eye(48), atol=1e-12)     # DCT atoms mixed by an orthogonal matrix
    assert a.min() >= 0.5 and a.max() <= 1.5
    k6, a6 = synth.filter_bank(6)
    assert np.array_equal(k6, k[:6]) and np.array_equal(a6, a[:6])


def test_microscopy_tiles():
    t = synth.microscopy_tile(256, 256, 3)
    assert t.max() == 1.0 and t.min() > 0.0
    # sparse blobs on a dark background: most pixels stay near the background level
    assert np.median(t) < 0.25


def test_batched_uneven_set():
    specs = synth.batched_uneven_specs(64, seed=3)
    assert len(specs) == 64
    sides = {128, 256, 384, 512, 768, 1024}
    assert all(s.H in sides and s.W in sides for s in specs)
    assert all(1.0 <= s.peak <= 30.0 and 100 <= s.iters <= 300 for s in specs)
    assert len({(s.H, s.W) for s in specs}) > 10


def test_serving_stream():
    arr = synth.serving_arrivals(2000, 200.0, 42)
    t = np.array([a for a, _ in arr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) <= 4 * (1 / 200.0) / math.sqrt(len(gaps))   # exponential gaps, rate 200/s
    micro = [s for _, s in arr if s.microscopy]
    assert abs(len(micro) / len(arr) - 0.05) <= 4 * math.sqrt(0.05 * 0.95 / len(arr))
    assert all(s.H == s.W == 4096 and 1.0 <= s.peak <= 2.0 for s in micro)
    rest = [s for _, s in arr if not s.microscopy]
    assert all(128 <= s.H <= 2048 and 128 <= s.W <= 2048 and 1.0 <= s.peak <= 30.0 for s in rest)
    assert all(s.iters == (150 if s.peak < 5 else 100) for _, s in arr)
