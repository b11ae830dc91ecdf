"""The seeded input recipe (CPU): generators are pure functions of their seeds and have the
properties the workloads rely on -- a skewed, peaked histogram for the frequent-value cache,
the stated value ranges, the ragged batch's side range and the serving stream's arrival rate
and operation mix."""
import numpy as np
import pytest

from paper_2409_03568_gb300 import inputs, metrics, workloads as W


def test_generators_are_deterministic_and_typed():
    a = inputs.random_field_image(20, 30, seed=5, channels=3)
    b = inputs.random_field_image(20, 30, seed=5, channels=3)
    c = inputs.random_field_image(20, 30, seed=6, channels=3)
    assert a.shape == (20, 30, 3) and a.dtype == np.uint8
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert inputs.random_field_image(7, 9, seed=1).shape == (7, 9)
    u = inputs.uniform_image(8, 8, seed=1)
    assert u.dtype == np.uint8 and np.array_equal(u, inputs.uniform_image(8, 8, seed=1))
    p = inputs.binary_pattern(16, 16, seed=5)
    assert set(np.unique(p)) <= {0, 255} and 0.3 < (p == 255).mean() < 0.7
    beta = inputs.brightness_beta(4)
    assert -40.0 <= beta <= 40.0 and beta == inputs.brightness_beta(4)


def test_random_field_histogram_is_skewed_like_an_image():
    img = W.image_for(W.ENC8192).reshape(-1)
    counts = np.bincount(img, minlength=256)
    top32 = np.sort(counts)[::-1][:32].sum() / img.size
    # uniform pixels would put 32/256 = 12.5 % in the 32 most frequent values
    assert 0.2 < top32 < 0.45
    assert 100 < img.mean() < 156 and 30 < img.std() < 70


def test_noisy_copy_has_the_stated_noise():
    img = inputs.random_field_image(64, 64, seed=3)
    noisy = inputs.noisy_copy(img, seed=6)
    d = noisy.astype(np.float64) - img
    assert abs(d.mean()) < 0.5 and 4.0 < d.std() < 6.0


def test_ragged_batch_shapes():
    wl = W.BATCH32
    imgs = inputs.ragged_batch(wl["n_images"], wl["batch_seed"], wl["side_lo"], wl["side_hi"])
    assert len(imgs) == 32
    for im in imgs:
        assert im.shape[0] == im.shape[1] and wl["side_lo"] <= im.shape[0] <= wl["side_hi"]
    assert sum(im.size for im in imgs) == 216613   # the batch the benchmark reports


def test_serving_stream_rate_and_mix():
    bench = pytest.importorskip("bench")
    wl = W.SERVE
    reqs = bench.serve_requests(wl, 20.0)
    rate = len(reqs) / 20.0
    assert abs(rate - wl["rate"]) < 0.1 * wl["rate"]
    times = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(times) > 0) and times[-1] < 20.0
    kinds = np.bincount([r["kind"] for r in reqs], minlength=5) / len(reqs)
    want = np.array(wl["op_weights"], dtype=np.float64) / sum(wl["op_weights"])
    assert np.max(np.abs(kinds - want)) < 0.03
    sides = np.array([r["h"] for r in reqs])
    assert sides.min() >= wl["side_lo"] and sides.max() <= wl["side_hi"]
    assert 0.45 < np.mean([r["ring"] for r in reqs]) < 0.55
    assert reqs == bench.serve_requests(wl, 20.0)


def test_package_metrics_match_the_paper_table():
    # the paper's pairs: MSE 0.453 -> 51.56 dB and MSE 218.13 -> 24.74 dB
    assert abs(metrics.psnr(0.453) - 51.57) < 0.02
    assert abs(metrics.psnr(218.13) - 24.74) < 0.01
    assert metrics.mse(np.zeros(4), np.full(4, 2.0)) == 4.0
