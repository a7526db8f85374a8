"""Recovery-quality evaluation (Sec. 5): the package's metrics against the
oracle's pinned definitions, the measurement noise against its SNR, and (GPU)
a short training run that must recover the held-out images much better than
the untrained network."""
import numpy as np
import pytest

import oracle
from paper_1701_03891_gb300 import evaluate, synth


def test_metrics_match_oracle():
    rng = np.random.default_rng(0)
    x = synth.voronoi_images(6, 16, 16, seed=1)
    xh = np.clip(x + 0.05 * rng.standard_normal(x.shape), 0, 1)
    np.testing.assert_allclose(evaluate.psnr(xh, x), oracle.psnr(xh, x), rtol=1e-12)
    bad = x + 0.6 * rng.standard_normal(x.shape)
    both = np.concatenate([xh, bad])
    ref = np.concatenate([x, x])
    np.testing.assert_array_equal(evaluate.success(both, ref), oracle.success(both, ref))
    assert evaluate.success(both, ref).tolist() == [1] * 6 + [0] * 6


@pytest.mark.parametrize("snr", [10.0, 20.0, 30.0])
def test_noise_has_the_requested_snr(snr):
    y = np.random.default_rng(2).standard_normal((64, 500)).astype(np.float32) * 3.0
    yn = evaluate.add_noise(y, snr, seed=3)
    e = yn.astype(np.float64) - y
    got = 10 * np.log10(np.sum(y.astype(np.float64) ** 2) / np.sum(e * e))
    assert abs(got - snr) < 0.1, got
    assert evaluate.add_noise(y, None, seed=3) is y


@pytest.mark.gpu
def test_training_improves_recovery():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build
    build.build()
    clean = evaluate.train_and_evaluate(32, 0.25, steps=3000, test_images=32)
    noisy = evaluate.train_and_evaluate(32, 0.25, steps=3000, test_images=32, snr_db=20.0)
    for r in (clean, noisy):
        assert r["loss_last"] < 0.05 * r["loss_first"], r
        assert r["psnr_db"] > r["psnr_db_before"] + 5.0, r
        assert 0.0 <= r["success"] <= 1.0
    assert noisy["psnr_db"] <= clean["psnr_db"] + 0.5


@pytest.mark.gpu
def test_convergence_curve_64():
    """Training a 64 x 64 network records test PSNR every 500 steps; the last point
    matches the returned result and training has raised it well above the start."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build
    build.build()
    r = evaluate.train_and_evaluate(64, 0.10, steps=1500, test_images=16, curve_every=500)
    steps = [c[0] for c in r["curve"]]
    assert steps == [0, 500, 1000, 1500]
    assert abs(r["curve"][-1][1] - r["psnr_db"]) < 1e-9
    assert r["curve"][-1][1] > r["curve"][0][1] + 5.0, r["curve"]
