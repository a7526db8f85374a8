"""The seeded input generators follow the recipe they state: M rounded half up
(reading C7), Phi i.i.d. N(0, 1/M) (C6), He-normal conv weights (C11), images
K-sparse in the orthonormal 2-D DCT and min-max normalised to [0, 1] (C13).
Both the oracle and the CUDA path take their inputs from these generators, so
a slip here (a transform along one axis only, a variance read as a standard
deviation, a truncating M) would go unnoticed by every parity test."""
import math

import numpy as np
import pytest
from scipy.fft import dctn

from paper_1701_03891_gb300 import synth


@pytest.mark.parametrize("ratio,N,M", [
    (0.1, 4096, 410), (0.05, 4096, 205), (0.25, 4096, 1024),     # 64 x 64
    (0.1, 1024, 102), (0.05, 1024, 51), (0.25, 1024, 256),       # 32 x 32
    (0.1, 65536, 6554),                                          # 256 x 256
    (0.5, 5, 3),                                                 # an exact half rounds up
    (0.001, 10, 1),                                              # never below one measurement
])
def test_m_for_ratio_rounds_half_up(ratio, N, M):
    assert synth.m_for_ratio(ratio, N) == M


def test_gaussian_phi_variance_and_seed():
    M, N = 410, 4096
    phi = synth.gaussian_phi(M, N, seed=0)
    assert phi.shape == (M, N) and phi.dtype == np.float32
    assert np.array_equal(phi, synth.gaussian_phi(M, N, seed=0))
    assert not np.array_equal(phi, synth.gaussian_phi(M, N, seed=1))
    f = phi.astype(np.float64)
    n = f.size
    # mean 0 and variance 1/M, within 6 standard errors of the estimates
    assert abs(f.mean()) <= 6 * math.sqrt(1.0 / M / n)
    assert abs(f.var() * M - 1.0) <= 6 * math.sqrt(2.0 / n)
    # hence columns of unit expected norm: E ||Phi e_j||^2 = 1
    assert abs(np.mean(np.sum(f * f, axis=0)) - 1.0) <= 6 * math.sqrt(2.0 / n)


def test_he_params_variances_and_layout():
    p = synth.he_params(seed=1)
    assert [p["w%d" % i].shape for i in (1, 2, 3)] == [(64, 1, 11, 11), (32, 64, 11, 11), (1, 32, 11, 11)]
    for i, fan_in in ((1, 121), (2, 64 * 121), (3, 32 * 121)):
        w = p["w%d" % i].astype(np.float64)
        assert not np.any(p["b%d" % i])                         # biases zero by default
        # sample variance of n normal draws: relative standard error sqrt(2 / n)
        assert abs(w.var() * fan_in / 2.0 - 1.0) <= 6 * math.sqrt(2.0 / w.size)
    b = synth.he_params(seed=1, bias_std=0.5)["b2"].astype(np.float64)
    assert b.shape == (32,) and 0.2 < b.std() < 0.8
    deep = synth.he_params(seed=1, hidden=2)
    assert sorted(deep) == sorted("%s%d" % (t, i) for t in "wb" for i in range(1, 6))
    assert np.array_equal(deep["w1"], p["w1"]) and np.array_equal(deep["w2"], p["w2"])
    assert deep["w3"].shape == deep["w4"].shape == (32, 32, 11, 11) and deep["w5"].shape == (1, 32, 11, 11)
    w3 = deep["w3"].astype(np.float64)
    assert abs(w3.var() * 32 * 121 / 2.0 - 1.0) <= 6 * math.sqrt(2.0 / w3.size)


@pytest.mark.parametrize("n1,n2,K", [(32, 32, 50), (64, 64, 200), (16, 24, 7)])
def test_dct_sparse_images_are_k_sparse_in_the_2d_dct(n1, n2, K):
    B = 6
    x = synth.dct_sparse_images(B, n1, n2, K=K, seed=2)
    assert x.shape == (B, n1 * n2) and x.dtype == np.float32
    assert np.array_equal(x, synth.dct_sparse_images(B, n1, n2, K=K, seed=2))
    for b in range(B):
        img = x[b].astype(np.float64)
        assert img.min() == 0.0 and abs(img.max() - 1.0) <= 1e-6
        c = dctn(img.reshape(n1, n2), norm="ortho")
        # min-max normalisation scales the K drawn coefficients and moves only
        # the DC term (a constant image is pure DC in the orthonormal DCT-II);
        # the float32 rounding of the pixels leaves the others near 1e-7
        big = np.abs(c) > 1e-5
        big[0, 0] = False
        assert K - 1 <= int(big.sum()) <= K, (b, int(big.sum()))


def test_voronoi_images_range_and_seed():
    x = synth.voronoi_images(8, 64, 64, seed=3)
    assert x.shape == (8, 4096) and x.dtype == np.float32
    assert np.array_equal(x, synth.voronoi_images(8, 64, 64, seed=3))
    assert np.all(x.min(axis=1) == 0.0) and np.all(np.abs(x.max(axis=1) - 1.0) <= 1e-6)
    assert len({x[b].tobytes() for b in range(8)}) == 8
    # piecewise smooth: horizontal neighbours differ far less than random pixels do
    img = x.reshape(8, 64, 64).astype(np.float64)
    near = np.median(np.abs(np.diff(img, axis=2)))
    far = np.median(np.abs(img[:, :, :32] - img[:, :, 32:]))
    assert near < 0.5 * far
