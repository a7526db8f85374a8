"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests.

This module holds input generation only -- none of the method's arithmetic.
Everything is drawn on the host with numpy's PCG64 generator from a fixed seed
and returned as float32, so the CUDA path and the FP64 oracle see the very same
bits.

* ``gaussian_phi``  -- the measurement matrix of Sec. 1 (y = Phi x).  The paper
  does not state Phi's distribution; entries are i.i.d. N(0, 1/M).
* ``m_for_ratio``   -- M for an undersampling ratio M/N, rounded half up.
* ``he_params``     -- conv weights for the three layers of Sec. 5 (64, 32 and
  1 filters of 11 x 11), He-normal N(0, 2 / fan_in), fan_in = C_in k^2.
* ``dct_sparse_images`` -- images K-sparse in the orthonormal 2-D DCT (the
  x = Psi s model of Sec. 1), min-max normalised to [0, 1].
* ``voronoi_images`` -- piecewise-smooth images (random Voronoi cells with
  linear ramps plus N(0, 0.01) noise), min-max normalised to [0, 1]; these stand
  in for the 64 x 64 ImageNet crops of Sec. 5, which are not available here.
"""
from __future__ import annotations

import math

import numpy as np


def m_for_ratio(ratio: float, N: int) -> int:
    """M = round-half-up(ratio * N), at least 1."""
    return max(1, int(math.floor(ratio * N + 0.5)))


def gaussian_phi(M: int, N: int, seed: int = 0) -> np.ndarray:
    """Phi [M][N] float32, entries i.i.d. N(0, 1/M)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((M, N)) / math.sqrt(M)).astype(np.float32)


def he_params(l1: int = 64, l2: int = 32, l3: int = 1, k: int = 11, seed: int = 1,
              bias_std: float = 0.0, hidden: int = 0) -> dict:
    """w_l [l_l][l_{l-1}][k][k] ~ N(0, 2 / (l_{l-1} k^2)), l_0 = 1; biases N(0, bias_std^2)
    (zero by default).  float32.  ``hidden`` inserts that many l2 -> l2 layers
    between conv2 and the last layer (keys w1..wL in network order, L = 3 + hidden);
    with hidden = 0 the draws are those of the three-layer network."""
    rng = np.random.default_rng(seed)
    out = {}
    cins = [1, l1] + [l2] * hidden + [l2]
    couts = [l1, l2] + [l2] * hidden + [l3]
    for i, (ci, co) in enumerate(zip(cins, couts), start=1):
        std = math.sqrt(2.0 / (ci * k * k))
        out["w%d" % i] = (rng.standard_normal((co, ci, k, k)) * std).astype(np.float32)
        if bias_std > 0:
            out["b%d" % i] = (rng.standard_normal(co) * bias_std).astype(np.float32)
        else:
            out["b%d" % i] = np.zeros(co, dtype=np.float32)
    return out


def _minmax(x: np.ndarray) -> np.ndarray:
    B = x.shape[0]
    f = x.reshape(B, -1)
    lo = f.min(axis=1, keepdims=True)
    hi = f.max(axis=1, keepdims=True)
    return ((f - lo) / np.maximum(hi - lo, 1e-30)).reshape(x.shape)


def dct_sparse_images(B: int, n1: int, n2: int, K: int, seed: int = 2) -> np.ndarray:
    """[B][n1*n2] float32: K support positions uniform without replacement over all
    n1*n2 orthonormal DCT-II coefficients (DC included), values N(0,1), inverse
    2-D DCT, then per-image min-max to [0, 1]."""
    from scipy.fft import idctn
    rng = np.random.default_rng(seed)
    N = n1 * n2
    out = np.empty((B, n1, n2), dtype=np.float64)
    for b in range(B):
        s = np.zeros(N)
        idx = rng.choice(N, size=min(K, N), replace=False)
        s[idx] = rng.standard_normal(idx.size)
        out[b] = idctn(s.reshape(n1, n2), norm="ortho")
    return _minmax(out).reshape(B, N).astype(np.float32)


def voronoi_images(B: int, n1: int, n2: int, seed: int = 3) -> np.ndarray:
    """[B][n1*n2] float32 piecewise-smooth images: 8..20 Voronoi cells (sites
    uniform over the image), each cell a ramp a + b r/n1 + c col/n2 with a, b, c
    ~ U(-1, 1), plus i.i.d. N(0, 0.01) noise (variance 0.01), then per-image
    min-max to [0, 1]."""
    rng = np.random.default_rng(seed)
    rr, cc = np.meshgrid(np.arange(n1, dtype=np.float64), np.arange(n2, dtype=np.float64),
                         indexing="ij")
    out = np.empty((B, n1, n2), dtype=np.float64)
    for b in range(B):
        ncell = int(rng.integers(8, 21))
        sr = rng.uniform(0, n1, ncell)
        sc = rng.uniform(0, n2, ncell)
        coef = rng.uniform(-1, 1, (ncell, 3))
        d2 = (rr[None] - sr[:, None, None]) ** 2 + (cc[None] - sc[:, None, None]) ** 2
        lab = np.argmin(d2, axis=0)
        a, bb, c = coef[lab, 0], coef[lab, 1], coef[lab, 2]
        img = a + bb * rr / n1 + c * cc / n2
        img = img + rng.standard_normal((n1, n2)) * 0.1
        out[b] = img
    return _minmax(out).reshape(B, n1 * n2).astype(np.float32)
