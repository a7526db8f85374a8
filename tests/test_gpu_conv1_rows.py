"""conv1 in row tiles (input windows kept in TMEM, each shared by the tiles of
several rows) against conv1 in tiles of 128 consecutive plane positions, and
against the FP64 oracle.

Both kernels issue the same tensor-core products in the same order per output
(kernel rows dy = 0..10, K = the 16 columns dx with zero weights past 11) and the
same epilogue (bias, ReLU, round to bfloat16 or scale and round to e4m3), so the
saved activation buffer (x~, a1 with its zero pad columns, a2, ...) and x^ must be
identical byte for byte.  Sizes cover every rows-per-tile count (1 to 5), a last
row block cut short, one-row images, column segments (2, 3 and 8 per image),
widths that do not fit (which keep the consecutive-position tiles), batches whose
CTAs take several tiles across column and image boundaries, e4m3 networks and the
benchmark workload in full.
"""
import numpy as np
import pytest

import oracle
from oracle import rounded
from paper_1701_03891_gb300 import synth
from _precision import check_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def di():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    deepinv.lib()
    return deepinv


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(n1, n2, ratio, B, seed):
    N = n1 * n2
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=seed)
    params = synth.he_params(seed=seed + 1, bias_std=0.01)
    x = synth.voronoi_images(B, n1, n2, seed=seed + 2)
    return phi, params, x


def _both_saved(di, phi, params, x, n1, n2):
    """x^ and the saved activation bytes with conv1 in row tiles and without."""
    import torch
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    B = x.shape[0]
    out = {}
    for rows in (False, True):
        net.set_conv1_rows(2 if rows else 0)
        saved = torch.zeros(net.saved_bytes(B), dtype=torch.uint8, device="cuda")
        xh = net.forward(y, saved=saved).cpu().numpy()
        out[rows] = (xh, saved.cpu().numpy())
    net.close()
    return out


@pytest.mark.parametrize("n1,n2,B", [
    (64, 64, 6),      # 2 rows per tile, all 128 lanes
    (63, 64, 3),      # last row block one row
    (1, 64, 4),       # one-row images
    (40, 32, 3),      # 4 rows per tile
    (37, 25, 3),      # 5 rows per tile, last block 2 rows
    (30, 48, 2),      # 96 lanes used
    (33, 100, 2),     # one row per tile, 100 lanes
    (20, 128, 2),     # one full row per tile
    (16, 256, 2),     # 2 segments of 128
    (9, 300, 2),      # 3 segments of 100
    (5, 1000, 1),     # 8 segments of 125
    (12, 70, 2),      # does not fit: consecutive-position tiles either way
])
def test_conv1_rows_bit_identical(di, n1, n2, B):
    phi, params, x = _case(n1, n2, 0.10, B, seed=n1 * 7 + n2)
    out = _both_saved(di, phi, params, x, n1, n2)
    np.testing.assert_array_equal(out[True][0], out[False][0])
    np.testing.assert_array_equal(out[True][1], out[False][1])
    assert np.all(np.isfinite(out[True][0]))


@pytest.mark.parametrize("n1,n2", [(64, 64), (37, 25), (9, 300)])
def test_conv1_rows_oracle(di, n1, n2):
    B, k = 3, 2
    phi, params, x = _case(n1, n2, 0.10, B, seed=n1 + 3 * n2)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    net.set_conv1_rows(2)
    xhat = net.forward(net.measure(_cuda(x))).cpu().numpy()
    net.close()
    ref = oracle.forward(oracle.measure(phi, x[:k]), params, n1, n2, phi=phi)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[:k]), params, n1, n2, phi=phi)
    check_images(xhat[:k], ref, rnd, what=("conv1 row tiles", n1, n2))
    assert float(np.max(oracle.rel_l2(xhat[:k], ref))) <= 1e-2


@pytest.mark.parametrize("n1,n2,B", [
    (64, 64, 64),     # CTAs take several tiles, runs cross image boundaries
    (24, 256, 40),    # runs cross segment boundaries
])
def test_conv1_rows_many_tiles_per_cta(di, n1, n2, B):
    phi, params, x = _case(n1, n2, 0.10, B, seed=n2 + B)
    out = _both_saved(di, phi, params, x, n1, n2)
    np.testing.assert_array_equal(out[True][0], out[False][0])
    np.testing.assert_array_equal(out[True][1], out[False][1])


def test_conv1_rows_full_batch_and_repeat(di):
    """64 x 64, M/N = 0.1, batch 1024 (the benchmark workload): x^ identical to the
    consecutive-position tiles on every image, and across repeated passes."""
    n1 = n2 = 64
    B = 1024
    phi, params, x = _case(n1, n2, 0.10, B, seed=21)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    net.set_conv1_rows(0)
    ref = net.forward(y).cpu().numpy()
    net.set_conv1_rows(2)
    got = net.forward(y).cpu().numpy()
    again = net.forward(y).cpu().numpy()
    net.close()
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(again, got)


@pytest.mark.parametrize("n1,n2,B", [(64, 64, 8), (128, 128, 2), (9, 300, 2)])
def test_conv1_rows_e4m3(di, n1, n2, B):
    """e4m3 networks: conv1 writes scaled e4m3 a1; identical either way."""
    phi, params, x = _case(n1, n2, 0.10, B, seed=n1 + n2 + 5)
    net = di.Net(phi, params, n1, n2, prec="fp8")
    y = net.measure(_cuda(x))
    net.calibrate(y)
    res = []
    for rows in (False, True):
        net.set_conv1_rows(2 if rows else 0)
        res.append(net.forward(y).cpu().numpy())
    net.close()
    np.testing.assert_array_equal(res[1], res[0])
    assert np.all(np.isfinite(res[1]))


def test_conv1_rows_modes(di):
    """Mode 1 (the default) picks row tiles only where they are faster; modes
    outside 0..2 are rejected; every mode gives the same x^."""
    n1, n2 = 8, 256
    phi, params, x = _case(n1, n2, 0.10, 2, seed=9)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    outs = []
    for mode in (0, 1, 2):
        net.set_conv1_rows(mode)
        outs.append(net.forward(y).cpu().numpy())
    with pytest.raises(RuntimeError):
        net.set_conv1_rows(3)
    net.close()
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])
