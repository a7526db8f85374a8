"""conv1's and conv2's output planes (a1, a2 of Eq. (1)) pixel by pixel against the
oracle with the bf16 path's rounding points (oracle/rounded.py).

The planes are read through the network itself: a probe network keeps the real
layers up to the plane of interest and replaces the rest by centre-tap
selectors (one weight 1 at the kernel centre, zero biases), so that x^ is that
plane's channel c, unchanged: selecting a bfloat16 value with weight 1 is exact
in every later layer.  With Phi = I the proxy x~ is y itself (one product per
output), so the GPU's x~ equals the rounded oracle's bit for bit and every
difference below comes from the layer under test:

  * a1 = bf16(ReLU(conv1(x~) + b1)): the 121 products of bfloat16 operands are
    exact in float32; the float32 sum differs from the exact one by at most
    121 * 2^-24 of the sum of their magnitudes, which can move the result across
    one bfloat16 rounding boundary: each pixel is either equal or one unit in
    the last place (2^-7 of its magnitude at most) apart, and almost all are
    equal.
  * a2 = bf16(ReLU(conv2(a1) + b2)): 7744 products; besides the sum order, the
    few a1 pixels one unit apart enter: each pixel within one unit of a2 plus
    2^-10 of the sum of the magnitudes of its products, most of them equal.

A wrong tap, shift, channel or tile edge moves pixels by far more than that, and
at most pixels.  Both conv1 kernels (position tiles and row tiles) are checked.
"""
import numpy as np
import pytest

from oracle import rounded
import oracle
from paper_1701_03891_gb300 import synth
from _planes import check_plane as _check, selector as _selector

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


def _run(di, params, y, n1, n2, rows_mode):
    import torch
    N = n1 * n2
    phi = np.eye(N, dtype=np.float32)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    net.set_conv1_rows(rows_mode)
    out = net.forward(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    net.close()
    return out


@pytest.mark.parametrize("n1,n2,B,rows_mode", [
    (64, 64, 2, 0),       # position tiles
    (64, 64, 2, 2),       # row tiles, 2 rows per tile
    (37, 50, 2, 0),       # ragged
    (37, 25, 2, 2),       # row tiles, 5 rows per tile
])
def test_planes_a1_a2(di, n1, n2, B, rows_mode):
    N = n1 * n2
    params = synth.he_params(seed=n1 + n2, bias_std=0.01)
    x = synth.voronoi_images(B, n1, n2, seed=n1 * n2)
    y = rounded.bf16(x).astype(np.float32)          # x~ = y exactly (Phi = I)
    ref, c = rounded.forward_bf16(y, params, n1, n2, phi=np.eye(N), keep=True)
    a0, a1, a2 = c["a0"], c["a1"], c["a2"]
    assert np.array_equal(a0.reshape(B, N), y.astype(np.float64))
    # magnitudes of each pixel's products (for the sum-order term)
    w1b = rounded.bf16(params["w1"])
    w2b = rounded.bf16(params["w2"])
    S1 = oracle.conv_same(np.abs(a0), np.abs(w1b)) + np.abs(params["b1"])[None, :, None, None]
    S2 = oracle.conv_same(np.abs(a1), np.abs(w2b)) + np.abs(params["b2"])[None, :, None, None]
    for ch in (0, 29, 63):
        p = dict(params)
        p["w2"] = _selector(32, 64, ch)
        p["b2"] = np.zeros(32, np.float32)
        p["w3"] = _selector(1, 32, 0)
        p["b3"] = np.zeros(1, np.float32)
        got = _run(di, p, y, n1, n2, rows_mode).reshape(B, n1, n2)
        _check(got, a1[:, ch], S1[:, ch], 121 * 2.0 ** -24, 0.97, ("a1", ch, n1, n2, rows_mode))
    for ch in (0, 17, 31):
        p = dict(params)
        p["w3"] = _selector(1, 32, ch)
        p["b3"] = np.zeros(1, np.float32)
        got = _run(di, p, y, n1, n2, rows_mode).reshape(B, n1, n2)
        _check(got, a2[:, ch], S2[:, ch], 2.0 ** -10, 0.6, ("a2", ch, n1, n2, rows_mode))
