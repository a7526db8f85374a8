"""Image sizes on both sides of every size-dependent switch of the bf16 forward
pass, each against the FP64 oracle (at the bf16 gates of tests/_precision.py),
the fused conv1 -> conv2 kernel bit for bit, and a repeated pass bit for bit:

  pitch 75 / 76        fused kernel: whole-width walk / column strips
  pitch 124 / 125      conv3: ring of row sums / ring of partial outputs
  64+ tiles per image  conv1: per-tile window pieces / one window ring per CTA
  tall and thin, one row, wide and short (many strips), pitch > 1000
  (the zero border rows conv2 and conv3 skip, ragged last tiles)
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


@pytest.mark.parametrize("n1,n2,B,k", [
    (10, 70, 3, 2),      # pitch 75: the widest whole-width fused walk; conv3 row-sum ring
    (10, 71, 3, 2),      # pitch 76: fused kernel in column strips
    (9, 119, 3, 2),      # pitch 124: conv3 ring of row sums
    (9, 120, 3, 2),      # pitch 125: conv3 ring of partial outputs
    (63, 127, 3, 1),     # 65 conv1 tiles per image: conv1's window ring
    (64, 126, 2, 1),     # 66 tiles, ring, partial-output ring
    (200, 8, 3, 2),      # tall and thin
    (1, 300, 4, 2),      # one row: every tile meets the zero border rows
    (5, 500, 2, 1),      # wide and short: ten column strips
    (12, 1000, 2, 1),    # pitch 1005: conv1's pieces again (window too tall for the ring)
])
def test_size_switches(di, n1, n2, B, k):
    N = n1 * n2
    M = synth.m_for_ratio(0.10, N)
    phi = synth.gaussian_phi(M, N, seed=n1)
    params = synth.he_params(seed=n2, bias_std=0.01)
    x = synth.voronoi_images(B, n1, n2, seed=n1 + n2)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    xhat = net.forward(y).cpu().numpy()
    np.testing.assert_array_equal(net.forward(y).cpu().numpy(), xhat)
    net.set_fused(True)
    np.testing.assert_array_equal(net.forward(y).cpu().numpy(), xhat)
    net.close()
    ref = oracle.forward(oracle.measure(phi, x[:k]), params, n1, n2, phi=phi)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[:k]), params, n1, n2, phi=phi)
    check_images(xhat[:k], ref, rnd, what=(n1, n2))
    assert float(np.max(oracle.rel_l2(xhat[:k], ref))) <= 1e-2
