"""The float32 path above the CUDA grid limits: a batch of more than 65 535 x 64
images, so that the measurement and FC GEMMs run their rows in two launches (at
most 65 535 row tiles of 64 rows each) and the convolutions run their images in
65-launch chunks (at most 65 535 images per launch).  A tiny network (2 x 2
images, 2 channels, 3 x 3 kernels) keeps it to a few hundred MB.

Every kernel computes each output from its own image only, in a fixed order, so
images on both sides of every launch boundary must match the same images run in
a small batch bit for bit, and the FP64 oracle to float32 accuracy.
"""
import numpy as np
import pytest

import oracle
from paper_1701_03891_gb300 import synth

pytestmark = pytest.mark.gpu

GEMM_ROWS = 65535 * 64          # rows of one sgemm launch
CONV_IMAGES = 65535             # images of one convolution launch


@pytest.fixture(scope="module")
def di():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    deepinv.lib()
    return deepinv


def test_f32_batches_past_grid_limits(di):
    import torch
    n1 = n2 = 2
    N = n1 * n2
    M = 2
    B = GEMM_ROWS + 100
    phi = synth.gaussian_phi(M, N, seed=7)
    params = synth.he_params(l1=2, l2=2, l3=1, k=3, seed=8, bias_std=0.05)
    rng = np.random.default_rng(9)
    x = rng.random((B, N), dtype=np.float32)
    net = di.Net(phi, params, n1, n2, prec="f32")
    xd = torch.from_numpy(x).cuda()
    y = net.measure(xd)
    xhat = net.forward(y)
    # images next to every kind of launch boundary, and the last ones
    picks = np.array([0, 1, CONV_IMAGES - 1, CONV_IMAGES, CONV_IMAGES + 1, 40 * CONV_IMAGES,
                      GEMM_ROWS - 1, GEMM_ROWS, GEMM_ROWS + 1, B - 1])
    sel = torch.from_numpy(picks).cuda()
    y_small = net.measure(xd[sel].contiguous())
    xh_small = net.forward(y_small)
    net.close()
    np.testing.assert_array_equal(y[sel].cpu().numpy(), y_small.cpu().numpy())
    np.testing.assert_array_equal(xhat[sel].cpu().numpy(), xh_small.cpu().numpy())
    # and against the FP64 oracle (float32 accumulation over a handful of terms)
    yo = oracle.measure(phi, x[picks])
    np.testing.assert_allclose(y[sel].cpu().numpy(), yo, rtol=1e-5, atol=1e-6)
    ref = oracle.forward(yo, params, n1, n2, phi=phi)
    got = xhat[sel].cpu().numpy()
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-5)
