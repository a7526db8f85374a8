"""conv1 + conv2 fused into one kernel (a1 kept in shared memory) against the
two-kernel path and the FP64 oracle.

The fused kernel issues the same tensor-core products in the same order per
output (conv1: kernel rows dy = 0..10; conv2: (dy, s, channel chunk)) and the
same epilogue arithmetic (add bias, ReLU, round to bfloat16), so x^ must be
bit-identical to the two-kernel path's on every image; against the oracle it
is held to the bfloat16 gates (tests/_precision.py).  Sizes cover the whole-width
walk (pitch <= 75: up to 70 columns, including the widest), column strips
(71, 130, 128 and 256 columns), tiny and ragged images, batches that split
images between CTAs, a deeper network and the benchmark workload in full.
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


def _case(n1, n2, ratio, B, seed=0, hidden=0):
    N = n1 * n2
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=seed)
    params = synth.he_params(seed=seed + 1, bias_std=0.01, hidden=hidden)
    x = synth.voronoi_images(B, n1, n2, seed=seed + 3)
    return phi, params, x


def _both(di, phi, params, x, n1, n2):
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    two = net.forward(y).cpu().numpy()
    net.set_fused(True)
    fused = net.forward(y).cpu().numpy()
    net.close()
    return y, two, fused


@pytest.mark.parametrize("n1,n2,ratio,B", [
    (64, 64, 0.10, 6),      # whole width, pitch 69
    (70, 70, 0.10, 2),      # widest whole-width walk, pitch 75
    (7, 9, 0.5, 5),         # tiny: most of every tile is padding
    (37, 20, 0.20, 3),      # ragged
    (3, 2, 0.5, 4),         # fewer positions than one a1 block
    (71, 71, 0.10, 2),      # first width walked as strips (2 x 36 columns)
    (20, 130, 0.10, 2),     # 3 strips, wide and short
    (128, 128, 0.10, 2),    # 3 strips of 43
    (256, 256, 0.10, 1),    # 5 strips of 52
])
def test_fused_bit_identical_and_oracle(di, n1, n2, ratio, B):
    phi, params, x = _case(n1, n2, ratio, B, seed=n1 + n2)
    y, two, fused = _both(di, phi, params, x, n1, n2)
    assert np.all(np.isfinite(fused))
    np.testing.assert_array_equal(fused, two)
    k = min(B, 2)
    ref = oracle.forward(oracle.measure(phi, x[:k]), params, n1, n2, phi=phi)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[:k]), params, n1, n2, phi=phi)
    check_images(fused[:k], ref, rnd, what=("fused", n1, n2))
    assert float(np.max(oracle.rel_l2(fused[:k], ref))) <= 1e-2


def test_fused_deeper_network(di):
    """Hidden layers after the fused pair read its a2 as usual."""
    n1 = n2 = 32
    phi, params, x = _case(n1, n2, 0.25, 3, seed=5, hidden=2)
    y, two, fused = _both(di, phi, params, x, n1, n2)
    np.testing.assert_array_equal(fused, two)


def test_fused_full_batch(di):
    """64 x 64, M/N = 0.1, batch 1024 (the benchmark workload): every image
    bit-identical to the two-kernel path; 4 sampled images against the oracle."""
    n1 = n2 = 64
    B = 1024
    phi, params, x = _case(n1, n2, 0.10, B, seed=11)
    y, two, fused = _both(di, phi, params, x, n1, n2)
    np.testing.assert_array_equal(fused, two)
    idx = np.array([0, 377, 800, 1023])
    ref = oracle.forward(oracle.measure(phi, x[idx]), params, n1, n2, phi=phi)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[idx]), params, n1, n2, phi=phi)
    check_images(fused[idx], ref, rnd, what="fused, batch 1024")


def test_fused_profile_stage_and_batch_sizes(di):
    """With fusion on the profiler counts the fused kernel under the conv2 stage and
    nothing under conv1; shrinking and growing the batch keeps results exact."""
    n1 = n2 = 48
    phi, params, x = _case(n1, n2, 0.10, 9, seed=2)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    full = net.forward(y).cpu().numpy()
    net.set_fused(True)
    net.profile(True)
    for b in (1, 9, 4):
        part = net.forward(y[:b].contiguous()).cpu().numpy()
        np.testing.assert_array_equal(part, full[:b])
    rec = net.profile_read()
    assert rec["conv1"][1] == 0 and rec["conv2"][1] == 3
    net.close()
