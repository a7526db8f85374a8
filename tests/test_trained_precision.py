"""Precision of the float32, bfloat16 and e4m3 paths on a TRAINED network,
against the FP64 oracle evaluated with the same (trained, float32) weights.

A network trained by the library's own bfloat16 training step (32 x 32,
M/N = 0.25, Voronoi images, SGD with momentum, seeded and deterministic) is
evaluated on held-out images.  Targets: rel-L2 <= 1e-5 (float32), <= 1e-2
(bfloat16), <= 3e-2 (e4m3), and a recovered-image PSNR (Sec. 5) within 0.1 dB
of the oracle's.  The reduced-precision paths are also held to the rounding
floor of their storage formats (tests/_precision.py, oracle/rounded.py), in
rel-L2 and in PSNR.  Measured on this configuration: float32 4e-7 / 2e-6 dB,
bfloat16 0.0037 / 0.03 dB, e4m3 0.028 / 0.24 dB.  e4m3 meets the rel-L2 target
here but not the 0.1 dB PSNR target, and so does the rounded oracle: rounding
both conv2 operands to 4 significant bits moves the trained network's output
by ~3 %, a sizeable fraction of its remaining error against the true image.
"""
import numpy as np
import pytest

import oracle
from oracle import rounded
from paper_1701_03891_gb300 import synth
from _precision import FLOOR_MARGIN, check_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    n, ratio, B, steps = 32, 0.25, 64, 6000
    N = n * n
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    xtrain = synth.voronoi_images(512, n, n, seed=21)
    net = deepinv.Net(phi, synth.he_params(seed=1), n, n, prec="bf16")
    saved, grads = net.new_saved(B), net.grad_buffers()
    xall = torch.from_numpy(xtrain).cuda()
    first = last = None
    for k in range(steps):
        xb = xall[(k * B) % 512:(k * B) % 512 + B].contiguous()
        yb = net.measure(xb)
        net.forward(yb, saved=saved)
        loss, dW, db, _ = net.backward(yb, xb, saved, grads=grads)
        net.sgd_momentum(dW, db, None, lr=3e-6, mu=0.9)
        if k == 0:
            first = float(loss)
    last = float(loss)
    params = {k: v.cpu().numpy() for k, v in net.get_params().items()}
    net.close()
    return deepinv, phi, params, xtrain, n, first, last


def test_training_reduces_loss(trained):
    *_, first, last = trained
    assert np.isfinite(last) and last < 0.05 * first, (first, last)


@pytest.mark.parametrize("prec", ["f32", "bf16", "fp8"])
def test_trained_network_precision(trained, prec):
    import torch
    deepinv, phi, params, xtrain, n, _, _ = trained
    xtest = synth.voronoi_images(8, n, n, seed=22)
    ref = oracle.forward(oracle.measure(phi, xtest), params, n, n, phi=phi)
    net = deepinv.Net(phi, params, n, n, prec=prec)
    if prec == "fp8":
        net.calibrate(net.measure(torch.from_numpy(xtrain[:64]).cuda()))
    xhat = net.forward(net.measure(torch.from_numpy(xtest).cuda())).cpu().numpy()
    net.close()
    rel = float(np.max(oracle.rel_l2(xhat, ref)))
    dpsnr = float(np.max(np.abs(oracle.psnr(xhat, xtest) - oracle.psnr(ref, xtest))))
    assert np.all(oracle.psnr(ref, xtest) > 14.0)         # the network does recover the images
    if prec == "f32":
        assert rel <= 1e-5 and dpsnr <= 0.1, (rel, dpsnr)
        return
    yb = rounded.measure_bf16(phi, xtest)
    if prec == "bf16":
        rnd = rounded.forward_bf16(yb, params, n, n, phi=phi)
    else:
        amax = rounded.amax_a1(rounded.measure_bf16(phi, xtrain[:64]), params, n, n, phi=phi)
        rnd = rounded.forward_e4m3(yb, params, n, n, phi=phi, amax_a1=amax)
    check_images(xhat, ref, rnd, what=("trained", prec))
    dpsnr_floor = float(np.max(np.abs(oracle.psnr(rnd, xtest) - oracle.psnr(ref, xtest))))
    assert dpsnr <= FLOOR_MARGIN * dpsnr_floor + 1e-3, (prec, dpsnr, dpsnr_floor)
    if prec == "bf16":
        assert rel <= 1e-2 and dpsnr <= 0.1, (rel, dpsnr)
    else:
        assert rel <= 3e-2, rel             # the stated rel-L2 bound holds on the trained network
        assert dpsnr_floor > 0.1            # the PSNR bound is below what e4m3 operands allow here
