"""Deeper networks (extra 32 -> 32 hidden layers between conv2 and conv3, the
larger-capacity networks Sec. 5 leaves to future work) through the C ABI,
against the FP64 oracle on the same seeded inputs.

Tolerances:
  float32 path   <= 1e-5 forward (rel-L2 per image), 1e-4 gradients (per
                    tensor), as for three layers;
  bfloat16 path  the gates of tests/_precision.py against the rounding floor of
                 the L-layer network, computed by the rounded-operand oracle
                 (oracle/rounded.py, which rounds every stored activation and
                 weight of every layer): within 0.75 floors of the rounded
                 oracle, within 1.25 floors of the exact one, every pixel and
                 gradient element checked.  Each layer adds a rounded, ReLU-masked
                 activation, so the floor grows with depth (measured 0.043 /
                 0.067 / 0.073 / 0.097 for conv1's weight gradient at L = 3 / 4 /
                 5 / 7 on 16 x 16); the gates follow it instead of a fixed bound;
  e4m3 conv2     the same gates against the e4m3 rounded oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import rounded
from paper_1701_03891_gb300 import synth
from _precision import check_images, check_tensors

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



def _case(n1, n2, ratio, B, hidden, seed=0):
    N = n1 * n2
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=seed)
    params = synth.he_params(seed=seed + 1, bias_std=0.01, hidden=hidden)
    x = synth.dct_sparse_images(B, n1, n2, K=max(1, N // 20), seed=seed + 2)
    return phi, params, x


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("hidden", [1, 2, 4])
@pytest.mark.parametrize("n1,n2,ratio,B", [(32, 32, 0.10, 3), (24, 40, 0.20, 2), (64, 64, 0.10, 2)])
def test_forward_deeper(di, prec, hidden, n1, n2, ratio, B):
    phi, params, x = _case(n1, n2, ratio, B, hidden, seed=hidden)
    net = di.Net(phi, params, n1, n2, prec=prec)
    assert net.desc.hidden == hidden and net.L == 3 + hidden
    y = net.measure(_cuda(x))
    xhat = net.forward(y).cpu().numpy()
    _check_fwd(xhat, phi, params, x, n1, n2, prec)
    net.close()


def _check_fwd(xhat, phi, params, x, n1, n2, prec):
    ref = oracle.forward(oracle.measure(phi, x), params, n1, n2, phi=phi)
    if prec == "f32":
        assert float(np.max(oracle.rel_l2(xhat, ref))) <= 1e-5
    else:
        rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x), params, n1, n2, phi=phi)
        check_images(xhat, ref, rnd, what=(n1, n2, oracle.num_layers(params)))


def test_forward_deeper_bf16_wide(di):
    """A wide image (conv2-type kernels in row mode, several tiles per row) with
    two hidden layers."""
    phi, params, x = _case(20, 300, 0.10, 2, 2, seed=5)
    net = di.Net(phi, params, 20, 300, prec="bf16")
    y = net.measure(_cuda(x))
    _check_fwd(net.forward(y).cpu().numpy(), phi, params, x, 20, 300, "bf16")


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_identity_hidden_layers_equal_three_layers(di, prec):
    """Hidden layers whose kernels are centred deltas of exactly 1.0 with zero
    bias pass their (non-negative) input through unchanged: every product is
    exact and all but one are zero, so the deeper network returns the same bits
    as the three-layer network built from the same conv1, conv2 and conv3."""
    phi, p3, x = _case(32, 32, 0.10, 4, 0, seed=7)
    deep = {"w1": p3["w1"], "b1": p3["b1"], "w2": p3["w2"], "b2": p3["b2"]}
    eye = np.zeros((32, 32, 11, 11), np.float32)
    for c in range(32):
        eye[c, c, 5, 5] = 1.0
    for l in (3, 4):
        deep["w%d" % l], deep["b%d" % l] = eye, np.zeros(32, np.float32)
    deep["w5"], deep["b5"] = p3["w3"], p3["b3"]
    a = di.Net(phi, p3, 32, 32, prec=prec)
    b = di.Net(phi, deep, 32, 32, prec=prec)
    y = a.measure(_cuda(x))
    np.testing.assert_array_equal(a.forward(y).cpu().numpy(), b.forward(y).cpu().numpy())


def test_forward_deeper_fp8(di):
    """e4m3 conv2 with a bfloat16 hidden layer after it."""
    phi, params, x = _case(64, 64, 0.10, 4, 1, seed=9)
    net = di.Net(phi, params, 64, 64, prec="fp8")
    y = net.measure(_cuda(x))
    net.calibrate(y)
    ref = oracle.forward(oracle.measure(phi, x), params, 64, 64, phi=phi)
    yb = rounded.measure_bf16(phi, x)
    rnd = rounded.forward_e4m3(yb, params, 64, 64, phi=phi, amax_a1=rounded.amax_a1(yb, params, 64, 64, phi=phi))
    check_images(net.forward(y).cpu().numpy(), ref, rnd, what="e4m3 conv2 + hidden layer")


def _check_grads(net, g, loss_ref, res, prec, y, x, params, phi):
    loss, dW, db, dWfc = res
    n1, n2 = net.n1, net.n2
    got = {}
    for i in range(net.L):
        got["w%d" % (i + 1)], got["b%d" % (i + 1)] = dW[i].cpu().numpy(), db[i].cpu().numpy()
    if dWfc is not None:
        got["wfc"] = dWfc.cpu().numpy()
    if prec == "f32":
        assert abs(float(loss) - loss_ref) <= 1e-6 * abs(loss_ref)
        for name, v in got.items():
            err = float(np.linalg.norm(v - g[name]) / max(np.linalg.norm(g[name]), 1e-30))
            assert err <= 1e-4, (name, err)
        return
    loss_rnd, g_rnd = rounded.backward_bf16(y, x, params, n1, n2, phi=phi, train_fc=dWfc is not None)
    check_tensors(got, g, g_rnd, what=(n1, n2, net.L))
    floor = abs(loss_rnd - loss_ref) / abs(loss_ref)
    assert abs(float(loss) - loss_rnd) <= (0.75 * floor + 1e-6) * abs(loss_ref)
    assert abs(float(loss) - loss_ref) <= (1.25 * floor + 1e-6) * abs(loss_ref)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("hidden,n1,n2,M,B", [(1, 16, 16, 32, 2), (2, 16, 16, 32, 2), (1, 24, 40, 96, 2),
                                              (2, 24, 40, 96, 2), (2, 64, 64, 1024, 2)])
def test_backward_deeper(di, prec, hidden, n1, n2, M, B):
    """Loss and every gradient (FC trained) of a deeper network against the oracle."""
    N = n1 * n2
    phi = synth.gaussian_phi(M, N, seed=3)
    params = synth.he_params(seed=4, bias_std=0.05, hidden=hidden)
    x = synth.dct_sparse_images(B, n1, n2, K=max(4, N // 40), seed=5)
    y = oracle.measure(phi, x).astype(np.float32)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi, train_fc=True)
    net = di.Net(phi, params, n1, n2, prec=prec, train_fc=True)
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)
    _check_grads(net, g, loss_ref, net.backward(yd, xd, saved), prec, y, x, params, phi)
    net.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_backward_deeper_recompute(di, prec):
    """Recomputed activations (no saved buffer): one chunk is bit-identical to
    the saved path; chunks of 2 images agree up to summation order."""
    n1 = n2 = 24
    N, M, B = n1 * n2, 144, 5
    phi = synth.gaussian_phi(M, N, seed=6)
    params = synth.he_params(seed=7, bias_std=0.02, hidden=2)
    x = synth.dct_sparse_images(B, n1, n2, K=20, seed=8)
    y = oracle.measure(phi, x).astype(np.float32)
    net = di.Net(phi, params, n1, n2, prec=prec, train_fc=True)
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)

    def flat(res):
        loss, dW, db, dWfc = res
        return [loss.clone()] + [t.clone() for t in dW] + [t.clone() for t in db] + [dWfc.clone()]

    ref = flat(net.backward(yd, xd, saved))
    for a, b in zip(ref, flat(net.backward(yd, xd))):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    net.set_act_budget(2 * net.saved_bytes(1) + 4096)
    for a, b in zip(ref, flat(net.backward(yd, xd))):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(a), 1e-30)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi, train_fc=True)
    _check_grads(net, g, loss_ref, net.backward(yd, xd), prec, y, x, params, phi)


def test_sgd_and_params_deeper(di):
    """Two SGD-momentum steps update all L layers as the oracle's rule says, and
    get_params returns w1..wL in network order."""
    n1 = n2 = 16
    phi = synth.gaussian_phi(32, n1 * n2, seed=0)
    params = synth.he_params(seed=1, bias_std=0.05, hidden=2)
    x = synth.dct_sparse_images(2, n1, n2, K=10, seed=2)
    y = oracle.measure(phi, x).astype(np.float32)
    net = di.Net(phi, params, n1, n2, prec="f32")
    got0 = net.get_params()
    assert sorted(got0) == sorted(params)
    for k in params:
        np.testing.assert_array_equal(got0[k].cpu().numpy(), params[k])
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(2)
    p = {k: v.astype(np.float64) for k, v in params.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    for step in range(2):
        net.forward(yd, saved=saved)
        loss, dW, db, _ = net.backward(yd, xd, saved)
        net.sgd_momentum(dW, db, lr=1e-2, mu=0.9)
        for i in range(net.L):
            for name, gg in (("w%d" % (i + 1), dW[i]), ("b%d" % (i + 1), db[i])):
                p[name], v[name] = oracle.sgd_momentum(p[name], v[name], gg.cpu().numpy(), 1e-2, 0.9)
    got = net.get_params()
    for k in p:
        np.testing.assert_allclose(got[k].cpu().numpy(), p[k], rtol=1e-5, atol=1e-7)


def test_autograd_deeper(di):
    import torch
    n1 = n2 = 16
    phi = synth.gaussian_phi(32, n1 * n2, seed=0)
    params = synth.he_params(seed=1, bias_std=0.05, hidden=1)
    x = synth.dct_sparse_images(2, n1, n2, K=10, seed=2)
    y = oracle.measure(phi, x).astype(np.float32)
    net = di.Net(phi, params, n1, n2, prec="f32")
    names = [n for i in range(1, 5) for n in ("w%d" % i, "b%d" % i)]
    ps = [torch.tensor(params[k], requires_grad=True, device="cuda") for k in names]
    loss = di.mse_loss(net, _cuda(y), _cuda(x), ps)
    loss.backward()
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi)
    assert abs(float(loss.detach()) - loss_ref) <= 1e-5 * loss_ref
    for name, t in zip(names, ps):
        err = np.linalg.norm(t.grad.cpu().numpy() - g[name]) / max(np.linalg.norm(g[name]), 1e-30)
        assert err <= 1e-4, (name, err)


def test_device_status_clean_after_deeper(di):
    assert di.device_status(reset=True) == 0
