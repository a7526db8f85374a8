"""Checkpoint / resume of training state and allocation failure, through the C ABI."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1701_03891_gb300 import synth

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


def _setup(n=16, M=32, B=2, hidden=1):
    phi = synth.gaussian_phi(M, n * n, seed=40)
    params = synth.he_params(seed=41, bias_std=0.05, hidden=hidden)
    x = synth.dct_sparse_images(B, n, n, K=10, seed=42)
    y = oracle.measure(phi, x).astype(np.float32)
    return n, phi, params, x, y


def _steps(net, yd, xd, k):
    saved = net.new_saved(yd.shape[0])
    grads = net.grad_buffers()
    for _ in range(k):
        net.forward(yd, saved=saved)
        loss, dW, db, dWfc = net.backward(yd, xd, saved, grads=grads)
        net.sgd_momentum(dW, db, dWfc, lr=1e-3, mu=0.9)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_resume_from_saved_state_is_bitwise(di, prec):
    """Four SGD-momentum steps in one go equal two steps, save, load into a fresh
    network, two more steps -- weights, biases and FC weights bit for bit (the
    momentum buffers travel with the state)."""
    import torch
    n, phi, params, x, y = _setup()
    yd, xd = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    a = di.Net(phi, params, n, n, prec=prec, train_fc=True)
    _steps(a, yd, xd, 4)
    b = di.Net(phi, params, n, n, prec=prec, train_fc=True)
    _steps(b, yd, xd, 2)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "state.bin")
        b.save_state(path)
        c = di.Net(phi, params, n, n, prec=prec, train_fc=True)
        c.load_state(path)
    _steps(c, yd, xd, 2)
    pa, pc = a.get_params(), c.get_params()
    assert sorted(pa) == sorted(pc)
    for k in pa:
        assert torch.equal(pa[k], pc[k]), k


def test_load_state_rejects_other_network_and_garbage(di):
    n, phi, params, x, y = _setup()
    a = di.Net(phi, params, n, n, prec="f32", train_fc=True)
    other = di.Net(phi, params, n, n, prec="f32", train_fc=False)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "state.bin")
        a.save_state(path)
        with pytest.raises(di.DeepInvError) as e:
            other.load_state(path)
        assert e.value.status == di.EINVAL
        bad = os.path.join(tmp, "bad.bin")
        with open(bad, "wb") as f:
            f.write(b"not a state file")
        with pytest.raises(di.DeepInvError) as e:
            a.load_state(bad)
        assert e.value.status == di.EINVAL
        with pytest.raises(di.DeepInvError):
            a.load_state(os.path.join(tmp, "missing.bin"))


def test_impossible_reservation_reports_enomem_and_net_stays_usable(di):
    """A workspace for 2^20 images of 64 x 64 (about a terabyte) cannot be
    allocated: DEEPINV_ENOMEM comes back, and the network still computes."""
    import torch
    phi = synth.gaussian_phi(410, 4096, seed=0)
    params = synth.he_params(seed=1, bias_std=0.01)
    net = di.Net(phi, params, 64, 64, prec="bf16")
    with pytest.raises(di.DeepInvError) as e:
        net.reserve(1 << 20)
    assert e.value.status == di.ENOMEM
    x = synth.voronoi_images(2, 64, 64, seed=3)
    y = torch.from_numpy(oracle.measure(phi, x).astype(np.float32)).cuda()
    ref = oracle.forward(y.cpu().numpy(), params, 64, 64, phi=phi)
    assert float(np.max(oracle.rel_l2(net.forward(y).cpu().numpy(), ref))) <= 1e-2
    assert di.device_status() == 0
