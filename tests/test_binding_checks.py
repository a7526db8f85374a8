"""The Python binding rejects tensors of the wrong kind or size before calling
the library (which cannot see a buffer's extent), on the CPU: a short gradient,
host or output buffer would otherwise be read or written past its end."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1701_03891_gb300 import deepinv, synth


def _fake_net(L=3, n1=4, n2=4, M=5, train_fc=False):
    """A Net object with shapes but no library handle: every call below must
    fail in the binding's checks, before the library is reached."""
    net = object.__new__(deepinv.Net)
    net._h = ctypes.c_void_p()
    net.L, net.n1, net.n2, net.N, net.M = L, n1, n2, n1 * n2, M
    shapes = [(64, 1, 11, 11), (32, 64, 11, 11)] + [(32, 32, 11, 11)] * (L - 3) + [(1, 32, 11, 11)]
    net.shapes = shapes
    net.desc = deepinv.NetDesc(n1, n2, M, 64, 32, 1, 11, 0, int(train_fc), deepinv.BF16, L - 3)
    net.device = torch.device("cpu")
    return net


def _raises(fn, *words):
    with pytest.raises(deepinv.DeepInvError) as e:
        fn()
    assert e.value.status == deepinv.EINVAL
    for w in words:
        assert w in str(e.value), str(e.value)


def test_batch_rows():
    assert deepinv._batch(torch.zeros(3, 16), "x", 16) == 3
    assert deepinv._batch(torch.zeros(3, 4, 4), "x", 16) == 3      # images [B][n1][n2]
    _raises(lambda: deepinv._batch(torch.zeros(3, 15), "x", 16), "x", "rows of 16")
    _raises(lambda: deepinv._batch(torch.zeros(48), "x", 16), "x")


def test_host_entry_points_check_buffers():
    net = _fake_net()
    good_x = torch.zeros(2, net.N)
    _raises(lambda: net.sense_recover_host(torch.zeros(2, net.N, dtype=torch.float64)), "x_host", "float32")
    _raises(lambda: net.sense_recover_host(torch.zeros(net.N, 2).t()), "x_host", "contiguous")
    _raises(lambda: net.sense_recover_host(good_x, torch.zeros(1, net.N)), "out_host", "expected %d" % (2 * net.N))
    _raises(lambda: net.sense_recover_host_submit(good_x, torch.zeros(2, net.N - 1)), "out_host")
    _raises(lambda: net.forward_host(torch.zeros(2, net.M + 1)), "y_host", "rows of %d" % net.M)
    _raises(lambda: net.forward_host(torch.zeros(2, net.M), torch.zeros(2 * net.N + 1)), "out_host")


def test_gradient_lists_checked_before_the_update():
    net = _fake_net(L=4)
    dW = [torch.zeros(s) for s in net.shapes]
    db = [torch.zeros(s[0]) for s in net.shapes]
    _raises(lambda: net.sgd_momentum(dW[:3], db[:3]), "need 4 weight and bias gradients")
    _raises(lambda: net.sgd_momentum(dW, db), "dW[0]", "CUDA")      # CPU tensors are not device memory


def test_net_create_checks_layer_shapes():
    n1 = n2 = 8
    phi = synth.gaussian_phi(6, n1 * n2, seed=0)
    p = synth.he_params(seed=1)
    bad = dict(p, w2=np.zeros((32, 63, 11, 11), np.float32))
    _raises(lambda: deepinv.Net(phi, bad, n1, n2, device="cpu"), "layer 2")
    bad = dict(p, b3=np.zeros(2, np.float32))
    _raises(lambda: deepinv.Net(phi, bad, n1, n2, device="cpu"), "layer 3")
    deep = synth.he_params(seed=1, hidden=2)
    deep["w4"] = np.zeros((16, 32, 11, 11), np.float32)
    deep["b4"] = np.zeros(16, np.float32)
    _raises(lambda: deepinv.Net(phi, deep, n1, n2, device="cpu"), "hidden layer 4 has 16 filters")
    _raises(lambda: deepinv.Net(phi[:, :-1], p, n1, n2, device="cpu"), "phi must be M x (n1*n2)")


@pytest.fixture(scope="module")
def built():
    from paper_1701_03891_gb300 import build
    build.build()


def test_server_checks_request_arrays(built):
    srv = deepinv.Server(hbm_budget_bytes=1 << 20, max_streams=1, max_batch=4)
    try:
        srv.nets.append(_fake_net())   # shapes only: nothing is submitted
        N, M = srv.nets[0].N, srv.nets[0].M
        y, xh = np.zeros(M, np.float32), np.zeros(N, np.float32)
        _raises(lambda: srv.serve([(0, np.zeros(M - 1, np.float32), xh, 0)]), "request 0: y")
        _raises(lambda: srv.serve([(0, y, np.zeros(N, np.float64), 0)]), "request 0: xhat")
        _raises(lambda: srv.serve([(0, y, xh, 0), (0, y, np.zeros((N, 2), np.float32)[:, 0], 1)]),
                "request 1: xhat")
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()
