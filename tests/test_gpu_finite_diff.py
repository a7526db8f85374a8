"""The float32 GPU backward against central finite differences of the GPU
forward's own loss, on the 16 x 16, M = 32, batch-2 instance (FC trained).

L(Omega) = (1/B) sum_b ||x^_b - x_b||^2 (Sec. 4) is summed in float64 on the
host from the GPU forward's float32 x^; a coordinate w of every parameter
tensor is moved by +-h and (L(w + h) - L(w - h)) / 2h compared with the
analytic gradient.  The quotient's error is float32 rounding noise (growing
as 1/h) plus ReLU kinks crossed by the step (growing with h); measured worst
discrepancies relative to the tensor's largest gradient at h = 1e-1 / 1e-2 /
1e-3: conv1 2.4e-2 / 9.2e-3 / 3.0e-3, conv2 1.3e-2 / 2.3e-3 / 1.3e-3, conv3
~1e-7 (linear there), FC 5.6e-3 / 2.6e-3 / 1.5e-3.  So h = 1e-3 and a
tolerance of 1e-2 of that scale.  The bf16
backward is checked against the FP64 oracle, itself pinned by finite
differences in test_oracle_pins.py.
"""
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
    return deepinv


@pytest.mark.parametrize("hidden", [0, 1])
def test_f32_backward_matches_finite_differences(di, hidden):
    """hidden = 1 adds a 32 -> 32 layer between conv2 and conv3 (four conv layers)."""
    import torch
    n1 = n2 = 16
    N, M, B = n1 * n2, 32, 2
    phi = synth.gaussian_phi(M, N, seed=30)
    params = synth.he_params(seed=31, bias_std=0.05, hidden=hidden)
    x = synth.dct_sparse_images(B, n1, n2, K=12, seed=32)
    y = oracle.measure(phi, x).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    xd = torch.from_numpy(x.astype(np.float32)).cuda()

    def loss_of(p, wfc):
        net = di.Net(phi, p, n1, n2, prec="f32", train_fc=True)
        if wfc is not None:
            # the FC copy starts as Phi^T; move it by one SGD step with lr = -1 on a one-hot gradient
            dW, db, dWfc = net.grad_buffers()
            for t in dW + db:
                t.zero_()
            dWfc.copy_(torch.from_numpy(wfc).cuda())
            net.sgd_momentum(dW, db, dWfc, lr=-1.0, mu=0.0)
        xh = net.forward(yd).cpu().numpy().astype(np.float64)
        net.close()
        return float(np.sum((xh - x.astype(np.float64)) ** 2) / B)

    net = di.Net(phi, params, n1, n2, prec="f32", train_fc=True)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)
    _, dW, db, dWfc = net.backward(yd, xd, saved)
    grads = {"w%d" % (i + 1): dW[i] for i in range(net.L)}
    grads.update({"b%d" % (i + 1): db[i] for i in range(net.L)})
    grads["wfc"] = dWfc
    grads = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    net.close()

    rng = np.random.default_rng(33)
    h = 1e-3
    checked = 0
    for name, g in grads.items():
        flat = g.reshape(-1)
        scale = float(np.max(np.abs(flat)))
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            vals = []
            for sgn in (1.0, -1.0):
                if name == "wfc":
                    e = np.zeros(N * M, np.float32)
                    e[i] = sgn * h
                    vals.append(loss_of(params, e.reshape(N, M)))
                else:
                    p = {k: v.copy() for k, v in params.items()}
                    p[name].reshape(-1)[i] += sgn * h
                    vals.append(loss_of(p, None))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - flat[i]) <= 1e-2 * max(scale, abs(flat[i])), (name, int(i), fd, flat[i])
            checked += 1
    assert checked == sum(min(6, g.size) for g in grads.values())
