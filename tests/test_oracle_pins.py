"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
values from the paper's definitions (tests/golden), closed forms, a library
routine in a special case, invariants, or central finite differences.  Each is
chosen so that a plausible slip (a dropped term, a flipped kernel, a wrong
sign, a transposed operand, a missing ReLU mask) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

from paper_1701_03891_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ y = Phi x (Sec. 1)
def test_measure_hand_values(orc):
    g = _golden("measure_tiny.json")
    y = orc.measure(np.array(g["phi"], float), np.array(g["x"], float))
    assert np.array_equal(y, np.array(g["y"], float))


def test_fc_adjoint_hand_values(orc):
    g = _golden("measure_tiny.json")
    phi = np.array(g["phi"], float)
    xt = orc.fc(phi.T, np.array(g["y"], float)[:1])
    assert np.array_equal(xt[0], np.array(g["phiT_y0"], float))


def test_measure_matches_library_matmul(orc):
    rng = np.random.default_rng(7)
    phi = rng.standard_normal((13, 37))
    x = rng.standard_normal((5, 37))
    np.testing.assert_allclose(orc.measure(phi, x), x @ phi.T, rtol=1e-12, atol=1e-12)


def test_fc_is_adjoint_of_measure(orc):
    """<Phi x, y> = <x, Phi^T y> (Sec. 4: the FC layer implements the adjoint)."""
    phi = synth.gaussian_phi(41, 97, seed=11).astype(float)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 97))
    y = rng.standard_normal((3, 41))
    lhs = np.sum(orc.measure(phi, x) * y, axis=1)
    rhs = np.sum(x * orc.fc(phi.T, y), axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


# ------------------------------------------------------------------ whole network, by hand (Sec. 4)
def test_tiny_network_forward_loss_and_gradients_by_hand(orc):
    """A two-pixel network with 1 x 1 kernels, two images (one pixel masked by
    conv1's ReLU), worked by hand: forward, loss and every gradient, FC
    included, exactly.  A missing 1/B, a missing or misplaced ReLU mask or a
    sign slip each changes one of these numbers."""
    g = _golden("tiny_net_hand.json")
    n1, n2 = g["n1"], g["n2"]
    phi, x = np.array(g["phi"], float), np.array(g["x"], float)
    params = {}
    for l in (1, 2, 3):
        params["w%d" % l] = np.full((1, 1, 1, 1), float(g["w%d" % l]))
        params["b%d" % l] = np.array([float(g["b%d" % l])])
    y = orc.measure(phi, x)
    assert np.array_equal(y, np.array(g["y"], float))
    xhat, c = orc.forward(y, params, n1, n2, phi=phi, keep=True)
    assert np.array_equal(c["xt"], np.array(g["xt"], float))
    assert np.array_equal(c["z1"].reshape(2, -1), np.array(g["z1"], float))
    assert np.array_equal(c["z2"].reshape(2, -1), np.array(g["z2"], float))
    assert np.array_equal(xhat, np.array(g["xhat"], float))
    assert orc.mse_loss(xhat, x) == g["loss"]
    loss, grads = orc.backward(y, x, params, n1, n2, phi=phi, train_fc=True)
    assert loss == g["loss"]
    assert np.shape(grads["wfc"]) == (n1 * n2, phi.shape[0])        # [N][M]
    for name, want in g["grads"].items():
        assert np.array_equal(np.asarray(grads[name], float).reshape(np.shape(want)), np.array(want, float)), name


# ------------------------------------------------------------------ Eq. (1)
def test_conv_hand_example(orc):
    g = _golden("conv_3x3_hand.json")
    a = np.array(g["input"], float)[None, None]
    w = np.array(g["kernel"], float)[None, None]
    z = orc.conv_same(a, w, np.array([g["bias"]]))
    assert np.array_equal(z[0, 0], np.array(g["z"], float))
    assert np.array_equal(orc.relu(z)[0, 0], np.array(g["relu_z"], float))


def test_conv_centred_delta_is_identity(orc):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3, 9, 7))
    k = 5
    w = np.zeros((3, 3, k, k))
    for c in range(3):
        w[c, c, k // 2, k // 2] = 1.0
    assert np.array_equal(orc.conv_same(a, w), a)


def test_conv_shifted_delta_is_zero_filled_shift(orc):
    """A delta at tap (h+1, h-2) reads in[r+1][c-2]: pins correlation (no flip) and the shift sign."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal((1, 1, 8, 10))
    k, h = 5, 2
    w = np.zeros((1, 1, k, k))
    w[0, 0, h + 1, h - 2] = 1.0
    z = orc.conv_same(a, w)[0, 0]
    ref = np.zeros((8, 10))
    ref[:-1, 2:] = a[0, 0, 1:, :-2]
    assert np.array_equal(z, ref)


def test_full_conv_then_crop_equals_same(orc):
    """Eq. (1): S(full correlation) is the 'same' correlation."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal((2, 3, 7, 6))
    w = rng.standard_normal((4, 3, 5, 5))
    b = rng.standard_normal(4)
    zf = orc.conv_full(a, w, b)
    assert zf.shape == (2, 4, 11, 10)
    np.testing.assert_allclose(orc.crop_S(zf, 5), orc.conv_same(a, w, b), rtol=1e-13, atol=1e-13)


def test_conv_matches_scipy_correlate2d(orc):
    from scipy.signal import correlate2d
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 3, 12, 9))
    w = rng.standard_normal((2, 3, 11, 11))
    b = rng.standard_normal(2)
    z = orc.conv_same(a, w, b)
    for bi in range(2):
        for co in range(2):
            ref = b[co] + sum(correlate2d(a[bi, ci], w[co, ci], mode="same", boundary="fill")
                              for ci in range(3))
            np.testing.assert_allclose(z[bi, co], ref, rtol=1e-11, atol=1e-11)


def test_conv_linearity(orc):
    rng = np.random.default_rng(5)
    a1, a2 = rng.standard_normal((2, 1, 2, 8, 8))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    al, be = 0.7, -1.3
    lhs = orc.conv_same(al * a1 + be * a2, w, b) - b[None, :, None, None]
    rhs = al * (orc.conv_same(a1, w, b) - b[None, :, None, None]) + \
        be * (orc.conv_same(a2, w, b) - b[None, :, None, None])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ the network (Sec. 4)
def _small_net(seed=0, l1=3, l2=2, l3=1, k=3, bias_std=0.1, hidden=0):
    return synth.he_params(l1, l2, l3, k, seed=seed, bias_std=bias_std, hidden=hidden)


@pytest.mark.parametrize("hidden", [0, 2])
def test_forward_all_positive_is_linear_chain(orc, hidden):
    """With every weight, bias and input >= 0 no ReLU clips, so the network is
    the composition of the linear maps (checked with scipy's correlate2d), for
    the three-layer network and one with two extra hidden layers."""
    from scipy.signal import correlate2d
    rng = np.random.default_rng(6)
    n1, n2, M = 6, 5, 7
    phi = np.abs(rng.standard_normal((M, n1 * n2)))
    y = np.abs(rng.standard_normal((2, M)))
    p = {k: np.abs(v).astype(float) for k, v in _small_net(hidden=hidden).items()}
    xhat = orc.forward(y, p, n1, n2, phi=phi)
    for b in range(2):
        a = (phi.T @ y[b]).reshape(1, n1, n2)
        for l in range(1, 4 + hidden):
            w, bb = p["w%d" % l], p["b%d" % l]
            a = np.stack([bb[co] + sum(correlate2d(a[ci], w[co, ci], mode="same") for ci in range(w.shape[1]))
                          for co in range(w.shape[0])])
        np.testing.assert_allclose(xhat[b], a.reshape(-1), rtol=1e-12)


def test_forward_negative_bias_gives_exactly_b3(orc):
    """A large negative conv2 bias zeroes a2, so x^ is exactly b3 everywhere."""
    rng = np.random.default_rng(8)
    p = _small_net()
    p["b2"] = np.full(2, -1e6)
    p["b3"] = np.array([0.25])
    phi = rng.standard_normal((5, 20))
    xhat = orc.forward(rng.standard_normal((3, 5)), p, 4, 5, phi=phi)
    assert np.all(xhat == 0.25)


def test_forward_identity_hidden_layers_reduce_to_three_layers(orc):
    """Hidden layers with centred-delta kernels (W[co][ci] = delta(co, ci) at the
    centre tap) and zero bias pass their input unchanged: the input is already
    >= 0 (a ReLU output), so the ReLU after them changes nothing, and the deeper
    network equals the three-layer one built from the same conv1/conv2/conv3."""
    rng = np.random.default_rng(15)
    n1, n2, M = 7, 6, 9
    phi = rng.standard_normal((M, n1 * n2))
    y = rng.standard_normal((3, M))
    p3 = _small_net(seed=5, bias_std=0.1)
    deep = {"w1": p3["w1"], "b1": p3["b1"], "w2": p3["w2"], "b2": p3["b2"]}
    l2, k = p3["w2"].shape[0], p3["w2"].shape[-1]
    eye = np.zeros((l2, l2, k, k))
    for c in range(l2):
        eye[c, c, k // 2, k // 2] = 1.0
    for l in (3, 4):
        deep["w%d" % l], deep["b%d" % l] = eye, np.zeros(l2)
    deep["w5"], deep["b5"] = p3["w3"], p3["b3"]
    np.testing.assert_allclose(orc.forward(y, deep, n1, n2, phi=phi), orc.forward(y, p3, n1, n2, phi=phi),
                               rtol=1e-13, atol=1e-13)


def test_forward_negative_bias_in_last_hidden_layer_gives_exactly_bL(orc):
    """A large negative bias in the last hidden layer zeroes its output, so x^ is
    exactly the last layer's bias everywhere."""
    rng = np.random.default_rng(16)
    p = _small_net(hidden=2)
    p["b4"] = np.full(2, -1e6)
    p["b5"] = np.array([-0.5])
    phi = rng.standard_normal((5, 20))
    xhat = orc.forward(rng.standard_normal((3, 5)), p, 4, 5, phi=phi)
    assert np.all(xhat == -0.5)


def test_forward_final_relu_flag(orc):
    rng = np.random.default_rng(9)
    p = _small_net()
    phi = rng.standard_normal((5, 20))
    y = rng.standard_normal((3, 5))
    a = orc.forward(y, p, 4, 5, phi=phi)
    b = orc.forward(y, p, 4, 5, phi=phi, final_relu=True)
    assert np.any(a < 0)
    assert np.array_equal(b, np.maximum(a, 0))


def test_loss_closed_forms(orc):
    rng = np.random.default_rng(10)
    x = rng.standard_normal((4, 30))
    assert orc.mse_loss(x, x) == 0.0
    # one pixel off by 3 in one of 4 signals: (1/4) * 9
    xh = x.copy()
    xh[2, 7] += 3.0
    assert abs(orc.mse_loss(xh, x) - 9.0 / 4) < 1e-12


def test_psnr_constant_error(orc):
    x = np.full((2, 16), 0.5)
    for e in (0.1, 0.01, 0.003):
        np.testing.assert_allclose(orc.psnr(x + e, x), -20 * np.log10(e), rtol=1e-12)


def test_success_threshold_inclusive(orc):
    x = np.ones((1, 10))                      # ||x||^2 = 10
    xh = x.copy()
    xh[0, 0] += 1.0                           # ||err||^2 = 1  -> ratio exactly 0.1
    assert orc.success(xh, x)[0] == 1
    xh[0, 0] += 1e-6
    assert orc.success(xh, x)[0] == 0


def test_rel_l2_closed_form(orc):
    x = np.array([[3.0, 4.0]])
    np.testing.assert_allclose(orc.rel_l2(x * 1.1, x), [0.1], rtol=1e-12)


def test_sgd_momentum_two_steps(orc):
    w, v = np.array([1.0]), np.array([0.0])
    w, v = orc.sgd_momentum(w, v, np.array([2.0]), lr=0.1, mu=0.9)   # v=2, w=0.8
    w, v = orc.sgd_momentum(w, v, np.array([1.0]), lr=0.1, mu=0.9)   # v=2.8, w=0.52
    np.testing.assert_allclose([w[0], v[0]], [0.52, 2.8], rtol=1e-12)


# ------------------------------------------------------------------ gradients (finite differences)
def _fd_check(orc, y, x, p, n1, n2, wfc, final_relu, train_fc, coords, h=1e-5, tol=1e-6):
    loss, g = orc.backward(y, x, p, n1, n2, wfc=wfc, final_relu=final_relu, train_fc=train_fc)

    def masks(pp, ww):
        _, c = orc.forward(y, pp, n1, n2, wfc=ww, final_relu=final_relu, keep=True)
        return [c["z%d" % l] > 0 for l in range(1, orc.num_layers(pp) + 1)]

    checked = 0
    for name, idx in coords:
        pp = {k: v.copy() for k, v in p.items()}
        ww = wfc.copy()
        tgt = ww if name == "wfc" else pp[name]
        base = tgt[idx]
        tgt[idx] = base + h
        mp = masks(pp, ww)
        lp = orc.mse_loss(orc.forward(y, pp, n1, n2, wfc=ww, final_relu=final_relu), x)
        tgt[idx] = base - h
        mm = masks(pp, ww)
        lm = orc.mse_loss(orc.forward(y, pp, n1, n2, wfc=ww, final_relu=final_relu), x)
        if any(np.any(a != b) for a, b in zip(mp, mm)):
            continue                         # the step crossed a ReLU kink
        fd = (lp - lm) / (2 * h)
        an = g[name][idx]
        assert abs(fd - an) <= tol * max(1.0, abs(an)), (name, idx, fd, an)
        checked += 1
    return checked


@pytest.mark.parametrize("final_relu,train_fc", [(False, False), (True, True)])
def test_gradients_every_coordinate_small_net(orc, final_relu, train_fc):
    """Central differences for every parameter of a reduced net (k=3, 3/2/1 filters, 6x5 image)."""
    rng = np.random.default_rng(12)
    n1, n2, M, B = 6, 5, 9, 2
    phi = rng.standard_normal((M, n1 * n2)) / 3
    y = rng.standard_normal((B, M))
    x = rng.uniform(0, 1, (B, n1 * n2))
    p = {k: v.astype(float) for k, v in _small_net(seed=3, bias_std=0.2).items()}
    wfc = phi.T.copy()
    coords = [(n, idx) for n in ("w1", "b1", "w2", "b2", "w3", "b3")
              for idx in np.ndindex(p[n].shape)]
    if train_fc:
        coords += [("wfc", idx) for idx in np.ndindex(wfc.shape)]
    n = _fd_check(orc, y, x, p, n1, n2, wfc, final_relu, train_fc, coords)
    assert n >= 0.9 * len(coords)


@pytest.mark.parametrize("hidden", [1, 2])
def test_gradients_every_coordinate_deeper_net(orc, hidden):
    """Central differences for every parameter of a reduced net with extra hidden
    layers (k=3, 3/2/(2)/1 filters, 6x5 image, FC trained): pins the layer loop of
    the backward pass (each layer's mask, its input activation, the order)."""
    rng = np.random.default_rng(14 + hidden)
    n1, n2, M, B = 6, 5, 9, 2
    phi = rng.standard_normal((M, n1 * n2)) / 3
    y = rng.standard_normal((B, M))
    x = rng.uniform(0, 1, (B, n1 * n2))
    p = {k: v.astype(float) for k, v in _small_net(seed=4, bias_std=0.2, hidden=hidden).items()}
    assert orc.num_layers(p) == 3 + hidden
    wfc = phi.T.copy()
    coords = [(n, idx) for n in sorted(p) for idx in np.ndindex(p[n].shape)]
    coords += [("wfc", idx) for idx in np.ndindex(wfc.shape)]
    n = _fd_check(orc, y, x, p, n1, n2, wfc, False, True, coords)
    assert n >= 0.9 * len(coords)


def test_gradients_sampled_full_shape(orc):
    """Paper shapes (64/32/1 filters of 11x11) on a 16x16 image, M = 32, batch 2, train_fc:
    central differences on sampled coordinates of every parameter tensor."""
    n1 = n2 = 16
    M, B = 32, 2
    phi = synth.gaussian_phi(M, n1 * n2, seed=0).astype(float)
    p = {k: v.astype(float) for k, v in synth.he_params(seed=1, bias_std=0.05).items()}
    x = synth.dct_sparse_images(B, n1, n2, K=10, seed=2).astype(float)
    y = phi @ x.T
    y = y.T
    rng = np.random.default_rng(13)
    coords = []
    for n in ("w1", "b1", "w2", "b2", "w3", "b3"):
        for _ in range(4):
            coords.append((n, tuple(int(rng.integers(0, s)) for s in p[n].shape)))
    coords += [("wfc", (int(rng.integers(0, 256)), int(rng.integers(0, M)))) for _ in range(4)]
    n = _fd_check(orc, y, x, p, n1, n2, phi.T.copy(), False, True, coords)
    assert n >= len(coords) - 3
