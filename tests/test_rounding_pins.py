"""Pins of oracle/rounded.py, the oracle's arithmetic on operands rounded the way a
bfloat16 or e4m3 path stores them (CPU only).

The rounding functions are pinned to the formats' definitions (hand values at
ties, at the largest finite e4m3 value, in the subnormal range) and to torch's
own conversions; the rounded network is pinned to hand-worked cases where one
rounding point changes the result (so a dropped or misplaced rounding fails),
and, where nothing needs rounding, to the exact oracle and the hand-worked
network of tests/golden/tiny_net_hand.json.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import rounded as R

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ formats
def test_bf16_ties_to_even_and_exact_values():
    # bfloat16 has 8 significant bits: spacing 2^-7 in [1, 2), 2 in [256, 512)
    assert R.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0000000)
    assert R.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie -> even (1.0000010)
    assert R.bf16(263.5) == 264.0 and R.bf16(257.0) == 256.0 and R.bf16(297.0) == 296.0
    assert R.bf16(-263.5) == -264.0
    for v in (0.0, 1.0, 15.5, 17.0, 1.125, 255.0, 256.0, 2.0 ** -130, -3.75):
        assert R.bf16(v) == v


def test_bf16_matches_torch_conversion():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        rng.standard_normal(1000) * 1e-39]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(R.bf16(x), ref)


def test_e4m3_definition_values():
    # normal binade [1, 2): spacing 1/8; [128, 256): 16; [256, 448]: 32
    assert R.e4m3(1.0 + 1 / 16) == 1.0                       # tie -> even (mantissa 000)
    assert R.e4m3(1.0 + 3 / 16) == 1.25                      # tie -> even (mantissa 010)
    assert R.e4m3(149.3333) == 144.0 and R.e4m3(152.0) == 160.0   # 152 = 144 + 8: tie -> 160 (mantissa 010)
    assert R.e4m3(448.0) == 448.0 and R.e4m3(460.0) == 448.0
    assert R.e4m3(1e6) == 448.0 and R.e4m3(-1e6) == -448.0     # saturation
    # subnormals m 2^-9, m = 1..7; the smallest normal is 2^-6
    assert R.e4m3(2.0 ** -9) == 2.0 ** -9 and R.e4m3(7 * 2.0 ** -9) == 7 * 2.0 ** -9
    assert R.e4m3(2.0 ** -10) == 0.0                         # tie between 0 and 2^-9 -> 0
    assert R.e4m3(3 * 2.0 ** -10) == 2.0 ** -8               # tie between 2^-9 and 2^-8 -> 2^-8
    assert R.e4m3(2.0 ** -6) == 2.0 ** -6
    # every one of the 126 positive finite values is a fixed point
    vals = [m * 2.0 ** -9 for m in range(1, 8)] + [(1 + f / 8) * 2.0 ** e for e in range(-6, 9)
                                                  for f in range(8) if (1 + f / 8) * 2.0 ** e <= 448]
    assert len(vals) == 126
    np.testing.assert_array_equal(R.e4m3(np.array(vals)), np.array(vals))


def test_e4m3_matches_torch_conversion_in_range():
    import torch
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(1)
    x = (rng.uniform(-1, 1, 50000) * 2.0 ** rng.uniform(-12, 8.8, 50000)).astype(np.float32)
    x = x[np.abs(x) <= 448]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(R.e4m3(x), ref)


# ------------------------------------------------------------------ rounded network
def _net1(w1=1.0, w2=1.0, w3=1.0, b=(0.0, 0.0, 0.0)):
    """One pixel, one filter per layer, 1 x 1 kernels: every layer a scale plus bias."""
    p = {}
    for l, w in ((1, w1), (2, w2), (3, w3)):
        p["w%d" % l] = np.full((1, 1, 1, 1), float(w))
        p["b%d" % l] = np.array([b[l - 1]])
    return p


@pytest.mark.parametrize("where,phi,y,w,expect,exact", [
    ("y", 1.0, 257.0, (1.0, 1.0, 1.0), 256.0, 257.0),                # y stored as bfloat16
    ("proxy x~", 17.0, 15.5, (1.0, 1.0, 1.0), 264.0, 263.5),        # x~ = 263.5 stored as bfloat16
    ("a1", 1.0, 15.5, (17.0, 1.0, 1.0), 264.0, 263.5),              # conv1 output
    ("a2", 1.0, 1.0, (15.5, 17.0, 1.0), 264.0, 263.5),              # conv2 output
    ("w3", 1.0, 1.0, (1.0, 1.0, 257.0), 256.0, 257.0),              # conv3 weight
])
def test_forward_bf16_each_rounding_point(where, phi, y, w, expect, exact):
    params = _net1(*w)
    args = (np.array([[y]]), params, 1, 1)
    assert oracle.forward(*args, phi=np.array([[phi]]))[0, 0] == exact, where
    assert R.forward_bf16(*args, phi=np.array([[phi]]))[0, 0] == expect, where


def test_rounded_network_equals_hand_network_when_nothing_rounds():
    """Every value of the hand-worked network (small integers) is exact in
    bfloat16, so the rounded forward, loss and gradients equal it exactly."""
    with open(os.path.join(HERE, "golden", "tiny_net_hand.json")) as f:
        g = json.load(f)
    phi, x = np.array(g["phi"], float), np.array(g["x"], float)
    params = {}
    for l in (1, 2, 3):
        params["w%d" % l] = np.full((1, 1, 1, 1), float(g["w%d" % l]))
        params["b%d" % l] = np.array([float(g["b%d" % l])])
    y = R.measure_bf16(phi, x)
    assert np.array_equal(y, np.array(g["y"], float))
    xhat = R.forward_bf16(y, params, g["n1"], g["n2"], phi=phi)
    assert np.array_equal(xhat, np.array(g["xhat"], float))
    loss, grads = R.backward_bf16(y, x, params, g["n1"], g["n2"], phi=phi, train_fc=True)
    assert loss == g["loss"]
    for name, want in g["grads"].items():
        assert np.array_equal(np.asarray(grads[name], float).reshape(np.shape(want)), np.array(want, float)), name


def test_backward_bf16_rounds_the_output_and_input_gradients():
    """One pixel, B = 1: x^ = 1, x = -130.75, so dL/dx^ = 2 (x^ - x) = 263.5,
    stored as 264; conv3's input gradient w3 * 264 = 297 with w3 = 1.125 is
    stored as 296 (a tie, to even); conv2's input gradient 296 passes through."""
    params = _net1(1.0, 1.0, 1.125, b=(0.0, 0.0, 1.0 - 1.125))      # x^ = 1.125 * 1 - 0.125 = 1
    y, x = np.array([[1.0]]), np.array([[-130.75]])
    loss, g = R.backward_bf16(y, x, params, 1, 1, phi=np.array([[1.0]]))
    assert loss == 131.75 ** 2
    assert g["w3"][0, 0, 0, 0] == 264.0 and g["b3"][0] == 264.0      # 264 * a2 (a2 = 1)
    assert g["w2"][0, 0, 0, 0] == 296.0 and g["b2"][0] == 296.0      # 296 * a1 (a1 = 1)
    assert g["w1"][0, 0, 0, 0] == 296.0 and g["b1"][0] == 296.0      # 296 * x~ (x~ = 1)
    _, ge = oracle.backward(y, x, params, 1, 1, phi=np.array([[1.0]]))
    assert ge["w3"][0, 0, 0, 0] == 263.5 and ge["w2"][0, 0, 0, 0] == 263.5 * 1.125


@pytest.mark.parametrize("per_channel", [False, True])
def test_forward_e4m3_hand_network(per_channel):
    """Two conv1 filters (w1 = 1 and 3), y = 5: a1 = (5, 15).  One scale for the
    layer: sa = 15 / 448, a1 / sa = (149.33, 448) -> e4m3 (144, 448); w2 = (1, 1)
    -> 448 / sw each; the sum times sw sa is (144 + 448) sa = 19.821, stored as
    bfloat16 19.875 (spacing 1/8); conv3 passes it through.  One scale per channel:
    a1 / sa = (448, 448) exactly, the weights w2 sa = (5, 15) / 448 -> e4m3
    (144, 448) sw: the same 592 sa and the same 19.875.  Exact: 20."""
    params = {"w1": np.array([1.0, 3.0]).reshape(2, 1, 1, 1), "b1": np.zeros(2),
              "w2": np.ones((1, 2, 1, 1)), "b2": np.zeros(1),
              "w3": np.ones((1, 1, 1, 1)), "b3": np.zeros(1)}
    y, phi = np.array([[5.0]]), np.array([[1.0]])
    amax = R.amax_a1(y, params, 1, 1, phi=phi, per_channel=per_channel)
    assert np.array_equal(np.atleast_1d(amax), [5.0, 15.0] if per_channel else [15.0])
    assert oracle.forward(y, params, 1, 1, phi=phi)[0, 0] == 20.0
    assert R.forward_e4m3(y, params, 1, 1, phi=phi, amax_a1=amax, per_channel=per_channel)[0, 0] == 19.875


# ------------------------------------------------------------------ floors on the seeded workloads
@pytest.mark.parametrize("n,ratio,B,images", [(32, 0.10, 4, "dct"), (64, 0.10, 2, "voronoi")])
def test_rounding_floors_of_the_seeded_networks(n, ratio, B, images):
    """What the storage formats alone cost on the seeded He-initialised networks
    (sums exact): bfloat16 stays well inside the stated 1e-2; e4m3 on conv2's
    operands costs more than the stated 3e-2, whether a1 is scaled once per
    layer or once per input channel (the per-channel factors folded into the
    per-filter weight scales move the rounding from a1 to the weights; they do
    not lower it).  The kernels' tests gate at these floors."""
    from paper_1701_03891_gb300 import synth
    N = n * n
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1, bias_std=0.01)
    x = (synth.voronoi_images(B, n, n, seed=3) if images == "voronoi"
         else synth.dct_sparse_images(B, n, n, K=max(1, N // 20), seed=2))
    ref = oracle.forward(oracle.measure(phi, x), params, n, n, phi=phi)
    yb = R.measure_bf16(phi, x)
    bf = float(np.max(oracle.rel_l2(R.forward_bf16(yb, params, n, n, phi=phi), ref)))
    assert 1e-3 < bf < 1e-2
    floors = []
    for per_channel in (False, True):
        amax = R.amax_a1(yb, params, n, n, phi=phi, per_channel=per_channel)
        f8 = R.forward_e4m3(yb, params, n, n, phi=phi, amax_a1=amax, per_channel=per_channel)
        floors.append(float(np.max(oracle.rel_l2(f8, ref))))
    assert min(floors) > 3e-2, floors
    assert floors[1] > 0.95 * floors[0], floors
