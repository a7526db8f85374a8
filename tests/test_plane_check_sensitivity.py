"""The plane-by-plane check of tests/test_gpu_intermediates.py catches the slips it
is there for.  Mistakes are planted in the oracle's computation of conv1's output
plane (one tap dropped, the kernel flipped, a one-pixel shift, the bias
dropped), on the CPU: each must fail the check that the exact plane passes."""
import numpy as np

import oracle
from oracle import rounded
from paper_1701_03891_gb300 import synth
from _planes import plane_violations

RULE_A1 = (121 * 2.0 ** -24, 0.97)     # rel_sum, min_equal used for a1


def _a1(a0, w, b):
    return rounded.bf16(oracle.relu(oracle.conv_same(a0, rounded.bf16(w), rounded.f32(b))))


def _fails(got, ref, S):
    bad, frac, _, _ = plane_violations(got, ref, S, RULE_A1[0])
    return bool(bad.any()) or frac < RULE_A1[1]


def test_plane_check_catches_planted_slips():
    n1, n2, B = 24, 20, 2
    params = synth.he_params(seed=3, bias_std=0.01)
    x = synth.voronoi_images(B, n1, n2, seed=4)
    a0 = rounded.bf16(x).reshape(B, 1, n1, n2)
    w1, b1 = params["w1"], params["b1"]
    ref = _a1(a0, w1, b1)
    S = oracle.conv_same(np.abs(a0), np.abs(rounded.bf16(w1))) + np.abs(b1)[None, :, None, None]
    assert not _fails(ref, ref, S)
    w_drop = w1.copy()
    w_drop[:, :, 3, 7] = 0.0                                   # one tap dropped
    w_flip = w1[:, :, ::-1, ::-1].copy()                       # convolution instead of correlation
    slips = {
        "tap dropped": _a1(a0, w_drop, b1),
        "kernel flipped": _a1(a0, w_flip, b1),
        "shifted one column": np.roll(ref, 1, axis=3),
        "bias dropped": _a1(a0, w1, np.zeros_like(b1)),
    }
    for name, got in slips.items():
        assert _fails(got, ref, S), name
