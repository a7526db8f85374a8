"""Helpers of the plane-by-plane checks (tests/test_gpu_intermediates.py): the
centre-tap selector weights that route one channel of a plane to x^, and the
pixel-wise comparison with the rounded oracle."""
import numpy as np


def selector(cout, cin, c_sel, k=11):
    """Weights [cout][cin][k][k] whose output channel 0 is input channel c_sel
    (weight 1 at the kernel centre), every other output channel zero."""
    w = np.zeros((cout, cin, k, k), np.float32)
    w[0, c_sel, k // 2, k // 2] = 1.0
    return w


def plane_violations(got, ref, S, rel_sum):
    """Pixels where got and ref are more than one bfloat16 unit (2^-7 of the larger
    magnitude) plus rel_sum * S apart, and the fraction of pixels that are equal."""
    diff = np.abs(got - ref)
    tol = 2.0 ** -7 * np.maximum(np.abs(ref), np.abs(got)) + rel_sum * S
    return diff > tol, float(np.mean(diff == 0)), diff, tol


def check_plane(got, ref, S, rel_sum, min_equal, what):
    bad, frac, diff, tol = plane_violations(got, ref, S, rel_sum)
    assert not bad.any(), "%s: %d pixels outside one unit (worst %.3g, tol %.3g)" % (
        what, int(bad.sum()), float(diff[bad].max()), float(tol[bad][np.argmax(diff[bad])]))
    assert frac >= min_equal, "%s: only %.4f of the pixels equal" % (what, frac)
