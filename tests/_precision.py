"""Tolerances of the reduced-precision paths, derived from the rounding floor.

oracle/rounded.py evaluates the network (and its MSE gradient, Sec. 4) with
every operand rounded where the bfloat16 or e4m3 path stores it and every sum
exact.  Its distance to the exact FP64 oracle is the floor: the error the
storage format forces on any kernel.  What a kernel adds on top comes from its
float32 sums (their order), and from a stored value that rounds to the other
neighbour when its float32 sum lands on the other side of a rounding tie.
The requirement is that a kernel add at most a quarter to the format's own
error.  The two are independent and add in quadrature, so:

  kernel vs rounded oracle   <= KERNEL_SHARE * floor,   KERNEL_SHARE = 0.75
  kernel vs exact oracle     <= FLOOR_MARGIN * floor,   FLOOR_MARGIN = sqrt(1 + 0.75^2) = 1.25

and, element by element (every pixel of every image, every entry of every
gradient tensor), the kernel's worst deviation from the rounded oracle may be
at most ELEMENT_FACTOR = 2 times the format's worst deviation (rounded vs
exact oracle) on the same image or tensor: a pixel or a tile edge that is
wrong by more than any rounding could make it fails.

The stated bounds (bfloat16 rel-L2 <= 1e-2) are checked beside these; where
the floor itself exceeds a stated bound (e4m3: 3e-2), the floor is what the
format allows and the tests say so.
"""
import numpy as np

import oracle

KERNEL_SHARE = 0.75
FLOOR_MARGIN = 1.25
ELEMENT_FACTOR = 2.0


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_images(got, exact, rounded, what=""):
    """Per image (max over the batch): the floor, the kernel against the rounded
    and the exact oracle, and every pixel against the rounded oracle.
    Returns (floor, kernel vs exact) for reporting."""
    got = np.asarray(got, np.float64)
    B = got.shape[0]
    floor = float(np.max(oracle.rel_l2(rounded, exact)))
    vs_rounded = float(np.max(oracle.rel_l2(got, rounded)))
    vs_exact = float(np.max(oracle.rel_l2(got, exact)))
    assert np.all(np.isfinite(got)), what
    assert vs_rounded <= KERNEL_SHARE * floor, (what, "vs rounded oracle", vs_rounded, floor)
    assert vs_exact <= FLOOR_MARGIN * floor, (what, "vs exact oracle", vs_exact, floor)
    r = np.asarray(rounded, np.float64).reshape(B, -1)
    e = np.asarray(exact, np.float64).reshape(B, -1)
    worst_kernel = np.max(np.abs(got.reshape(B, -1) - r), axis=1)
    worst_format = np.max(np.abs(r - e), axis=1)
    bad = worst_kernel > ELEMENT_FACTOR * worst_format
    assert not np.any(bad), (what, "worst pixel", worst_kernel[bad], worst_format[bad])
    return floor, vs_exact


def check_tensors(got: dict, exact: dict, rounded: dict, what=""):
    """The same per gradient tensor (rel-L2 over the tensor; element-wise against
    the tensor's rms).  Returns {name: (floor, kernel vs exact)}."""
    out = {}
    for name, g in got.items():
        g = np.asarray(g, np.float64).ravel()
        e, r = np.asarray(exact[name], np.float64).ravel(), np.asarray(rounded[name], np.float64).ravel()
        floor = _rel(r, e)
        vs_rounded, vs_exact = _rel(g, r), _rel(g, e)
        assert np.all(np.isfinite(g)), (what, name)
        assert vs_rounded <= KERNEL_SHARE * floor, (what, name, "vs rounded oracle", vs_rounded, floor)
        assert vs_exact <= FLOOR_MARGIN * floor, (what, name, "vs exact oracle", vs_exact, floor)
        worst_kernel, worst_format = float(np.max(np.abs(g - r))), float(np.max(np.abs(r - e)))
        assert worst_kernel <= ELEMENT_FACTOR * worst_format, (what, name, "worst element", worst_kernel,
                                                               worst_format)
        out[name] = (floor, vs_exact)
    return out
