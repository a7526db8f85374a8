"""The oracle's arithmetic on operands rounded as a reduced-precision path stores them.

TEST INFRASTRUCTURE ONLY, under the same rules as ``oracle.py``: only ``tests/``
may use it; it shares no code with the CUDA path and imports nothing from it.

Why it exists.  The float64 oracle sees the float32 master weights and inputs.
A path that stores its operands in bfloat16 or e4m3 cannot match it closer than
the rounding of those operands allows, whatever its kernels do.  This module
computes that floor: the network of Sec. 4 (and its MSE gradient) with every
operand rounded where a reduced-precision path rounds it, all sums in float64.
Against it, a kernel's own error (sum order, a slip at a tile edge) can be
told apart from the format's; against the exact oracle, the rounding floor
follows, and the tests gate each path at that floor plus a margin.

Rounding points (the path's storage formats; sums are exact here):
  * measurement y = Phi x (Sec. 1): Phi and x as bfloat16, y as float32.
  * FC: y and Phi^T as bfloat16; the proxy x~ stored as bfloat16 (Sec. 4).
  * conv layers (Eq. 1): weights as bfloat16; every ReLU output stored as
    bfloat16; the last layer's output is the float32 image.
  * e4m3 variant: the second layer's input a1 as e4m3 after scaling by a
    calibrated factor, its weights as e4m3 with one scale per filter, the
    layer's sum multiplied back by both scales before bias and ReLU.
  * backward (Sec. 4, backpropagation of the MSE loss): dL/dx^ = (2/B)(x^ - x)
    in float32, then stored as bfloat16; each layer's input gradient stored as
    bfloat16 after its ReLU mask; weight and bias gradients summed from those
    bfloat16 planes and the stored activations; with a trained FC layer, dx~
    and y as bfloat16 for dWfc.

Formats, from their definitions:
  * bfloat16: 1 sign, 8 exponent and 7 fraction bits, the upper half of an
    IEEE-754 binary32; a binary32 is rounded to it to nearest, ties to even.
  * e4m3 (the OCP 8-bit format E4M3): 1 sign, 4 exponent bits with bias 7,
    3 fraction bits; normal numbers from 2^-6 to 448 (= 1.75 * 2^8, the
    all-ones pattern is NaN, there is no infinity), subnormals m * 2^-9 for
    m = 1..7; rounded to nearest, ties to even, magnitudes past 448
    saturated to 448.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o

E4M3_MAX = 448.0


# ---------------------------------------------------------------- formats
def f32(a) -> np.ndarray:
    """Round to IEEE binary32 (nearest, ties to even), returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def bf16(a) -> np.ndarray:
    """Round to bfloat16 (via binary32, as a path holding float32 values does),
    nearest with ties to even; returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32)).view(np.uint32)
    u = u.astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def e4m3(a) -> np.ndarray:
    """Round to e4m3 (via binary32), nearest with ties to even, saturating at
    +-448; returned as float64."""
    x = f32(a)
    m = np.abs(x)
    _, e = np.frexp(m)                              # m = f 2^e, f in [0.5, 1): binade 2^(e - 1)
    E = np.maximum(e - 1, -6)                       # below 2^-6 the subnormal spacing 2^-9 holds
    q = np.ldexp(1.0, E - 3)                        # 3 fraction bits: spacing 2^(E - 3)
    r = np.minimum(np.round(m / q) * q, E4M3_MAX)   # np.round: half to even
    return np.copysign(r, x)


# ---------------------------------------------------------------- forward
def measure_bf16(phi, x) -> np.ndarray:
    """y = Phi x (Sec. 1) with Phi and x in bfloat16, stored as float32."""
    return f32(_o.measure(bf16(phi), bf16(x)))


def _fc_bf16(y, phi):
    """x~ = Phi^T y with both operands in bfloat16, stored as bfloat16 (Sec. 4)."""
    return bf16(_o.fc(bf16(np.asarray(phi, np.float64).T), bf16(y)))


def forward_bf16(y, params: dict, n1: int, n2: int, *, phi, final_relu: bool = False, keep: bool = False):
    """x^ = M(y, Omega) (Sec. 4, Eq. 1) with the bfloat16 path's rounding points.
    Returns x^ [B][N] (float32 values); with ``keep`` also the stored planes
    a0 (= x~), a1, ..., a_{L-1} (bfloat16 values) and the pre-activations z_l."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    L = _o.num_layers(params)
    a = _fc_bf16(y, phi).reshape(B, 1, n1, n2)
    c = {"a0": a}
    for l in range(1, L + 1):
        z = _o.conv_same(a, bf16(params["w%d" % l]), f32(params["b%d" % l]))
        if l < L:
            a = bf16(_o.relu(z))
        else:
            a = f32(_o.relu(z) if final_relu else z)
        c["z%d" % l] = z
        c["a%d" % l] = a
    xhat = a.reshape(B, n1 * n2)
    return (xhat, c) if keep else xhat


def e4m3_scales(params: dict, amax_a1, per_channel: bool = False):
    """Scales of the e4m3 layer (the second conv layer).

    Activations: sa = amax(a1) / 448 over a calibration batch, one factor for
    the layer (``per_channel`` = False) or one per input channel ci.  With
    per-channel factors, sa[ci] is folded into the weights first,
    W'[co][ci] = W[co][ci] sa[ci], so that the layer's sum needs no factor per
    channel.  Weights: sw[co] = max |W'[co]| / 448, one per filter.
    Returns (inv_sa, w_scaled, sw, oscale), with the kernel's float32 arithmetic:
    a1 is stored as e4m3(a1 inv_sa), W as e4m3(W' / sw), and the sum is
    multiplied by oscale = sw (times sa when there is one factor)."""
    w2 = np.asarray(params["w2"], np.float64)
    amax = f32(np.maximum(np.asarray(amax_a1, np.float64), 0.0))
    sa = f32(np.where(amax > 0, amax / E4M3_MAX, 1.0))
    inv_sa = f32(1.0 / sa)
    if per_channel:
        wsc = f32(w2 * sa[None, :, None, None])
    else:
        wsc = f32(w2)
    amax_w = np.abs(wsc).reshape(w2.shape[0], -1).max(axis=1)
    sw = f32(np.where(amax_w > 0, amax_w / E4M3_MAX, 1.0))
    oscale = sw if per_channel else f32(sw * sa)
    return inv_sa, wsc, sw, oscale


def forward_e4m3(y, params: dict, n1: int, n2: int, *, phi, amax_a1, per_channel: bool = False,
                 final_relu: bool = False):
    """x^ with the second conv layer on e4m3 operands (the rest as ``forward_bf16``).
    ``amax_a1``: the calibrated maximum of a1, a scalar or one value per channel."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    L = _o.num_layers(params)
    inv_sa, wsc, sw, oscale = e4m3_scales(params, amax_a1, per_channel)
    a = _fc_bf16(y, phi).reshape(B, 1, n1, n2)
    a1 = f32(_o.relu(_o.conv_same(a, bf16(params["w1"]), f32(params["b1"]))))
    isa = inv_sa[None, :, None, None] if per_channel else inv_sa
    a1q = e4m3(f32(a1 * isa))
    w2q = e4m3(f32(wsc / sw[:, None, None, None]))
    t = f32(_o.conv_same(a1q, w2q))
    z2 = t * oscale[None, :, None, None] + f32(params["b2"])[None, :, None, None]
    a = bf16(_o.relu(z2))
    for l in range(3, L + 1):
        z = _o.conv_same(a, bf16(params["w%d" % l]), f32(params["b%d" % l]))
        a = bf16(_o.relu(z)) if l < L else f32(_o.relu(z) if final_relu else z)
    return a.reshape(B, n1 * n2)


def amax_a1(y, params: dict, n1: int, n2: int, *, phi, per_channel: bool = False):
    """Calibration: the largest first-layer activation of a batch (bfloat16 proxy,
    bfloat16 weights, float32 ReLU output), over the batch or per channel."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    a = _fc_bf16(y, phi).reshape(B, 1, n1, n2)
    a1 = f32(_o.relu(_o.conv_same(a, bf16(params["w1"]), f32(params["b1"]))))
    return a1.max(axis=(0, 2, 3)) if per_channel else np.float64(a1.max())


def forward_abs(y, params: dict, n1: int, n2: int, *, phi, final_relu: bool = False):
    """Per pixel, the sum of the magnitudes of every term on the path to x^:
    S_0 = |Phi^T| |y|, S_l = conv(S_{l-1}, |W_l|) + |b_l| (Eq. 1 with every
    operand replaced by its magnitude).  |x^| <= S_L, and a sum's float32
    rounding error is bounded by a multiple of the unit roundoff times S, so S
    scales element-wise tolerances.  Returns S_L [B][N]."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    L = _o.num_layers(params)
    a = _o.fc(np.abs(np.asarray(phi, np.float64)).T, np.abs(y)).reshape(B, 1, n1, n2)
    for l in range(1, L + 1):
        a = _o.conv_same(a, np.abs(params["w%d" % l]), np.abs(params["b%d" % l]))
    return a.reshape(B, n1 * n2)


# ---------------------------------------------------------------- backward
def backward_bf16(y, x, params: dict, n1: int, n2: int, *, phi, train_fc: bool = False,
                  final_relu: bool = False):
    """Gradient of (1/B) sum_b ||x^_b - x_b||^2 (Sec. 4) with the bfloat16 path's
    rounding points: the forward of ``forward_bf16``, the output gradient and
    every input gradient stored as bfloat16, the weights of the input gradients
    in bfloat16.  Returns (loss, grads) like ``oracle.backward``."""
    y, x = np.asarray(y, np.float64), np.asarray(x, np.float64)
    B = y.shape[0]
    L = _o.num_layers(params)
    k = params["w1"].shape[-1]
    xhat, c = forward_bf16(y, params, n1, n2, phi=phi, final_relu=final_relu, keep=True)
    d = f32(xhat - x.reshape(B, -1))
    loss = float(np.sum(d * d) / B)
    g = f32(f32(2.0 / B) * d)
    if final_relu:
        g = g * (xhat > 0)
    g = bf16(g).reshape(B, 1, n1, n2)
    grads = {}
    for l in range(L, 0, -1):
        grads["w%d" % l], grads["b%d" % l] = _o.conv_same_wgrad(c["a%d" % (l - 1)], g, k)
        if l > 1:
            # the mask of the stored activation (bfloat16 keeps the sign of ReLU's output)
            g = bf16(_o.conv_same_dgrad(g, bf16(params["w%d" % l]), n1, n2) * (c["a%d" % (l - 1)] > 0))
    if train_fc:
        dxt = f32(_o.conv_same_dgrad(g, bf16(params["w1"]), n1, n2)).reshape(B, n1 * n2)
        grads["wfc"] = _o.fc_wgrad(bf16(dxt), bf16(y))
    return loss, grads
