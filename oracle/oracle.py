"""FP64 CPU oracle for the DeepInverse hot path (Mousavi & Baraniuk, arXiv 1701.03891).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA path (``paper_1701_03891_gb300``) and imports
nothing from it; the two meet only through the seeded input arrays the tests
hand to both.

What it computes, each step citing the paper:
  * ``measure``      y = Phi x                              (Sec. 1)
  * ``fc``           x~ = W y, W = Phi^T by default          (Sec. 4, the fixed FC layer)
  * ``conv_same``    Eq. (1) before the ReLU, 'same' size    (Sec. 4, Eq. 1; crop S)
  * ``forward``      x^ = M(y, Omega): FC, reshape n1 x n2, three conv layers,
                     ReLU after the first two                (Sec. 4, Sec. 5 layer sizes);
                     more layers in between when params hold them (the deeper
                     networks Sec. 5 names as future work)
  * ``mse_loss``     L = (1/l) sum_i ||x^(i) - x(i)||^2      (Sec. 4, the MSE objective)
  * ``backward``     the hand-derived gradient of that loss  (Sec. 4, backpropagation)
  * ``rel_l2``, ``psnr``, ``success``                        (Sec. 5 metrics)

The arithmetic lives in ``oracle.c`` (plain loops, double precision); this file
composes those routines in the paper's order and holds the small elementwise
steps (ReLU, loss, metrics) in numpy float64.

Parity status: every routine here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, library special cases, finite differences).  The
paper's own accuracy numbers (Tables 2-3, Figs. 2-5) need ImageNet and trained
weights: parity unpinned for those, and no routine here reproduces them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            lib.oracle_measure.argtypes = [dp, i, i, dp, i, dp]
            lib.oracle_fc.argtypes = [dp, i, i, dp, i, dp]
            lib.oracle_conv_same.argtypes = [dp, i, i, i, i, dp, dp, i, i, dp]
            lib.oracle_conv_full.argtypes = [dp, i, i, i, i, dp, dp, i, i, dp]
            lib.oracle_conv_same_wgrad.argtypes = [dp, dp, i, i, i, i, i, i, dp, dp]
            lib.oracle_conv_same_dgrad.argtypes = [dp, dp, i, i, i, i, i, i, dp]
            lib.oracle_fc_wgrad.argtypes = [dp, dp, i, i, i, dp]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_num_threads.argtypes = [i]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(_get().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    _get().oracle_set_num_threads(int(n))


# ---------------------------------------------------------------- primitives
def measure(phi, x) -> np.ndarray:
    """Sec. 1: y = Phi x.  phi [M][N], x [B][N] -> y [B][M] (float64)."""
    phi, x = _f64(phi), _f64(x)
    M, N = phi.shape
    x2 = x.reshape(-1, N)
    y = np.empty((x2.shape[0], M))
    _get().oracle_measure(_p(phi), M, N, _p(x2), x2.shape[0], _p(y))
    return y


def fc(w, y) -> np.ndarray:
    """Sec. 4 FC layer: w [N][M], y [B][M] -> x~ [B][N].  w = Phi^T gives the adjoint."""
    w, y = _f64(w), _f64(y)
    N, M = w.shape
    y2 = y.reshape(-1, M)
    xt = np.empty((y2.shape[0], N))
    _get().oracle_fc(_p(w), N, M, _p(y2), y2.shape[0], _p(xt))
    return xt


def conv_same(a, w, bias=None) -> np.ndarray:
    """Eq. (1) before ReLU with the crop S read as 'same' zero padding.
    a [B][Cin][H][W], w [Cout][Cin][k][k], bias [Cout] -> z [B][Cout][H][W]."""
    a, w = _f64(a), _f64(w)
    B, Cin, H, W = a.shape
    Cout, Cin2, k, k2 = w.shape
    assert Cin2 == Cin and k == k2 and k % 2 == 1
    b = _f64(bias) if bias is not None else None
    z = np.empty((B, Cout, H, W))
    _get().oracle_conv_same(_p(a), B, Cin, H, W, _p(w), _p(b) if b is not None else None,
                            Cout, k, _p(z))
    return z


def conv_full(a, w, bias=None) -> np.ndarray:
    """Eq. (1) literally: full correlation, output (H+k-1) x (W+k-1), before the crop S."""
    a, w = _f64(a), _f64(w)
    B, Cin, H, W = a.shape
    Cout, _, k, _ = w.shape
    b = _f64(bias) if bias is not None else None
    z = np.empty((B, Cout, H + k - 1, W + k - 1))
    _get().oracle_conv_full(_p(a), B, Cin, H, W, _p(w), _p(b) if b is not None else None,
                            Cout, k, _p(z))
    return z


def crop_S(zf, k: int) -> np.ndarray:
    """The crop S of Eq. (1): drop the (k-1)/2 border rows/columns the zero padding created."""
    h = (k - 1) // 2
    return zf[..., h:zf.shape[-2] - h, h:zf.shape[-1] - h]


def conv_same_wgrad(a, g, k: int):
    """dL/dw and dL/db of one 'same' layer given g = dL/dz and its input a."""
    a, g = _f64(a), _f64(g)
    B, Cin, H, W = a.shape
    Cout = g.shape[1]
    dw = np.empty((Cout, Cin, k, k))
    db = np.empty(Cout)
    _get().oracle_conv_same_wgrad(_p(a), _p(g), B, Cin, H, W, Cout, k, _p(dw), _p(db))
    return dw, db


def conv_same_dgrad(g, w, H: int, W: int) -> np.ndarray:
    """dL/da of one 'same' layer given g = dL/dz and the layer weights."""
    g, w = _f64(g), _f64(w)
    B, Cout = g.shape[:2]
    _, Cin, k, _ = w.shape
    da = np.empty((B, Cin, H, W))
    _get().oracle_conv_same_dgrad(_p(g), _p(w), B, Cin, H, W, Cout, k, _p(da))
    return da


def fc_wgrad(dxt, y) -> np.ndarray:
    dxt, y = _f64(dxt), _f64(y)
    B, N = dxt.shape
    M = y.shape[1]
    dw = np.empty((N, M))
    _get().oracle_fc_wgrad(_p(dxt), _p(y), B, N, M, _p(dw))
    return dw


def relu(z) -> np.ndarray:
    """ReLU(x) = max(0, x) (Sec. 4, after Eq. 1)."""
    return np.maximum(z, 0.0)


# ---------------------------------------------------------------- the network
def num_layers(params: dict) -> int:
    """Number L of convolutional layers: params holds w1, b1, ..., wL, bL."""
    L = 0
    while "w%d" % (L + 1) in params:
        L += 1
    return L


def forward(y, params: dict, n1: int, n2: int, *, phi=None, wfc=None, final_relu: bool = False,
            keep: bool = False):
    """x^ = M(y, Omega) (Sec. 4).

    y [B][M]; params holds w1,b1,...,wL,bL with w_l [l_l][l_{l-1}][k][k]
    (L = 3 is the paper's network; a larger L adds layers in between, the
    larger-capacity networks Sec. 5 leaves to future work).
    The FC weights are Phi^T (fixed, Sec. 4) unless ``wfc`` [N][M] is given.
    The proxy x~ = W y is reshaped row-major to n1 x n2 (Sec. 4).  Every
    convolutional layer follows Eq. (1); ReLU follows every layer but the
    last, and the last too only when ``final_relu`` (the paper's literal
    'each layer').  Returns x^ [B][n1*n2] (and, when ``keep``, the proxy
    xt, a0 = the reshaped proxy and z_l, a_l for every layer).
    """
    y = _f64(y)
    B = y.shape[0]
    L = num_layers(params)
    if wfc is None:
        wfc = _f64(phi).T
    xt = fc(wfc, y)
    a = xt.reshape(B, 1, n1, n2)
    c = dict(xt=xt, a0=a)
    for l in range(1, L + 1):
        z = conv_same(a, params["w%d" % l], params["b%d" % l])
        a = relu(z) if (l < L or final_relu) else z
        c["z%d" % l] = z
        c["a%d" % l] = a
    xhat = a.reshape(B, n1 * n2)
    if keep:
        return xhat, c
    return xhat


def mse_loss(xhat, x) -> float:
    """L(Omega) = (1/l) sum_i ||x^(i) - x(i)||_2^2 over the l signals of the batch (Sec. 4)."""
    xhat, x = _f64(xhat), _f64(x)
    B = xhat.shape[0]
    d = (xhat - x).reshape(B, -1)
    return float(np.sum(d * d) / B)


def backward(y, x, params: dict, n1: int, n2: int, *, phi=None, wfc=None,
             final_relu: bool = False, train_fc: bool = False):
    """Gradient of ``mse_loss(forward(y), x)`` with respect to every parameter.

    Chain rule through Sec. 4's network, layer by layer from the output:
      g_L = dL/dz_L = 2 (x^ - x) / B        (times [z_L > 0] when final_relu)
      for l = L .. 1:  dW_l, db_l from g_l and a_{l-1};
                       for l > 1:  g_{l-1} = dgrad(g_l) * [z_{l-1} > 0]
      with train_fc: dx~ = dgrad(g_1), dWfc = sum_b dx~ y^T.
    The ReLU derivative at 0 is taken as 0.
    Returns (loss, grads dict).
    """
    y, x = _f64(y), _f64(x)
    B = y.shape[0]
    L = num_layers(params)
    if wfc is None:
        wfc = _f64(phi).T
    xhat, c = forward(y, params, n1, n2, wfc=wfc, final_relu=final_relu, keep=True)
    loss = mse_loss(xhat, x)
    k = params["w1"].shape[-1]
    g = (2.0 / B) * (xhat - x.reshape(B, -1)).reshape(c["z%d" % L].shape)
    if final_relu:
        g = g * (c["z%d" % L] > 0)
    grads = {}
    for l in range(L, 0, -1):
        grads["w%d" % l], grads["b%d" % l] = conv_same_wgrad(c["a%d" % (l - 1)], g, k)
        if l > 1:
            g = conv_same_dgrad(g, params["w%d" % l], n1, n2) * (c["z%d" % (l - 1)] > 0)
    if train_fc:
        dxt = conv_same_dgrad(g, params["w1"], n1, n2).reshape(B, n1 * n2)
        grads["wfc"] = fc_wgrad(dxt, y)
    return loss, grads


def sgd_momentum(w, v, g, lr: float, mu: float):
    """One heavy-ball step on a master weight: v <- mu v + g ; w <- w - lr v.
    (The paper trains by backpropagation without naming the optimiser; this is
    the optimiser the build uses.)"""
    v_new = mu * _f64(v) + _f64(g)
    return _f64(w) - lr * v_new, v_new


# ---------------------------------------------------------------- metrics (Sec. 5)
def rel_l2(a, b) -> np.ndarray:
    """Per-signal ||a - b||_2 / ||b||_2."""
    a, b = _f64(a), _f64(b)
    B = a.shape[0]
    a2, b2 = a.reshape(B, -1), b.reshape(B, -1)
    return np.linalg.norm(a2 - b2, axis=1) / np.linalg.norm(b2, axis=1)


def psnr(xhat, x, peak: float = 1.0) -> np.ndarray:
    """PSNR = 10 log10(max^2 / MSE) per image, MSE the mean over pixels (Sec. 5 footnote)."""
    xhat, x = _f64(xhat), _f64(x)
    B = x.shape[0]
    mse = np.mean((xhat.reshape(B, -1) - x.reshape(B, -1)) ** 2, axis=1)
    return 10.0 * np.log10(peak * peak / mse)


def success(xhat, x) -> np.ndarray:
    """Sec. 5 success variable: 1 if ||x^ - x||^2 / ||x||^2 <= 0.1 (inclusive)."""
    xhat, x = _f64(xhat), _f64(x)
    B = x.shape[0]
    d = np.sum((xhat.reshape(B, -1) - x.reshape(B, -1)) ** 2, axis=1)
    n = np.sum(x.reshape(B, -1) ** 2, axis=1)
    return (d / n <= 0.1).astype(np.int64)
