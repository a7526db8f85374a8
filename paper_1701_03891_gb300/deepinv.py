"""Thin Python binding of libdeepinv.so (C ABI in include/deepinv.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides device memory and streams; tensors are passed
as raw device pointers.  There is no fallback: if the library is missing or
a call fails, a ``DeepInvError`` is raised.

Paper: Mousavi & Baraniuk, "Learning to Invert: Signal Recovery via Deep
Convolutional Networks", arXiv 1701.03891 -- y = Phi x (Sec. 1), the network
x^ = M(y, Omega) of Sec. 4 with the layer sizes of Sec. 5, and its MSE loss.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdeepinv.so")

F32 = 0
BF16 = 1
FP8 = 2
PRECISIONS = {"f32": F32, "fp32": F32, "bf16": BF16, "fp8": FP8, "e4m3": FP8}

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5, -6
_STATUS_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EUNSUPPORTED: "EUNSUPPORTED",
                 ETIMEOUT: "ETIMEOUT", EBUSY: "EBUSY"}


class DeepInvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (_STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class Request(ctypes.Structure):
    _fields_ = [("net_id", ctypes.c_int), ("y", ctypes.c_void_p), ("xhat", ctypes.c_void_p),
                ("tag", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("net_id", ctypes.c_int),
                ("batch", ctypes.c_int), ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_in_flight", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("peak_workspace_bytes", ctypes.c_size_t),
                ("evictions", ctypes.c_uint64), ("admission_waits", ctypes.c_uint64)]


class NetDesc(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("M", ctypes.c_int),
                ("l1", ctypes.c_int), ("l2", ctypes.c_int), ("l3", ctypes.c_int),
                ("k", ctypes.c_int), ("final_relu", ctypes.c_int), ("train_fc", ctypes.c_int),
                ("prec", ctypes.c_int), ("hidden", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/deepinv.h
SIGNATURES = {
    "deepinv_last_error": (ctypes.c_char_p, []),
    "deepinv_version": (_I, []),
    "deepinv_device_status": (_I, [_I]),
    "deepinv_launch_count": (ctypes.c_ulonglong, []),
    "deepinv_selftest_bounded_wait": (_I, [_P]),
    "deepinv_measure": (_I, [_P, _I, _I, _P, _I, _P, _I, _P]),
    "deepinv_measure_noalloc": (_I, [_P, _I, _I, _P, _I, _P, _P]),
    "deepinv_net_create": (_I, [ctypes.POINTER(NetDesc), _P, _PP, _PP, _P, ctypes.POINTER(_P)]),
    "deepinv_net_destroy": (_I, [_P]),
    "deepinv_net_calibrate": (_I, [_P, _P, _I, _P]),
    "deepinv_net_get_desc": (_I, [_P, ctypes.POINTER(NetDesc)]),
    "deepinv_net_reserve": (_I, [_P, _I, _P]),
    "deepinv_net_set_act_budget": (_I, [_P, ctypes.c_size_t]),
    "deepinv_net_set_fused": (_I, [_P, _I]),
    "deepinv_net_set_conv1_rows": (_I, [_P, _I]),
    "deepinv_net_measure": (_I, [_P, _P, _I, _P, _P]),
    "deepinv_saved_bytes": (ctypes.c_size_t, [_P, _I]),
    "deepinv_forward": (_I, [_P, _P, _I, _P, _P, _P]),
    "deepinv_forward_host": (_I, [_P, _P, _I, _P, _P]),
    "deepinv_sense_recover_host": (_I, [_P, _P, _I, _P, _P]),
    "deepinv_sense_recover_host_submit": (_I, [_P, _P, _I, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "deepinv_host_wait": (_I, [_P, ctypes.c_uint64]),
    "deepinv_backward": (_I, [_P, _P, _P, _I, _P, _PP, _PP, _P, _P, _P]),
    "deepinv_sgd_momentum": (_I, [_P, _PP, _PP, _P, ctypes.c_float, ctypes.c_float, _P]),
    "deepinv_get_params": (_I, [_P, _PP, _PP, _P, _P]),
    "deepinv_net_save_state": (_I, [_P, ctypes.c_char_p]),
    "deepinv_net_load_state": (_I, [_P, ctypes.c_char_p, _P]),
    "deepinv_serve_open": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_P)]),
    "deepinv_serve_add_net": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "deepinv_serve": (_I, [_P, ctypes.POINTER(Request), _I, ctypes.POINTER(Result), _I, ctypes.POINTER(_I), _I]),
    "deepinv_serve_get_stats": (_I, [_P, ctypes.POINTER(ServeStats)]),
    "deepinv_serve_close": (_I, [_P]),
    "deepinv_profile_enable": (_I, [_P, _I]),
    "deepinv_profile_read": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]),
}

NSTAGES = 6
STAGES = ("measure", "fc", "conv1", "conv2", "conv3", "hidden")
MAX_HIDDEN = 16


def lib():
    """Load libdeepinv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise DeepInvError(ECUDA, "libdeepinv.so not built (run __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        msg = lib().deepinv_last_error()
        raise DeepInvError(rc, msg.decode() if msg else "")


def _ptr(t) -> int:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# The library cannot see the extent of a buffer it is handed, so the binding
# checks every tensor's kind and size before the call: a short buffer would
# otherwise be read or written past its end.
def _need_f32_cuda(t, name, numel=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise DeepInvError(EINVAL, "%s must be a contiguous float32 CUDA tensor" % name)
    if numel is not None and t.numel() != numel:
        raise DeepInvError(EINVAL, "%s has %d elements, expected %d" % (name, t.numel(), numel))


def _need_f32_host(t, name, numel):
    import torch
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float32
            and t.is_contiguous()):
        raise DeepInvError(EINVAL, "%s must be a contiguous float32 CPU tensor" % name)
    if t.numel() != numel:
        raise DeepInvError(EINVAL, "%s has %d elements, expected %d" % (name, t.numel(), numel))


def _batch(t, name, cols):
    """Rows B of a tensor holding B rows of `cols` values ([B][cols] or any
    shape with B leading and cols values per row)."""
    B = t.shape[0] if t.dim() >= 1 else 0
    if t.numel() != B * cols:
        raise DeepInvError(EINVAL, "%s: %d elements are not %d rows of %d" % (name, t.numel(), B, cols))
    return B


def _need_cuda_bytes(t, name, nbytes):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise DeepInvError(EINVAL, "%s must be a contiguous CUDA tensor" % name)
    if t.numel() * t.element_size() < nbytes:
        raise DeepInvError(EINVAL, "%s holds %d bytes, the call needs %d"
                           % (name, t.numel() * t.element_size(), nbytes))


def _arr(ptrs):
    a = (ctypes.c_void_p * len(ptrs))(*ptrs)
    return ctypes.cast(a, _PP), a


def device_status(reset: bool = False) -> int:
    return lib().deepinv_device_status(1 if reset else 0)


def launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().deepinv_launch_count())


def selftest_bounded_wait(stream=None):
    """Run one kernel whose bounded wait never completes (about 1 s); afterwards
    device_status() reports ETIMEOUT until reset."""
    _check(lib().deepinv_selftest_bounded_wait(_stream(stream)))


def measure(phi, x, prec="f32", out=None, stream=None):
    """y = Phi x (Sec. 1).  phi [M][N], x [B][N] float32 CUDA -> y [B][M]."""
    import torch
    _need_f32_cuda(phi, "phi")
    _need_f32_cuda(x, "x")
    M, N = phi.shape
    B = _batch(x, "x", N)
    y = out if out is not None else torch.empty((B, M), device=x.device, dtype=torch.float32)
    _need_f32_cuda(y, "out", B * M)
    _check(lib().deepinv_measure(_ptr(phi), M, N, _ptr(x), B, _ptr(y), PRECISIONS.get(prec, prec),
                                 _stream(stream)))
    return y


def measure_noalloc(phi, x, out, stream=None):
    """y = Phi x in bfloat16 without any device allocation by the library: the
    packed operands live in a static 32 MiB device array (see deepinv.h).
    ``out`` [B][M] must be supplied by the caller."""
    _need_f32_cuda(phi, "phi")
    _need_f32_cuda(x, "x")
    M, N = phi.shape
    B = _batch(x, "x", N)
    _need_f32_cuda(out, "out", B * M)
    _check(lib().deepinv_measure_noalloc(_ptr(phi), M, N, _ptr(x), B, _ptr(out), _stream(stream)))
    return out


def num_layers(params: dict) -> int:
    """Conv layers L of a parameter dict holding w1, b1, ..., wL, bL."""
    L = 0
    while "w%d" % (L + 1) in params:
        L += 1
    return L


class Net:
    """A DeepInverse network (Sec. 4) held by the library: FC = Phi^T, then
    conv layers (Eq. 1).  ``params`` maps w1,b1,...,wL,bL (network order;
    L = 3 is the paper's network, L > 3 adds L - 3 hidden l2 -> l2 layers
    before the last) to float32 tensors (CUDA or CPU; copied)."""

    def __init__(self, phi, params: dict, n1: int, n2: int, *, prec="bf16", final_relu=False,
                 train_fc=False, device="cuda"):
        import torch
        dev = torch.device(device)
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).to(dev).contiguous()
        phi_t = t(phi)
        if phi_t.dim() != 2 or phi_t.shape[1] != n1 * n2:
            raise DeepInvError(EINVAL, "phi must be M x (n1*n2), got %s" % (tuple(phi_t.shape),))
        M, N = phi_t.shape
        L = num_layers(params)
        if L < 3:
            raise DeepInvError(EINVAL, "params need w1..wL, b1..bL with L >= 3")
        ws = [t(params["w%d" % i]) for i in range(1, L + 1)]
        bs = [t(params["b%d" % i]) for i in range(1, L + 1)]
        # layer l maps cin -> cout channels with k x k kernels: w [cout][cin][k][k],
        # b [cout]; the hidden layers (between the second and the last) keep the
        # second layer's channel count
        k = ws[0].shape[-1]
        cin = 1
        for i, (w, b) in enumerate(zip(ws, bs)):
            cout = w.shape[0] if w.dim() == 4 else -1
            if 2 <= i < L - 1 and cout != ws[1].shape[0]:
                raise DeepInvError(EINVAL, "hidden layer %d has %d filters, the second layer %d"
                                   % (i + 1, cout, ws[1].shape[0]))
            if tuple(w.shape) != (cout, cin, k, k) or tuple(b.shape) != (cout,):
                raise DeepInvError(EINVAL, "layer %d: w %s and b %s, expected w [cout][%d][%d][%d] and b [cout]"
                                   % (i + 1, tuple(w.shape), tuple(b.shape), cin, k, k))
            cin = cout
        self.L = L
        self.desc = NetDesc(n1, n2, M, ws[0].shape[0], ws[1].shape[0], ws[-1].shape[0], ws[0].shape[-1],
                            int(final_relu), int(train_fc), PRECISIONS.get(prec, prec), L - 3)
        self.n1, self.n2, self.M, self.N = n1, n2, M, N
        self.prec = prec
        self.device = dev
        self._h = ctypes.c_void_p()
        wp, _k1 = _arr([w.data_ptr() for w in ws])
        bp, _k2 = _arr([b.data_ptr() for b in bs])
        _check(lib().deepinv_net_create(ctypes.byref(self.desc), phi_t.data_ptr(), wp, bp,
                                        _stream(), ctypes.byref(self._h)))
        self.shapes = [tuple(w.shape) for w in ws]

    def close(self):
        if self._h:
            lib().deepinv_net_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def calibrate(self, y, stream=None):
        """Fix the e4m3 activation scale from a calibration batch y [B][M] (no-op otherwise)."""
        _need_f32_cuda(y, "y")
        _check(lib().deepinv_net_calibrate(self._h, _ptr(y), _batch(y, "y", self.M), _stream(stream)))

    def reserve(self, max_B: int, stream=None):
        _check(lib().deepinv_net_reserve(self._h, max_B, _stream(stream)))

    def measure(self, x, out=None, stream=None):
        import torch
        _need_f32_cuda(x, "x")
        B = _batch(x, "x", self.N)
        y = out if out is not None else torch.empty((B, self.M), device=x.device, dtype=torch.float32)
        _need_f32_cuda(y, "out", B * self.M)
        _check(lib().deepinv_net_measure(self._h, _ptr(x), B, _ptr(y), _stream(stream)))
        return y

    def saved_bytes(self, B: int) -> int:
        return int(lib().deepinv_saved_bytes(self._h, B))

    def forward(self, y, out=None, saved=None, stream=None):
        """x^ = M(y, Omega).  y [B][M] -> x^ [B][N]."""
        import torch
        _need_f32_cuda(y, "y")
        B = _batch(y, "y", self.M)
        xh = out if out is not None else torch.empty((B, self.N), device=y.device, dtype=torch.float32)
        _need_f32_cuda(xh, "out", B * self.N)
        if saved is not None:
            _need_cuda_bytes(saved, "saved", self.saved_bytes(B))
        _check(lib().deepinv_forward(self._h, _ptr(y), B, _ptr(xh), _ptr(saved), _stream(stream)))
        return xh

    __call__ = forward

    def forward_host(self, y_host, out_host=None, stream=None):
        """End to end from host memory (pinned for async copies); returns a CPU tensor."""
        import torch
        _need_f32_host(y_host, "y_host", y_host.numel())
        B = _batch(y_host, "y_host", self.M)
        xh = out_host if out_host is not None else torch.empty((B, self.N), dtype=torch.float32)
        _need_f32_host(xh, "out_host", B * self.N)
        _check(lib().deepinv_forward_host(self._h, y_host.data_ptr(), B, xh.data_ptr(), _stream(stream)))
        return xh

    def sense_recover_host(self, x_host, out_host=None, stream=None):
        import torch
        _need_f32_host(x_host, "x_host", x_host.numel())
        B = _batch(x_host, "x_host", self.N)
        xh = out_host if out_host is not None else torch.empty((B, self.N), dtype=torch.float32)
        _need_f32_host(xh, "out_host", B * self.N)
        _check(lib().deepinv_sense_recover_host(self._h, x_host.data_ptr(), B, xh.data_ptr(),
                                                _stream(stream)))
        return xh

    def sense_recover_host_submit(self, x_host, out_host, stream=None) -> int:
        """Queue sense + recover of a pinned host batch x [B][N] into the pinned
        out_host [B][N] and return a ticket (two batches' copies and compute
        overlap); keep both buffers alive until host_wait(ticket)."""
        _need_f32_host(x_host, "x_host", x_host.numel())
        B = _batch(x_host, "x_host", self.N)
        _need_f32_host(out_host, "out_host", B * self.N)
        t = ctypes.c_uint64()
        _check(lib().deepinv_sense_recover_host_submit(self._h, x_host.data_ptr(), B,
                                                       out_host.data_ptr(), _stream(stream), ctypes.byref(t)))
        return t.value

    def host_wait(self, ticket: int):
        _check(lib().deepinv_host_wait(self._h, ctypes.c_uint64(ticket)))

    def new_saved(self, B: int):
        import torch
        return torch.empty(self.saved_bytes(B), dtype=torch.uint8, device=self.device)

    def _check_grads(self, dW, db, dWfc):
        if len(dW) != self.L or len(db) != self.L:
            raise DeepInvError(EINVAL, "need %d weight and bias gradients, got %d and %d"
                               % (self.L, len(dW), len(db)))
        for i, s in enumerate(self.shapes):
            _need_f32_cuda(dW[i], "dW[%d]" % i, s[0] * s[1] * s[2] * s[3])
            _need_f32_cuda(db[i], "db[%d]" % i, s[0])
        if self.desc.train_fc:
            _need_f32_cuda(dWfc, "dWfc", self.N * self.M)

    def grad_buffers(self):
        import torch
        dW = [torch.empty(s, device=self.device, dtype=torch.float32) for s in self.shapes]
        db = [torch.empty(s[0], device=self.device, dtype=torch.float32) for s in self.shapes]
        dWfc = (torch.empty((self.N, self.M), device=self.device, dtype=torch.float32)
                if self.desc.train_fc else None)
        return dW, db, dWfc

    def set_act_budget(self, nbytes: int):
        """Activation budget of backward(saved=None): the forward activations are
        recomputed in chunks of images whose activations fit nbytes (0: one chunk)."""
        _check(lib().deepinv_net_set_act_budget(self._h, int(nbytes)))

    def set_fused(self, enable: bool):
        """conv1 + conv2 as one fused kernel in inference forward passes (bf16 networks)."""
        _check(lib().deepinv_net_set_fused(self._h, 1 if enable else 0))

    def set_conv1_rows(self, mode: int):
        """conv1 in row tiles with its input windows in TMEM: 0 never, 1 where they
        are faster (the default), 2 wherever they fit."""
        _check(lib().deepinv_net_set_conv1_rows(self._h, int(mode)))

    def backward(self, y, x, saved=None, grads=None, stream=None):
        """Gradient of L = (1/B) sum_b ||x^_b - x_b||^2 (Sec. 4).  Returns (loss tensor, dW, db, dWfc).
        saved: the buffer forward(..., saved=) filled, or None to recompute the activations."""
        import torch
        _need_f32_cuda(y, "y")
        _need_f32_cuda(x, "x")
        B = _batch(y, "y", self.M)
        _need_f32_cuda(x, "x", B * self.N)
        if saved is not None:
            _need_cuda_bytes(saved, "saved", self.saved_bytes(B))
        dW, db, dWfc = grads if grads is not None else self.grad_buffers()
        self._check_grads(dW, db, dWfc)
        loss = torch.empty((), device=self.device, dtype=torch.float64)
        wp, _k1 = _arr([t.data_ptr() for t in dW])
        bp, _k2 = _arr([t.data_ptr() for t in db])
        _check(lib().deepinv_backward(self._h, _ptr(y), _ptr(x), B, _ptr(saved), wp, bp, _ptr(dWfc),
                                      _ptr(loss), _stream(stream)))
        return loss, dW, db, dWfc

    def sgd_momentum(self, dW, db, dWfc=None, lr=1e-3, mu=0.9, stream=None):
        self._check_grads(dW, db, dWfc)
        wp, _k1 = _arr([t.data_ptr() for t in dW])
        bp, _k2 = _arr([t.data_ptr() for t in db])
        _check(lib().deepinv_sgd_momentum(self._h, wp, bp, _ptr(dWfc), float(lr), float(mu),
                                          _stream(stream)))

    def profile(self, enable: bool = True):
        """Start (or stop) recording CUDA events around each stage of measure/forward."""
        _check(lib().deepinv_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{stage: (total device ms, count)} since profile(True); clears the record."""
        ms = (ctypes.c_float * NSTAGES)()
        cnt = (ctypes.c_int * NSTAGES)()
        _check(lib().deepinv_profile_read(self._h, ms, cnt))
        return {STAGES[i]: (float(ms[i]), int(cnt[i])) for i in range(NSTAGES)}

    def save_state(self, path: str):
        """Write the training state (masters, momentum, FC) to ``path``."""
        _check(lib().deepinv_net_save_state(self._h, os.fsencode(path)))

    def load_state(self, path: str, stream=None):
        """Read a training state saved from a network of the same description."""
        _check(lib().deepinv_net_load_state(self._h, os.fsencode(path), _stream(stream)))

    def get_params(self, stream=None) -> dict:
        import torch
        W = [torch.empty(s, device=self.device, dtype=torch.float32) for s in self.shapes]
        Bv = [torch.empty(s[0], device=self.device, dtype=torch.float32) for s in self.shapes]
        wfc = (torch.empty((self.N, self.M), device=self.device, dtype=torch.float32)
               if self.desc.train_fc else None)
        wp, _k1 = _arr([t.data_ptr() for t in W])
        bp, _k2 = _arr([t.data_ptr() for t in Bv])
        _check(lib().deepinv_get_params(self._h, wp, bp, _ptr(wfc), _stream(stream)))
        out = {}
        for i in range(self.L):
            out["w%d" % (i + 1)], out["b%d" % (i + 1)] = W[i], Bv[i]
        if wfc is not None:
            out["wfc"] = wfc
        return out


def _make_autograd():
    import torch

    class DeepInverseMSE(torch.autograd.Function):
        """L(Omega) of Sec. 4 as an autograd node over the network's parameters.

        forward(net, y, x, *params) runs the library's forward (saving the
        activations) and its hand-written backward in one go and returns the
        loss; backward hands the stored parameter gradients, scaled by the
        incoming gradient, to autograd.  ``params`` are placeholders that
        carry requires_grad (the library holds the weights themselves)."""

        @staticmethod
        def forward(ctx, net, y, x, *params):
            B = y.shape[0]
            saved = net.new_saved(B)
            net.forward(y, saved=saved)
            loss, dW, db, dWfc = net.backward(y, x, saved)
            grads = [g for pair in zip(dW, db) for g in pair]
            if dWfc is not None:
                grads.append(dWfc)
            ctx.grads = grads
            return loss.to(torch.float32)

        @staticmethod
        def backward(ctx, gout):
            g = [t * gout for t in ctx.grads]
            return (None, None, None, *g[:len(ctx.needs_input_grad) - 3])

    return DeepInverseMSE


_autograd_cls = None


def mse_loss(net: Net, y, x, params):
    """Differentiable L(Omega); ``params`` is the list [w1, b1, ..., wL, bL(, wfc)]."""
    global _autograd_cls
    if _autograd_cls is None:
        _autograd_cls = _make_autograd()
    return _autograd_cls.apply(net, y, x, *params)


def _need_host_vec(a, name, n):
    """A float32 host array (numpy or CPU tensor) of exactly n contiguous values."""
    import numpy as np
    import torch
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.size == n
    else:
        ok = (isinstance(a, torch.Tensor) and a.device.type == "cpu" and a.dtype == torch.float32
              and a.is_contiguous() and a.numel() == n)
    if not ok:
        raise DeepInvError(EINVAL, "%s must be %d contiguous float32 values in host memory" % (name, n))


class Server:
    """Continuous-batching recovery server (deepinv_serve_*): host y in, host x^ out."""

    def __init__(self, hbm_budget_bytes: int, max_streams: int = 4, max_batch: int = 64):
        self._h = ctypes.c_void_p()
        _check(lib().deepinv_serve_open(int(hbm_budget_bytes), max_streams, max_batch, ctypes.byref(self._h)))
        self.nets = []

    def add(self, net: "Net") -> int:
        nid = ctypes.c_int()
        _check(lib().deepinv_serve_add_net(self._h, net.handle, ctypes.byref(nid)))
        self.nets.append(net)
        return nid.value

    def serve(self, requests=(), max_out: int = 4096, timeout_us: int = 0):
        """Submit [(net_id, y_host_array, xhat_host_array, tag), ...] and harvest finished results.
        Returns (status, [Result, ...])."""
        n_in = len(requests)
        arr = (Request * max(1, n_in))()
        for i, (nid, y, xh, tag) in enumerate(requests):
            if 0 <= nid < len(self.nets):   # (an unknown net_id is the library's to reject)
                _need_host_vec(y, "request %d: y" % i, self.nets[nid].M)
                _need_host_vec(xh, "request %d: xhat" % i, self.nets[nid].N)
            arr[i] = Request(nid, y.ctypes.data if hasattr(y, "ctypes") else y.data_ptr(),
                             xh.ctypes.data if hasattr(xh, "ctypes") else xh.data_ptr(), tag)
        out = (Result * max(1, max_out))()
        n_out = ctypes.c_int()
        rc = lib().deepinv_serve(self._h, arr, n_in, out, max_out, ctypes.byref(n_out), timeout_us)
        if rc not in (OK, ETIMEOUT):
            _check(rc)
        return rc, [out[i] for i in range(n_out.value)]

    def serve_raw(self, reqs, offset: int, count: int, results, max_out: int, timeout_us: int = 0):
        """Low-overhead form: ``reqs`` and ``results`` are preallocated ctypes arrays of
        Request / Result; submits reqs[offset:offset+count]; returns (rc, n_out)."""
        n_out = ctypes.c_int()
        base = ctypes.cast(ctypes.byref(reqs, offset * ctypes.sizeof(Request)), ctypes.POINTER(Request))
        rc = lib().deepinv_serve(self._h, base, count, results, max_out, ctypes.byref(n_out), timeout_us)
        if rc not in (OK, ETIMEOUT):
            _check(rc)
        return rc, n_out.value

    def stats(self) -> dict:
        st = ServeStats()
        _check(lib().deepinv_serve_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def close(self):
        if self._h:
            lib().deepinv_serve_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
