"""Recovery quality of trained networks (Sec. 5): train a network on seeded
synthetic images with the library's own training step, then measure the
recovered images' PSNR and success rate on held-out images, optionally with
noisy measurements (Table 3: y = Phi x + e at a given SNR).

Everything on the GPU runs in libdeepinv (measurement, forward, backward,
update); this module only draws the data and the measurement noise (seeded, on
the host, like synth.py) and computes the metrics from the results:

    PSNR    = 10 log10(1 / MSE), MSE the mean over the image's pixels, images in
              [0, 1] (Sec. 5);
    success = 1 when ||x^ - x||^2 / ||x||^2 <= 0.1 (Sec. 5).
"""
from __future__ import annotations

import numpy as np

from . import synth


def psnr(xhat: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Per-image PSNR in dB for images in [0, 1]."""
    d = (np.asarray(xhat, np.float64) - np.asarray(x, np.float64)).reshape(len(x), -1)
    return 10.0 * np.log10(1.0 / np.mean(d * d, axis=1))


def success(xhat: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Per-image success indicator, ||x^ - x||^2 / ||x||^2 <= 0.1."""
    xh = np.asarray(xhat, np.float64).reshape(len(x), -1)
    xx = np.asarray(x, np.float64).reshape(len(x), -1)
    return (np.sum((xh - xx) ** 2, axis=1) / np.sum(xx * xx, axis=1) <= 0.1).astype(np.int64)


def add_noise(y: np.ndarray, snr_db: float | None, seed: int) -> np.ndarray:
    """y + e with e ~ N(0, s^2) i.i.d. per measurement vector, s^2 = ||y||^2 / (M 10^(snr/10))."""
    if snr_db is None:
        return y
    rng = np.random.default_rng(seed)
    y = np.asarray(y, np.float64)
    power = np.mean(y * y, axis=1, keepdims=True) / (10.0 ** (snr_db / 10.0))
    return (y + rng.standard_normal(y.shape) * np.sqrt(power)).astype(np.float32)


def train_and_evaluate(n: int = 32, ratio: float = 0.25, *, images: str = "voronoi", train_images: int = 512,
                       test_images: int = 64, batch: int = 64, steps: int = 6000, lr: float | None = None,
                       lr_scale: float = 1e-3,
                       mu: float = 0.9, snr_db: float | None = None, prec: str = "bf16", seed: int = 0,
                       hidden: int = 0, curve_every: int | None = None) -> dict:
    """Train an n x n network at measurement ratio M/N (the FC layer fixed to Phi^T)
    with SGD with momentum on the bfloat16 path and evaluate it.  The loss is a
    sum over pixels (Sec. 4), so its scale varies with M/N and the images; the
    step is lr, or lr_scale / (the first batch's loss) when lr is None.  With snr_db,
    training and test measurements carry Gaussian noise at that SNR.  ``hidden``
    adds that many 32 -> 32 layers before the last (the deeper networks of
    Sec. 5).  Returns the mean PSNR and success rate on the test images, before
    and after training, and the first and last training losses; with
    ``curve_every``, also the test PSNR and success rate every that many steps
    (the convergence of training, Fig. 5's analogue)."""
    import torch
    from . import deepinv

    N = n * n
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=seed)
    make = synth.voronoi_images if images == "voronoi" else (
        lambda B, a, b, seed: synth.dct_sparse_images(B, a, b, K=max(1, N // 20), seed=seed))
    xtrain = make(train_images, n, n, seed=seed + 21)
    xtest = make(test_images, n, n, seed=seed + 22)

    net = deepinv.Net(phi, synth.he_params(seed=seed + 1, hidden=hidden), n, n, prec="bf16")
    xt = torch.from_numpy(xtrain).cuda()

    def measure(x, noise_seed):
        y = net.measure(torch.from_numpy(x).cuda()).cpu().numpy()      # y = Phi x on the device
        return torch.from_numpy(np.ascontiguousarray(add_noise(y, snr_db, noise_seed), np.float32)).cuda()

    yt, yv = measure(xtrain, seed + 23), measure(xtest, seed + 24)

    def quality(model):
        xh = model.forward(yv).cpu().numpy()
        return float(np.mean(psnr(xh, xtest))), float(np.mean(success(xh, xtest)))

    before = quality(net)
    saved, grads = net.new_saved(batch), net.grad_buffers()
    first = last = loss = None
    step = lr
    curve = [(0, before[0], before[1])] if curve_every else None
    for k in range(steps):
        lo = (k * batch) % train_images
        yb, xb = yt[lo:lo + batch].contiguous(), xt[lo:lo + batch].contiguous()
        net.forward(yb, saved=saved)
        loss, dW, db, _ = net.backward(yb, xb, saved, grads=grads)
        if k == 0:
            first = float(loss)
            if step is None:
                step = lr_scale / first
        net.sgd_momentum(dW, db, None, lr=step, mu=mu)
        if curve_every and (k + 1) % curve_every == 0:
            curve.append((k + 1,) + quality(net))
    if loss is not None:
        last = float(loss)
    if prec == "bf16":
        after = quality(net)
    else:
        params = {k: v.cpu().numpy() for k, v in net.get_params().items()}
        other = deepinv.Net(phi, params, n, n, prec=prec)
        if prec == "fp8":
            other.calibrate(yt[:batch].contiguous())
        after = quality(other)
        other.close()
    net.close()
    return {"n": n, "ratio": ratio, "M": M, "snr_db": snr_db, "images": images, "steps": steps, "lr": step,
            "conv_layers": 3 + hidden, "curve": curve,
            "psnr_db_before": before[0], "success_before": before[1],
            "psnr_db": after[0], "success": after[1], "loss_first": first, "loss_last": last}


def sweep(n: int = 32, ratios=(0.05, 0.10, 0.25), snrs=(None, 20.0), **kw) -> list:
    """PSNR and success rate against M/N, with and without measurement noise
    (the analogue of Sec. 5's quality-versus-ratio experiments on synthetic data)."""
    return [train_and_evaluate(n, r, snr_db=s, **kw) for r in ratios for s in snrs]


def depth_sweep(n: int = 32, ratio: float = 0.10, hiddens=(0, 1, 2), **kw) -> list:
    """PSNR and success rate of networks with 3 + h conv layers (h in hiddens)
    trained the same way -- the larger-capacity question Sec. 5 leaves open, on
    synthetic data.  Every network takes the same SGD step: the first one's
    (lr_scale / its first loss, unless lr is given), since a deeper He-initialised
    network starts from a larger loss and a step relative to it would be smaller."""
    lr = kw.pop("lr", None)
    out = []
    for h in hiddens:
        r = train_and_evaluate(n, ratio, hidden=h, lr=lr, **kw)
        lr = r["lr"]
        out.append(r)
    return out
