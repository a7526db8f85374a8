"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 per image, max over the batch):
  float32 path  <= 1e-5   (float32 products, float32 accumulation), and every
                 pixel within 8e-5 of the image's rms (8 standard deviations
                 of an error of 1e-5 rms);
  bfloat16 path <= 1e-2   (the stated bound), and the tighter gates of
                 tests/_precision.py: within 0.75 of the bfloat16 rounding floor
                 of the rounded-operand oracle (oracle/rounded.py), within
                 1.25 floors of the exact oracle, every pixel and every
                 gradient element checked.
The exact oracle sees the float32 master weights and inputs, so its distance
includes the rounding of weights, inputs and activations: the floor.
"""
import numpy as np
import pytest

import oracle
from oracle import rounded
from paper_1701_03891_gb300 import synth
from _precision import ELEMENT_FACTOR, check_images, check_tensors

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 1e-2}


def _check_f32(got, ref):
    """float32 path: rel-L2 per image and every pixel against the image's rms."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    B = got.shape[0]
    assert np.all(np.isfinite(got))
    assert _maxrel(got, ref) <= TOL["f32"]
    r = ref.reshape(B, -1)
    rms = np.sqrt(np.mean(r * r, axis=1, keepdims=True))
    assert float(np.max(np.abs(got.reshape(B, -1) - r) / rms)) <= 8 * TOL["f32"]


def _check_sense_recover(xhat, phi, params, x, n1, n2, prec, **kw):
    """x^ of the path's own y = Phi x against the exact oracle, and for bf16 against
    the rounded-operand oracle fed by the bf16 measurement."""
    ref = oracle.forward(oracle.measure(phi, x), params, n1, n2, phi=phi, **kw)
    if prec == "f32":
        _check_f32(xhat, ref)
        return
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x), params, n1, n2, phi=phi, **kw)
    check_images(xhat, ref, rnd, what=(n1, n2))
    assert _maxrel(xhat, ref) <= TOL["bf16"]


@pytest.fixture(scope="module")
def di():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    deepinv.lib()
    return deepinv


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _maxrel(got, ref):
    return float(np.max(oracle.rel_l2(got, ref)))


# ------------------------------------------------------------------ y = Phi x
@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("M,N,B", [(13, 37, 5), (102, 1024, 4), (410, 4096, 130), (1, 16, 1), (300, 300, 257)])
def test_measure(di, prec, M, N, B):
    rng = np.random.default_rng(M * 7 + N)
    phi = synth.gaussian_phi(M, N, seed=M)
    x = rng.uniform(0, 1, (B, N)).astype(np.float32)
    y = di.measure(_cuda(phi), _cuda(x), prec=prec).cpu().numpy()
    ref = oracle.measure(phi, x)
    assert _maxrel(y, ref) <= TOL[prec]


def test_measure_empty_batch(di):
    import torch
    phi = _cuda(synth.gaussian_phi(8, 32))
    x = torch.empty((0, 32), device="cuda")
    assert di.measure(phi, x, prec="bf16").shape == (0, 8)


# ------------------------------------------------------------------ forward
def _case(n1, n2, ratio, B, seed=0, images="dct", bias_std=0.01):
    N = n1 * n2
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=seed)
    params = synth.he_params(seed=seed + 1, bias_std=bias_std)
    if images == "dct":
        x = synth.dct_sparse_images(B, n1, n2, K=max(1, N // 20), seed=seed + 2)
    else:
        x = synth.voronoi_images(B, n1, n2, seed=seed + 3)
    return phi, params, x


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("n1,n2,ratio,B", [
    (32, 32, 0.10, 4),      # the 32 x 32 float32 parity workload
    (64, 64, 0.25, 3),
    (64, 64, 0.10, 3),
    (64, 64, 0.05, 3),
    (16, 16, 0.125, 2),
    (24, 40, 0.10, 3),      # non-square
    (20, 37, 0.20, 2),      # ragged width
    (7, 9, 0.5, 5),         # tiny image: one tile, most of it padding
])
def test_forward(di, prec, n1, n2, ratio, B):
    phi, params, x = _case(n1, n2, ratio, B)
    net = di.Net(phi, params, n1, n2, prec=prec)
    xd = _cuda(x)
    y = net.measure(xd)
    xhat = net.forward(y).cpu().numpy()
    _check_sense_recover(xhat, phi, params, x, n1, n2, prec)
    net.close()


@pytest.mark.parametrize("n1,n2,ratio,B", [
    (128, 128, 0.05, 2),    # wide images: conv2 streams per-kernel-row pieces
    (90, 100, 0.10, 2),
    (256, 256, 0.01, 1),
])
def test_forward_bf16_wide(di, n1, n2, ratio, B):
    phi, params, x = _case(n1, n2, ratio, B)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    xhat = net.forward(y).cpu().numpy()
    _check_sense_recover(xhat, phi, params, x, n1, n2, "bf16")


def test_gemm_two_row_tiles_odd_counts(di):
    """GEMMs with a large B operand take two 128-row tiles per CTA; with an odd
    tile count the last CTA has one.  Measurement: Phi 520 x 65536 (68 MB) and
    260 images = 3 row tiles; FC layer: a 200 x 200 image = 313 pixel tiles."""
    rng = np.random.default_rng(21)
    N, M, B = 256 * 256, 520, 260
    phi = synth.gaussian_phi(M, N, seed=21)
    x = rng.uniform(0, 1, (B, N)).astype(np.float32)
    net = di.Net(phi, synth.he_params(seed=1), 256, 256, prec="bf16")
    y = net.measure(_cuda(x)).cpu().numpy()
    assert _maxrel(y, oracle.measure(phi, x)) <= TOL["bf16"]
    net.close()
    phi2, params, x2 = _case(200, 200, 0.02, 2, seed=4)
    net2 = di.Net(phi2, params, 200, 200, prec="bf16")
    y2 = oracle.measure(phi2, x2)
    ref = oracle.forward(y2, params, 200, 200, phi=phi2)
    rnd = rounded.forward_bf16(rounded.f32(y2), params, 200, 200, phi=phi2)
    check_images(net2.forward(_cuda(y2)).cpu().numpy(), ref, rnd, what="FC 313 pixel tiles")


@pytest.mark.parametrize("n1,n2,ratio,B", [
    (6, 119, 0.10, 2),      # pitch 124: conv3 keeps row sums in its shared-memory ring
    (6, 120, 0.10, 2),      # pitch 125: conv3 keeps partial outputs instead
    (1, 4960, 0.10, 2),     # too wide for either ring: row sums through global scratch
])
def test_forward_bf16_conv3_modes(di, n1, n2, ratio, B):
    phi, params, x = _case(n1, n2, ratio, B)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(_cuda(x))
    xhat = net.forward(y).cpu().numpy()
    _check_sense_recover(xhat, phi, params, x, n1, n2, "bf16")


@pytest.mark.parametrize("n1,n2,M,B", [
    (4, 130, 52, 2),        # pitch 135: conv1's input gradient in the partial-output ring
    (1, 4250, 425, 2),      # too wide for the 64-channel ring: global row-sum scratch
    (72, 120, 864, 2),      # 71 tiles of 128 per image: conv1 and conv3's input gradient
                            # read their expanded input from the window ring
])
def test_backward_bf16_wide_train_fc(di, n1, n2, M, B):
    """bf16 backward with the FC layer trained (conv1's input gradient runs through
    the fused conv3 kernel over 64 channels) on wide images."""
    N = n1 * n2
    phi = synth.gaussian_phi(M, N, seed=7)
    params = synth.he_params(seed=8, bias_std=0.02)
    x = synth.dct_sparse_images(B, n1, n2, K=max(4, N // 40), seed=9)
    y = oracle.measure(phi, x).astype(np.float32)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi, train_fc=True)
    net = di.Net(phi, params, n1, n2, prec="bf16", train_fc=True)
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)
    loss, dW, db, dWfc = net.backward(yd, xd, saved)
    _check_bf16_grads(loss, dW, db, dWfc, y, x, params, n1, n2, phi, True, loss_ref, g)


def test_backward_bf16_multi_image_ranges_deterministic(di):
    """Training backward on a batch whose per-CTA tile ranges cross image boundaries
    (72 x 120: 71 conv1 tiles per image, conv1's and conv3's input-gradient window
    rings; conv3's partial-output ring): three passes bit for bit, and the
    gradients against the float32 path's (an independent set of kernels) within
    the bfloat16 gradient floor's range (rel-L2 <= 1.25 x 3.6e-2 per tensor: the
    kernel margin over the largest per-tensor floor of the seeded networks)."""
    n1, n2, B = 72, 120, 8
    N = n1 * n2
    M = synth.m_for_ratio(0.10, N)
    phi = synth.gaussian_phi(M, N, seed=7)
    params = synth.he_params(seed=8, bias_std=0.02)
    x = synth.voronoi_images(B, n1, n2, seed=9)
    yd, xd = _cuda(oracle.measure(phi, x)), _cuda(x)
    grads = {}
    for prec in ("bf16", "f32"):
        net = di.Net(phi, params, n1, n2, prec=prec, train_fc=True)
        saved = net.new_saved(B)
        runs = []
        for _ in range(3 if prec == "bf16" else 1):
            net.forward(yd, saved=saved)
            loss, dW, db, dWfc = net.backward(yd, xd, saved)
            runs.append([t.cpu().numpy() for t in list(dW) + list(db) + [dWfc, loss]])
        for r in runs[1:]:
            for a, b in zip(r, runs[0]):
                np.testing.assert_array_equal(a, b)
        grads[prec] = runs[0]
        net.close()
    for a, b in zip(grads["bf16"], grads["f32"]):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1.25 * 3.6e-2 * max(np.linalg.norm(b), 1e-30), (
            np.linalg.norm(a - b) / np.linalg.norm(b))


def test_conv2_row_mode_matches_window_mode(di, tmp_path):
    """Both conv2 pipelines (window slabs vs per-row pieces) give identical bits."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys; sys.path.insert(0, %r);"
        "from paper_1701_03891_gb300 import deepinv, synth;"
        "phi = synth.gaussian_phi(410, 4096, 0); p = synth.he_params(seed=1, bias_std=0.01);"
        "x = synth.voronoi_images(8, 64, 64, seed=5);"
        "net = deepinv.Net(phi, p, 64, 64, prec='bf16');"
        "y = net.measure(torch.from_numpy(x).cuda()); out = net.forward(y).cpu().numpy();"
        "np.save(sys.argv[1], out)" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    outs = []
    for window in ("0", "1"):
        f = str(tmp_path / ("xhat_window%s.npy" % window))
        env = dict(os.environ, DEEPINV_CONV2_WINDOW=window)
        subprocess.check_call([sys.executable, "-c", code, f], env=env)
        outs.append(np.load(f))
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_forward_final_relu(di, prec):
    phi, params, x = _case(32, 32, 0.1, 3)
    net = di.Net(phi, params, 32, 32, prec=prec, final_relu=True)
    y = rounded.f32(oracle.measure(phi, x))
    xhat = net.forward(_cuda(y)).cpu().numpy()
    ref = oracle.forward(y, params, 32, 32, phi=phi, final_relu=True)
    assert np.all(xhat >= 0)
    assert float(np.linalg.norm(xhat - ref) / np.linalg.norm(ref)) <= TOL[prec]
    if prec == "bf16":
        check_images(xhat, ref, rounded.forward_bf16(y, params, 32, 32, phi=phi, final_relu=True), what="final ReLU")


def test_forward_f32_reduced_net(di):
    """The float32 path takes any filter counts and odd kernel sizes."""
    n1, n2, M, B = 13, 19, 30, 3
    phi = synth.gaussian_phi(M, n1 * n2, seed=5)
    params = synth.he_params(5, 3, 1, 5, seed=6, bias_std=0.1)
    x = synth.dct_sparse_images(B, n1, n2, K=12, seed=7)
    net = di.Net(phi, params, n1, n2, prec="f32")
    y = _cuda(oracle.measure(phi, x))
    got = net.forward(y).cpu().numpy()
    ref = oracle.forward(y.cpu().numpy(), params, n1, n2, phi=phi)
    assert _maxrel(got, ref) <= TOL["f32"]


def test_forward_bf16_full_batch_sampled(di):
    """64 x 64, M/N = 0.1, batch 1024 (the benchmark workload, in its launch
    configuration).  Every image of the bf16 result against the float32 path's
    (an independent set of kernels, itself held to 1e-5 of the oracle on sampled
    images here); 24 sampled images against the exact and the rounded-operand
    oracle; and batch invariance."""
    n1 = n2 = 64
    B = 1024
    phi, params, x = _case(n1, n2, 0.10, B, images="voronoi", bias_std=0.0)
    xd = _cuda(x)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    y = net.measure(xd)
    xhat = net.forward(y).cpu().numpy()
    netf = di.Net(phi, params, n1, n2, prec="f32")
    xf = netf.forward(netf.measure(xd)).cpu().numpy()
    netf.close()
    assert np.all(np.isfinite(xhat)) and np.all(np.isfinite(xf))
    idx = np.r_[0, 1, 511, 777, 1023, np.random.default_rng(30).choice(np.arange(2, 1023), 19, replace=False)]
    ref = oracle.forward(oracle.measure(phi, x[idx]), params, n1, n2, phi=phi)
    _check_f32(xf[idx], ref)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[idx]), params, n1, n2, phi=phi)
    floor, _ = check_images(xhat[idx], ref, rnd, what="batch 1024, sampled")
    # all 1024 images against the float32 path: the stated bound; the floor's margin
    # (the float32 path is the exact oracle to 1e-5, and these images' floors match
    # the sampled ones' to a few per cent, so 1.25 * 1.1 floors); every image's worst
    # pixel within ELEMENT_FACTOR of the sampled images' worst rounding deviation
    allrel = oracle.rel_l2(xhat, xf)
    assert float(allrel.max()) <= TOL["bf16"]
    assert float(allrel.max()) <= 1.25 * 1.1 * floor, (float(allrel.max()), floor)
    worst_format = float(np.max(np.abs(rnd - ref)))
    assert float(np.max(np.abs(xhat - xf))) <= ELEMENT_FACTOR * 1.1 * worst_format
    # batch invariance: the same images alone give the same result
    alone = net.forward(y[idx[:5]].contiguous()).cpu().numpy()
    np.testing.assert_allclose(alone, xhat[idx[:5]], rtol=0, atol=1e-6 * np.abs(xhat[idx[:5]]).max())
    net.close()


@pytest.mark.parametrize("n,B", [(256, 32), (128, 48), (64, 512)])
def test_forward_bf16_multi_image_ranges_deterministic(di, n, B):
    """Batches whose per-CTA tile ranges cross many image boundaries, in both of
    conv3's ring modes (pitch >= 125: one partial sum per pending output; < 125:
    row sums) and with conv1's window ring: every image against the float32 path
    (an independent set of kernels), two sampled images against the oracle, and
    three repeated passes bit for bit (a race between the tiles of a CTA shows up
    as a difference)."""
    phi, params, x = _case(n, n, 0.10, B, images="voronoi", bias_std=0.01)
    xd = _cuda(x)
    net = di.Net(phi, params, n, n, prec="bf16")
    y = net.measure(xd)
    runs = [net.forward(y).cpu().numpy() for _ in range(3)]
    for r in runs[1:]:
        np.testing.assert_array_equal(r, runs[0])
    xhat = runs[0]
    netf = di.Net(phi, params, n, n, prec="f32")
    xf = netf.forward(netf.measure(xd)).cpu().numpy()
    netf.close()
    idx = np.array([0, B - 1])
    ref = oracle.forward(oracle.measure(phi, x[idx]), params, n, n, phi=phi)
    rnd = rounded.forward_bf16(rounded.measure_bf16(phi, x[idx]), params, n, n, phi=phi)
    floor, _ = check_images(xhat[idx], ref, rnd, what=("multi-image", n, B))
    allrel = oracle.rel_l2(xhat, xf)
    assert float(allrel.max()) <= TOL["bf16"], (n, B, float(allrel.max()), int(np.argmax(allrel)))
    assert float(allrel.max()) <= 1.25 * 1.25 * floor, (n, B, float(allrel.max()), floor)
    net.close()


def test_forward_batch_sizes_reuse_workspace(di):
    """Growing and shrinking the batch on one network keeps results exact (zero borders preserved)."""
    phi, params, x = _case(32, 32, 0.1, 40)
    net = di.Net(phi, params, 32, 32, prec="bf16")
    y = _cuda(oracle.measure(phi, x))
    full = net.forward(y).cpu().numpy()
    for b in (1, 7, 40, 3):
        part = net.forward(y[:b].contiguous()).cpu().numpy()
        np.testing.assert_array_equal(part, full[:b])


def test_forward_empty_batch(di):
    import torch
    phi, params, _ = _case(16, 16, 0.125, 1)
    net = di.Net(phi, params, 16, 16, prec="bf16")
    out = net.forward(torch.empty((0, phi.shape[0]), device="cuda"))
    assert out.shape == (0, 256)


def test_host_entry_points(di):
    import torch
    phi, params, x = _case(32, 32, 0.1, 6)
    for prec in ("f32", "bf16"):
        net = di.Net(phi, params, 32, 32, prec=prec)
        xd = _cuda(x)
        y = net.measure(xd)
        dev = net.forward(y).cpu()
        yh = y.cpu().pin_memory()
        host = net.forward_host(yh, torch.empty((6, 1024)).pin_memory())
        assert torch.equal(host, dev)
        sr = net.sense_recover_host(torch.from_numpy(x).pin_memory(), torch.empty((6, 1024)).pin_memory())
        assert torch.equal(sr, dev)


def test_host_submit_overlapped_batches(di):
    """deepinv_sense_recover_host_submit with up to three batches queued (both
    staging slots in use and one reused) gives the same bits as the synchronous
    call for every batch, and host_wait of an older ticket returns too."""
    import torch
    n1 = n2 = 32
    phi, params, x = _case(n1, n2, 0.1, 300, seed=3)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    parts = [torch.from_numpy(x[i * 100:(i + 1) * 100]).pin_memory() for i in range(3)]
    want = [net.sense_recover_host(p, torch.empty((100, n1 * n2)).pin_memory()).clone() for p in parts]
    outs = [torch.full((100, n1 * n2), float("nan")).pin_memory() for _ in range(3)]
    tickets = [net.sense_recover_host_submit(p, o) for p, o in zip(parts, outs)]
    assert tickets == sorted(tickets) and len(set(tickets)) == 3
    net.host_wait(tickets[0])
    assert torch.equal(outs[0], want[0])
    net.host_wait(tickets[2])
    for o, w in zip(outs, want):
        assert torch.equal(o, w)
    ref = oracle.forward(oracle.measure(phi, x[:8]), params, n1, n2, phi=phi)
    assert _maxrel(outs[0][:8].numpy(), ref) <= TOL["bf16"]
    net.close()


# ------------------------------------------------------------------ backward
def _train_case(train_fc):
    n1 = n2 = 16
    M, B = 32, 2
    phi = synth.gaussian_phi(M, n1 * n2, seed=0)
    params = synth.he_params(seed=1, bias_std=0.05)
    x = synth.dct_sparse_images(B, n1, n2, K=10, seed=2)
    y = oracle.measure(phi, x).astype(np.float32)
    return n1, n2, phi, params, x, y


def _grad_dict(dW, db, dWfc):
    got = {}
    for i in range(len(dW)):
        got["w%d" % (i + 1)] = dW[i].cpu().numpy()
        got["b%d" % (i + 1)] = db[i].cpu().numpy()
    if dWfc is not None:
        got["wfc"] = dWfc.cpu().numpy()
    return got


def _check_bf16_grads(loss, dW, db, dWfc, y, x, params, n1, n2, phi, train_fc, loss_ref, g):
    """bf16 gradients against the exact oracle's and the rounded-operand oracle's
    (tests/_precision.py); the loss within the bfloat16 floor of the loss."""
    loss_rnd, g_rnd = rounded.backward_bf16(y, x, params, n1, n2, phi=phi, train_fc=train_fc)
    check_tensors(_grad_dict(dW, db, dWfc if train_fc else None), g, g_rnd, what=(n1, n2))
    floor = abs(loss_rnd - loss_ref) / abs(loss_ref)
    assert abs(float(loss) - loss_rnd) <= 0.75 * floor * abs(loss_ref) + 1e-6 * abs(loss_ref)
    assert abs(float(loss) - loss_ref) <= 1.25 * floor * abs(loss_ref) + 1e-6 * abs(loss_ref)


@pytest.mark.parametrize("prec,train_fc", [("f32", False), ("f32", True), ("bf16", False), ("bf16", True)])
def test_backward_matches_oracle(di, prec, train_fc):
    n1, n2, phi, params, x, y = _train_case(train_fc)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi, train_fc=train_fc)
    net = di.Net(phi, params, n1, n2, prec=prec, train_fc=train_fc)
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(2)
    net.forward(yd, saved=saved)
    loss, dW, db, dWfc = net.backward(yd, xd, saved)
    if prec == "bf16":
        _check_bf16_grads(loss, dW, db, dWfc, y, x, params, n1, n2, phi, train_fc, loss_ref, g)
        return
    tol = 1e-4
    assert abs(float(loss) - loss_ref) <= 1e-6 * abs(loss_ref)
    for i in range(3):
        for name, got in (("w%d" % (i + 1), dW[i]), ("b%d" % (i + 1), db[i])):
            ref = g[name]
            err = float(np.linalg.norm(got.cpu().numpy() - ref) / max(np.linalg.norm(ref), 1e-30))
            assert err <= tol, (name, err)
    if train_fc:
        err = float(np.linalg.norm(dWfc.cpu().numpy() - g["wfc"]) / np.linalg.norm(g["wfc"]))
        assert err <= tol, ("wfc", err)


@pytest.mark.parametrize("n1,n2,M,B", [(32, 32, 102, 3), (24, 40, 96, 2), (64, 64, 410, 2), (20, 37, 74, 2)])
def test_backward_bf16_shapes(di, n1, n2, M, B):
    """bf16 backward (tensor-core conv2/conv3 input gradients and conv2 weight
    gradient) against the FP64 oracle on several image shapes."""
    N = n1 * n2
    phi = synth.gaussian_phi(M, N, seed=4)
    params = synth.he_params(seed=5, bias_std=0.02)
    x = synth.dct_sparse_images(B, n1, n2, K=max(4, N // 40), seed=6)
    y = oracle.measure(phi, x).astype(np.float32)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi)
    net = di.Net(phi, params, n1, n2, prec="bf16")
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)
    loss, dW, db, _ = net.backward(yd, xd, saved)
    _check_bf16_grads(loss, dW, db, None, y, x, params, n1, n2, phi, False, loss_ref, g)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_backward_recompute(di, prec):
    """backward without a saved buffer recomputes the activations: with no budget
    (one chunk) it is bit-identical to the saved path; with a budget of three
    images' activations it runs three chunks (3 + 3 + 1) whose gradients agree
    with the saved path up to summation order, and with the oracle."""
    n1 = n2 = 24
    N, M, B = n1 * n2, 144, 7
    phi = synth.gaussian_phi(M, N, seed=10)
    params = synth.he_params(seed=11, bias_std=0.02)
    x = synth.dct_sparse_images(B, n1, n2, K=20, seed=12)
    y = oracle.measure(phi, x).astype(np.float32)
    net = di.Net(phi, params, n1, n2, prec=prec, train_fc=True)
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(B)
    net.forward(yd, saved=saved)
    ref = [t.clone() if t is not None else None for t in _flat(net.backward(yd, xd, saved))]
    one = _flat(net.backward(yd, xd))                            # recompute, one chunk
    for a, b in zip(ref, one):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    net.set_act_budget(3 * net.saved_bytes(1) + 4096)            # chunks of 3 images
    assert net.saved_bytes(3) <= 3 * net.saved_bytes(1) + 4096 < net.saved_bytes(4)
    chunked = _flat(net.backward(yd, xd))
    for a, b in zip(ref, chunked):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(a), 1e-30)
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi, train_fc=True)
    names = ["loss", "w1", "w2", "w3", "b1", "b2", "b3", "wfc"]
    if prec == "bf16":
        c = dict(zip(names, chunked))
        _check_bf16_grads(c["loss"], [c["w1"], c["w2"], c["w3"]], [c["b1"], c["b2"], c["b3"]], c["wfc"],
                          y, x, params, n1, n2, phi, True, loss_ref, g)
    else:
        for name, got in zip(names, chunked):
            want = loss_ref if name == "loss" else g[name]
            got = got.cpu().numpy()
            err = float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30))
            assert err <= 1e-4, (name, err)
    net.close()


def _flat(res):
    loss, dW, db, dWfc = res
    return [loss] + list(dW) + list(db) + [dWfc]


def test_sgd_momentum_step(di):
    n1, n2, phi, params, x, y = _train_case(False)
    net = di.Net(phi, params, n1, n2, prec="f32")
    yd, xd = _cuda(y), _cuda(x)
    saved = net.new_saved(2)
    p = {k: v.astype(np.float64) for k, v in params.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    for step in range(2):
        net.forward(yd, saved=saved)
        loss, dW, db, _ = net.backward(yd, xd, saved)
        net.sgd_momentum(dW, db, lr=1e-2, mu=0.9)
        for i in range(3):
            for name, gg in (("w%d" % (i + 1), dW[i]), ("b%d" % (i + 1), db[i])):
                p[name], v[name] = oracle.sgd_momentum(p[name], v[name], gg.cpu().numpy(), 1e-2, 0.9)
    got = net.get_params()
    for k in p:
        np.testing.assert_allclose(got[k].cpu().numpy(), p[k], rtol=1e-5, atol=1e-7)


def test_autograd_function(di):
    import torch
    n1, n2, phi, params, x, y = _train_case(False)
    net = di.Net(phi, params, n1, n2, prec="f32")
    ps = [torch.tensor(params[k], requires_grad=True, device="cuda")
          for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
    loss = di.mse_loss(net, _cuda(y), _cuda(x), ps)
    loss.backward()
    loss_ref, g = oracle.backward(y, x, params, n1, n2, phi=phi)
    assert abs(float(loss.detach()) - loss_ref) <= 1e-5 * loss_ref
    err = np.linalg.norm(ps[2].grad.cpu().numpy() - g["w2"]) / np.linalg.norm(g["w2"])
    assert err <= 1e-4


def test_bounded_wait_timeout_reported_and_context_usable(di):
    """A wait that nothing satisfies runs out (about 1 s), the kernel returns, the
    host reads DEEPINV_ETIMEOUT from the status word, and after the reset the
    device keeps computing correct results."""
    import time
    assert di.device_status(reset=True) == 0
    t0 = time.perf_counter()
    di.selftest_bounded_wait()
    assert time.perf_counter() - t0 >= 0.9
    assert di.device_status(reset=True) == di.ETIMEOUT
    assert di.device_status() == 0
    phi, params, x = _case(32, 32, 0.1, 2)
    net = di.Net(phi, params, 32, 32, prec="bf16")
    y = _cuda(oracle.measure(phi, x))
    ref = oracle.forward(y.cpu().numpy(), params, 32, 32, phi=phi)
    assert _maxrel(net.forward(y).cpu().numpy(), ref) <= TOL["bf16"]
    assert di.device_status() == 0


def test_device_status_clean(di):
    assert di.device_status() == 0
