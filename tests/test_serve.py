"""Continuous-batching server (deepinv_serve_*): results equal the network run
alone, admission respects the HBM budget, bounded waits, bad requests."""
import numpy as np
import pytest

import oracle
from paper_1701_03891_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def di():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    return deepinv


SHAPES = [(16, 16, 0.125), (32, 32, 0.10), (24, 40, 0.20)]


def _nets(di, prec="bf16", hidden=(0, 0, 0)):
    out = []
    for i, (n1, n2, r) in enumerate(SHAPES):
        N = n1 * n2
        M = synth.m_for_ratio(r, N)
        phi = synth.gaussian_phi(M, N, seed=10 + i)
        p = synth.he_params(seed=20 + i, bias_std=0.01, hidden=hidden[i])
        out.append((di.Net(phi, p, n1, n2, prec=prec), phi, p, n1, n2))
    return out


def _requests(nets, count, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for t in range(count):
        k = int(rng.integers(0, len(nets)))
        net, phi, p, n1, n2 = nets[k]
        x = synth.dct_sparse_images(1, n1, n2, K=8, seed=1000 + t)
        y = np.ascontiguousarray(oracle.measure(phi, x)[0], dtype=np.float32)
        reqs.append((k, y, np.full(n1 * n2, np.nan, dtype=np.float32), t))
    return reqs


def _drain(srv, n_expected, first=()):
    got = {}
    rc, res = srv.serve(list(first), timeout_us=200000)
    for r in res:
        got[r.tag] = r
    tries = 0
    while len(got) < n_expected and tries < 200:
        rc, res = srv.serve([], timeout_us=200000)
        for r in res:
            got[r.tag] = r
        tries += 1
    return got


@pytest.mark.parametrize("prec,hidden", [("bf16", (0, 0, 0)), ("f32", (0, 0, 0)), ("bf16", (0, 1, 2))])
def test_mixed_stream_equals_alone(di, prec, hidden):
    """Requests of three networks (the last case mixes 3-, 4- and 5-layer
    networks) give the same bits batched in the mix as alone."""
    import torch
    nets = _nets(di, prec, hidden)
    srv = di.Server(hbm_budget_bytes=4 << 30, max_streams=4, max_batch=8)
    ids = [srv.add(n[0]) for n in nets]
    assert ids == [0, 1, 2]
    reqs = _requests(nets, 60)
    # submit in three waves so that later requests join while earlier batches run
    got = {}
    for w in range(3):
        rc, res = srv.serve(reqs[w * 20:(w + 1) * 20], timeout_us=0)
        for r in res:
            got[r.tag] = r
    got.update(_drain(srv, 60))
    assert len(got) == 60 and all(r.status == 0 for r in got.values())
    st = srv.stats()
    srv.close()
    assert st["completed"] == 60 and st["batches"] < 60      # requests were batched
    for k, y, xh, t in reqs:
        net = nets[k][0]
        alone = net.forward(torch.from_numpy(y[None]).cuda()).cpu().numpy()[0]
        np.testing.assert_array_equal(xh, alone)              # same bits alone and in the mix
    # and within the precision's tolerance of the FP64 oracle
    k, y, xh, t = reqs[0]
    _, phi, p, n1, n2 = nets[k]
    ref = oracle.forward(y[None], p, n1, n2, phi=phi)
    assert float(oracle.rel_l2(xh[None], ref)[0]) <= (1e-2 if prec == "bf16" else 1e-5)


def test_large_batches_parallel_copies(di):
    """Batches of up to 128 requests of 64 x 64 and 128 x 128 networks, whose
    staging and result copies the server splits between its threads: every result
    lands in its own buffer, bit-identical to the network run alone."""
    import torch
    nets = []
    for i, (n, r) in enumerate([(128, 0.10), (64, 0.25)]):
        N = n * n
        phi = synth.gaussian_phi(synth.m_for_ratio(r, N), N, seed=40 + i)
        p = synth.he_params(seed=50 + i, bias_std=0.01)
        nets.append((di.Net(phi, p, n, n, prec="bf16"), phi, p, n, n))
    srv = di.Server(hbm_budget_bytes=8 << 30, max_streams=2, max_batch=128)
    for n in nets:
        srv.add(n[0])
    rng = np.random.default_rng(3)
    reqs = []
    for t in range(400):
        k = int(rng.integers(0, 2))
        net, phi, p, n1, n2 = nets[k]
        y = rng.standard_normal(phi.shape[0]).astype(np.float32)
        reqs.append((k, y, np.full(n1 * n2, np.nan, dtype=np.float32), t))
    got = _drain(srv, len(reqs), first=reqs)
    st = srv.stats()
    srv.close()
    assert len(got) == len(reqs) and all(r.status == 0 for r in got.values())
    assert max(r.batch for r in got.values()) > 64          # large batches were formed
    assert st["batches"] < len(reqs) // 8
    for k in range(2):
        mine = [q for q in reqs if q[0] == k]
        ys = torch.from_numpy(np.stack([q[1] for q in mine])).cuda()
        alone = nets[k][0].forward(ys).cpu().numpy()
        for j, (_, y, xh, t) in enumerate(mine):
            np.testing.assert_array_equal(xh, alone[j])


def test_admission_under_tight_budget(di):
    """A budget that holds the largest workspace but not two of them: every request
    still finishes, the workspaces held never exceed the budget, batches wait for
    room, and idle workspaces of other networks are released."""
    nets = _nets(di)
    leases = []
    for n in nets:                                  # workspace size of each network alone
        probe = di.Server(hbm_budget_bytes=1 << 40, max_streams=1, max_batch=4)
        probe.add(n[0])
        k = nets.index(n)
        _drain(probe, 1, [r for r in _requests([n], 1, seed=9)])
        leases.append(probe.stats()["peak_workspace_bytes"])
        probe.close()
    budget = max(leases) + 1                        # the largest fits, no two of the largest do
    srv = di.Server(hbm_budget_bytes=budget, max_streams=4, max_batch=4)
    for n in nets:
        srv.add(n[0])
    reqs = _requests(nets, 24, seed=2)
    got = _drain(srv, 24, reqs)
    st = srv.stats()
    srv.close()
    assert len(got) == 24 and all(r.status == 0 for r in got.values())
    assert st["peak_workspace_bytes"] <= budget
    assert st["max_in_flight"] < 4                  # the budget, not the 4 streams, limited concurrency
    assert st["evictions"] > 0 and st["admission_waits"] > 0


def test_budget_too_small_fails_requests(di):
    from paper_1701_03891_gb300 import deepinv
    nets = _nets(di)
    srv = di.Server(hbm_budget_bytes=1024, max_streams=2, max_batch=4)
    for n in nets:
        srv.add(n[0])
    reqs = _requests(nets, 5, seed=3)
    got = _drain(srv, 5, reqs)
    srv.close()
    assert len(got) == 5 and all(r.status == deepinv.ENOMEM for r in got.values())


def test_bounded_wait_and_bad_request(di):
    """A harvest with nothing finished returns DEEPINV_ETIMEOUT after its bounded
    wait; a request for an unknown network is rejected before submission."""
    from paper_1701_03891_gb300 import deepinv
    n1 = n2 = 128
    N = n1 * n2
    M = synth.m_for_ratio(0.05, N)
    net = di.Net(synth.gaussian_phi(M, N, seed=3), synth.he_params(seed=4), n1, n2, prec="bf16")
    srv = di.Server(hbm_budget_bytes=16 << 30, max_streams=1, max_batch=512)
    srv.add(net)
    rc, res = srv.serve([], timeout_us=1000)           # nothing pending: returns at once
    assert rc == deepinv.OK and res == []
    rng = np.random.default_rng(5)
    reqs = [(0, rng.standard_normal(M).astype(np.float32), np.empty(N, np.float32), t) for t in range(512)]
    # one batch of 512 recoveries of 128 x 128 images takes milliseconds
    rc, res = srv.serve(reqs, timeout_us=200)
    assert rc == deepinv.ETIMEOUT and res == []
    got = _drain(srv, 512)
    assert len(got) == 512 and all(r.status == 0 for r in got.values())
    assert max(r.batch for r in got.values()) > 1
    bad = [(7, reqs[0][1], reqs[0][2], 99)]
    with pytest.raises(deepinv.DeepInvError):
        srv.serve(bad)
    srv.close()
