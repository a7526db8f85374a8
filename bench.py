#!/usr/bin/env python
"""DeepInverse recovery throughput on GB300 (images/s), one JSON line.

Workload: 64 x 64 images (N = 4096), M/N = 0.1 (M = 410), batch 1024 per GPU,
the paper's network (FC = Phi^T, then 64 / 32 / 1 filters of 11 x 11, Sec. 4-5),
seeded synthetic piecewise-smooth images standing in for the 64 x 64 ImageNet
crops of Sec. 5.  One step = sense and recover one batch: y = Phi x, then
x^ = M(y, Omega), on the bfloat16 tensor-core path (float32 accumulation).

Also reported: per-stage and per-step times, the conv2 roofline fraction and
DRAM traffic, the float32 CUDA-core path on the same batch (images/s and the
rel-L2 between the two paths), the end-to-end rate through the host-memory
entry points (two batches in flight, and one at a time), continuous-batching
serving latency, 256 x 256 bf16 and e4m3 recovery, a training step, a
five-layer network (inference and training), the clocks seen during the timed
region, and the FP64 CPU oracle's rate on a bounded sample of the batch (with
the host's thread count and CPU model);
--eval adds recovery quality of networks trained by the library.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank recovers its own batch (weak scaling, no
collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "images/s at 64x64, M/N=0.1: BF16 vs FP32 at rel-L2<=1e-2; serving p50/p99 ms"
CONV2_MAC_PER_PX = 64 * 32 * 121
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=64)
    ap.add_argument("--ratio", type=float, default=0.10)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-deep", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-ratios", action="store_true")
    ap.add_argument("--conv1-rows", type=int, default=1, choices=[0, 1, 2],
                    help="conv1 kernel of the headline network: 0 position tiles, 1 row tiles where "
                         "faster (the library default), 2 row tiles wherever they fit")
    ap.add_argument("--fused-steps", type=int, default=20)
    ap.add_argument("--deep-steps", type=int, default=10)
    ap.add_argument("--train-steps", type=int, default=10)
    ap.add_argument("--large-steps", type=int, default=10)
    ap.add_argument("--serve-rates", default="20000,50000,100000,200000,400000,800000",
                    help="offered request rates (requests/s) of the serving sweep, log-spaced up to past saturation")
    ap.add_argument("--serve-seconds", type=float, default=0.5, help="arrival window per rate")
    ap.add_argument("--eval", action="store_true",
                    help="also train 32x32 networks at M/N 0.05/0.10/0.25, clean and 20 dB SNR, and report "
                         "the recovered images' PSNR and success rate, 3-, 4- and 5-layer networks at M/N 0.10, and a 64x64 convergence curve (about a minute)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sust=float(d["bf16_tflops_sustained"]), src="measured",
                    sust_mhz=(d.get("clocks_under_load") or {}).get("sm_mhz_median"))
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sust=1700.0, src="fallback", sust_mhz=None)


class Clocks:
    """nvidia-smi sampler (200 ms) around the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            self.f.close()
            os.unlink(self.f.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(dev_ms, per_rank_batch, steps, world, dist=None, device="cpu"):
    """Whole-job throughput: every rank recovers its own batch (no collective on the data
    path); the job's time is the slowest rank's.  Returns (max ms over ranks, images/s)."""
    import torch
    t = torch.tensor([float(dev_ms)], device=device, dtype=torch.float64)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * per_rank_batch * steps / (ms / 1000.0)


def workload(args, rank=0):
    from paper_1701_03891_gb300 import synth
    n = args.size
    N = n * n
    M = synth.m_for_ratio(args.ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1)
    x = synth.voronoi_images(args.batch, n, n, seed=3 + rank)
    return n, N, M, phi, params, x


def config(args, n, M, world):
    return {"workload": "DeepInverse sense+recover %dx%d, M/N=%.2f (M=%d), batch %d per GPU, "
                        "FC=Phi^T + conv 64/32/1 @ 11x11" % (n, n, args.ratio, M, args.batch),
            "image_size": n, "M": M, "global_batch": args.batch * world,
            "parallelism": "replicas (dp%d, no collective)" % world,
            "l2": "flushed (%d MiB write) before every timed step, outside its events" % (L2_FLUSH_BYTES >> 20)}


def host_cpu():
    """Model name of the host CPU (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(args, phi, params, x, n, gpu_xhat=None):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the batch."""
    import numpy as np
    import oracle
    oracle.build()
    done, t0 = 0, time.perf_counter()
    errs, dps = [], []
    chunk = 4
    while done < x.shape[0] and (time.perf_counter() - t0) < args.cpu_seconds:
        xs = x[done:done + chunk]
        ref = oracle.forward(oracle.measure(phi, xs), params, n, n, phi=phi)
        if gpu_xhat is not None:
            errs.append(oracle.rel_l2(gpu_xhat[done:done + chunk], ref))
            dps.append(np.abs(oracle.psnr(gpu_xhat[done:done + chunk], xs) - oracle.psnr(ref, xs)))
        done += xs.shape[0]
    dt = time.perf_counter() - t0
    out = {"value": done / dt, "unit": "images/s", "cores": oracle.num_threads(), "cpu": host_cpu(),
           "kind": "oracle", "sample": "%d of the %d batch images (FP64 oracle, OpenMP over output channels, %.1f s)"
                     % (done, x.shape[0], dt)}
    if errs:
        out["bf16_vs_oracle_max_rel_l2"] = float(np.max(np.concatenate(errs)))
        out["bf16_vs_oracle_max_psnr_diff_db"] = float(np.max(np.concatenate(dps)))
    return out


CONV2_SOURCES = ("tc_kernels.cu", "tc.cuh", "common.cuh")
CONV2_BEGIN = "// ---------------------------------------------------------------- conv2\n"
CONV2_END = "// ---------------------------------------------------------------- conv3\n"


def conv2_source_hash():
    """Hash of the conv2 kernel's code: its section of tc_kernels.cu and the headers it uses."""
    h = hashlib.sha256()
    for name in CONV2_SOURCES:
        with open(os.path.join(ROOT, "paper_1701_03891_gb300", "csrc", name)) as f:
            text = f.read()
        if name == "tc_kernels.cu":
            text = text[text.index(CONV2_BEGIN):text.index(CONV2_END)]
        h.update(text.encode())
    return h.hexdigest()[:16]


def traffic_record():
    """ncu DRAM bytes per conv2 image from profiles/, valid only while conv2's code is unchanged."""
    rec = os.path.join(ROOT, "profiles", "conv2_traffic.json")
    try:
        with open(rec) as f:
            d = json.load(f)
        if d.get("kernel_sha") == conv2_source_hash():
            return float(d["dram_bytes_per_image"])
    except Exception:
        pass
    return None


CONV_FLOP_PER_PX = 2 * (64 * 121 + 64 * 32 * 121 + 32 * 121)   # conv1 + conv2 + conv3 (518 848)


def algorithmic_bytes(B, n, M):
    """Minimum HBM bytes per launch of the four HBM-side stages of one step: each
    input read once and each output written once (activations bf16, planes
    counted at their n x n pixels, not their padding)."""
    N = n * n
    px = B * N
    return {"measure": 4 * px + 2 * M * N + 4 * B * M,     # x fp32 in, Phi bf16 once, y fp32 out
            "fc": 4 * B * M + 2 * M * N + 2 * px,          # y fp32 in, Phi^T bf16 once, x~ bf16 plane out
            "conv1": 2 * px + 128 * px,                    # x~ in, a1 (64 ch bf16) out
            "conv3": 64 * px + 4 * px}                     # a2 (32 ch bf16) in, x^ fp32 out


def roofline(stage_ms, B, n, M, pk, clk):
    """The dominant kernel (conv2) against the measured dense-bf16 burst peak (the
    timed region is tens of ms at full clocks); the three conv layers together
    (the target is on them); the HBM-side stages against the measured copy
    bandwidth.  Per-launch work / mean launch time from the library's own
    CUDA events on the launching stream."""
    px = B * n * n
    conv2_flop = 2.0 * CONV2_MAC_PER_PX * px
    conv2_ms = stage_ms["conv2"]
    achieved = conv2_flop / (conv2_ms / 1e3) / 1e12
    src = pk["src"]
    conv_ms = stage_ms["conv1"] + stage_ms["conv2"] + stage_ms["conv3"]
    conv_tflops = CONV_FLOP_PER_PX * px / (conv_ms / 1e3) / 1e12
    hbm = {}
    for k, nbytes in algorithmic_bytes(B, n, M).items():
        gbs = nbytes / (stage_ms[k] / 1e3) / 1e9
        hbm[k] = {"ms": stage_ms[k], "algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                  "frac": gbs / pk["hbm"]}
    dram = traffic_record()
    return {"bound": "tensor", "kernel": "conv2 (tap-stacked tcgen05 implicit GEMM)",
            "achieved": achieved, "peak": pk["bf16"], "unit": "TFLOP/s", "frac": achieved / pk["bf16"],
            "peak_note": "dense bf16 burst peak of %s (MEASURED_PEAKS.json bf16_tflops)" % src,
            "traffic": (dram * B) if dram is not None else None,
            "algorithmic_flop_per_launch": conv2_flop,
            "frac_of_sustained": achieved / pk["bf16_sust"],
            "sustained_note": "bf16_tflops_sustained of %s was taken power-capped (median %s MHz); this run's "
                              "median SM clock under load: %s MHz" % (src, pk.get("sust_mhz"), clk.get("sm_mhz")),
            "conv_layers": {"flop_per_px": CONV_FLOP_PER_PX, "ms": conv_ms, "achieved": conv_tflops,
                            "peak": pk["bf16"], "unit": "TFLOP/s", "frac": conv_tflops / pk["bf16"],
                            "note": "conv1 + conv2 + conv3 (the target: >= 0.5 of dense bf16 peak)"},
            "hbm_stages": {"peak_gbs": pk["hbm"], "peak_note": "hbm_gbs of %s" % src, "stages": hbm}}


def ratios_bench(args):
    """The 64 x 64, batch-1024 workload at the other measurement ratios of the
    batched-inference configuration (M/N = 0.25 and 0.05; 0.10 is the headline):
    sense + recover per step, L2 flushed between steps, CUDA events, stage times."""
    import torch
    from paper_1701_03891_gb300 import deepinv, synth
    n, B = 64, args.batch
    N = n * n
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    stream = torch.cuda.current_stream()
    x = synth.voronoi_images(B, n, n, seed=3)
    xd = torch.from_numpy(x).cuda()
    for ratio in (0.25, 0.05):
        M = synth.m_for_ratio(ratio, N)
        net = deepinv.Net(synth.gaussian_phi(M, N, seed=0), synth.he_params(seed=1), n, n, prec="bf16")
        net.reserve(B)
        yd = torch.empty((B, M), device="cuda")
        xh = torch.empty((B, N), device="cuda")
        for _ in range(3):
            net.measure(xd, out=yd)
            net.forward(yd, out=xh)
        net.profile(True)
        times = []
        for _ in range(args.fused_steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.measure(xd, out=yd)
            net.forward(yd, out=xh)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        st = net.profile_read()
        net.close()
        ms = sorted(times)[len(times) // 2]
        out["%.2f" % ratio] = {"M": M, "images_per_s": B / (ms / 1000.0), "ms_per_step": ms,
                               "stage_ms": {k: v[0] / max(1, v[1]) for k, v in st.items() if v[1]}}
    out["workload"] = "sense+recover 64x64, batch %d, L2 flushed between steps (median step)" % B
    return out


def large_bench(args):
    """256 x 256 images (N = 65536), M/N = 0.1 (M = 6554), batch 256 of DCT-sparse
    images (K = 2000, seed 5): the bf16 path and the e4m3-conv2 path on the same batch.
    Step = y = Phi x then x^ = M(y); images/s by CUDA events; conv2 TFLOP/s from the
    library's stage events; rel-L2 of the e4m3 result against the bf16 one."""
    import numpy as np
    import torch
    from paper_1701_03891_gb300 import deepinv, synth
    n, B, ratio = 256, 256, 0.10
    N = n * n
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1)
    x = synth.dct_sparse_images(B, n, n, K=2000, seed=5)
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.current_stream()
    out = {"workload": "sense+recover 256x256, M/N=0.10 (M=%d), batch %d, DCT-sparse K=2000" % (M, B)}
    pk = peaks()
    results = {}
    for prec in ("bf16", "fp8"):
        net = deepinv.Net(phi, params, n, n, prec=prec)
        net.reserve(B)
        yd = torch.empty((B, M), device="cuda")
        xh = torch.empty((B, N), device="cuda")
        net.measure(xd, out=yd)
        if prec == "fp8":
            net.calibrate(yd)
        for _ in range(2):
            net.measure(xd, out=yd)
            net.forward(yd, out=xh)
        torch.cuda.synchronize()
        net.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.large_steps):
            net.measure(xd, out=yd)
            net.forward(yd, out=xh)
        e1.record(stream)
        torch.cuda.synchronize()
        st = net.profile_read()
        net.profile(False)
        ms = e0.elapsed_time(e1) / args.large_steps
        c2 = st["conv2"][0] / max(1, st["conv2"][1])
        results[prec] = xh.cpu().numpy()
        tf = 2.0 * 64 * 32 * 121 * B * N / (c2 / 1000.0) / 1e12
        # e4m3 against twice the measured bf16 burst peak (the nominal fp8 : bf16 dense ratio)
        peak = pk["bf16"] * (2.0 if prec == "fp8" else 1.0)
        out[prec] = {"images_per_s": B / (ms / 1000.0), "ms_per_step": ms,
                     "conv2_ms": c2, "conv2_tflops": tf, "conv2_peak_tflops": peak, "conv2_frac": tf / peak,
                     "conv2_peak_note": ("2 x the measured bf16 burst peak (nominal e4m3 : bf16 dense ratio)"
                                         if prec == "fp8" else "measured bf16 burst peak"),
                     "stage_ms": {k: v[0] / max(1, v[1]) for k, v in st.items()}}
        net.close()
        del yd, xh
    rel = np.linalg.norm(results["fp8"] - results["bf16"], axis=1) / np.linalg.norm(results["bf16"], axis=1)
    out["fp8_over_bf16"] = out["fp8"]["images_per_s"] / out["bf16"]["images_per_s"]
    out["fp8_vs_bf16_max_rel_l2"] = float(rel.max())
    return out


def fused_bench(args):
    """conv1 + conv2 fused into one kernel (a1 kept in shared memory) against the
    two kernels, on the bf16 forward pass: 64 x 64, M/N = 0.1, batch 1024 (the
    benchmark workload, walked whole) and 256 x 256, M/N = 0.1, batch 256 (walked
    as column strips).  Step = x^ = M(y) with y resident; CUDA events over the
    steps; the library's stage events give conv1 + conv2 against the fused kernel.
    The two results are compared bit for bit."""
    import numpy as np
    import torch
    from paper_1701_03891_gb300 import deepinv, synth
    out = {}
    stream = torch.cuda.current_stream()
    for n, B in ((64, 1024), (256, 256)):
        N = n * n
        M = synth.m_for_ratio(0.10, N)
        phi = synth.gaussian_phi(M, N, seed=0)
        params = synth.he_params(seed=1)
        x = synth.voronoi_images(B, n, n, seed=3)
        net = deepinv.Net(phi, params, n, n, prec="bf16")
        net.reserve(B)
        yd = net.measure(torch.from_numpy(x).cuda())
        xh = torch.empty((B, N), device="cuda")
        res, outs = {}, {}
        for mode in ("two_kernels", "fused"):
            net.set_fused(mode == "fused")
            for _ in range(3):
                net.forward(yd, out=xh)
            torch.cuda.synchronize()
            net.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.fused_steps):
                net.forward(yd, out=xh)
            e1.record(stream)
            torch.cuda.synchronize()
            st = net.profile_read()
            net.profile(False)
            ms = e0.elapsed_time(e1) / args.fused_steps
            stage = {k: v[0] / max(1, v[1]) for k, v in st.items() if v[1]}
            res[mode] = {"forward_ms": ms, "images_per_s": B / (ms / 1000.0),
                         "conv1_plus_conv2_ms": stage.get("conv1", 0.0) + stage.get("conv2", 0.0),
                         "stage_ms": stage}
            outs[mode] = xh.cpu().numpy()
        net.close()
        res["fused_over_two_kernels"] = res["fused"]["images_per_s"] / res["two_kernels"]["images_per_s"]
        res["bit_identical"] = bool(np.array_equal(outs["fused"], outs["two_kernels"]))
        res["workload"] = "forward %dx%d, M/N=0.10 (M=%d), batch %d, y resident" % (n, n, M, B)
        out["%dx%d" % (n, n)] = res
    return out


def train_bench(args):
    """Training step at 64 x 64, M/N = 0.25 (M = 1024), batch 256, bf16 compute with
    float32 masters: forward (activations saved) + MSE loss + backward (conv
    dgrad/wgrad, ReLU masks, FC weight gradient) + SGD with momentum."""
    import numpy as np
    import torch
    from paper_1701_03891_gb300 import deepinv, synth
    n, B, ratio = 64, 256, 0.25
    N = n * n
    M = synth.m_for_ratio(ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1)
    x = synth.voronoi_images(B, n, n, seed=7)
    net = deepinv.Net(phi, params, n, n, prec="bf16", train_fc=True)
    net.reserve(B)
    xd = torch.from_numpy(x).cuda()
    yd = net.measure(xd)
    xh = torch.empty((B, N), device="cuda")
    saved = net.new_saved(B)
    grads = net.grad_buffers()
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev: ev[0].record(stream)
        net.forward(yd, out=xh, saved=saved)
        if ev: ev[1].record(stream)
        loss, dW, db, dWfc = net.backward(yd, xd, saved, grads=grads)
        if ev: ev[2].record(stream)
        net.sgd_momentum(dW, db, dWfc, lr=1e-4, mu=0.9)
        if ev: ev[3].record(stream)
        return loss

    losses = [float(step()) for _ in range(2)]
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.train_steps)]
    for k in range(args.train_steps):
        loss = step(evs[k])
    torch.cuda.synchronize()
    losses.append(float(loss))
    fwd = np.mean([e[0].elapsed_time(e[1]) for e in evs])
    bwd = np.mean([e[1].elapsed_time(e[2]) for e in evs])
    upd = np.mean([e[2].elapsed_time(e[3]) for e in evs])
    tot = np.mean([e[0].elapsed_time(e[3]) for e in evs])
    net.close()
    return {"workload": "training step 64x64, M/N=0.25 (M=%d), batch %d, bf16 compute, fp32 masters, FC trained" % (M, B),
            "images_per_s": B / (tot / 1000.0), "ms_per_step": tot,
            "phase_ms": {"forward_saved": fwd, "loss_and_backward": bwd, "sgd_momentum": upd},
            "loss_first": losses[0], "loss_last": losses[-1]}


def deep_bench(args):
    """Deeper network (two extra 32 -> 32 hidden layers: five conv layers, the
    larger-capacity networks Sec. 5 leaves to future work) at 64 x 64:
    sense + recover at M/N = 0.10, batch 1024 (Voronoi images, seed 3, as the
    headline), and a training step at M/N = 0.25, batch 256 (FC trained).
    Hidden-layer TFLOP/s from the library's stage events (2 x 32 x 32 x 121
    FLOP per pixel and layer)."""
    import numpy as np
    import torch
    from paper_1701_03891_gb300 import deepinv, synth
    n, hidden = 64, 2
    N = n * n
    stream = torch.cuda.current_stream()
    out = {"hidden_layers": hidden, "conv_layers": 3 + hidden}
    # inference
    B = 1024
    M = synth.m_for_ratio(0.10, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1, hidden=hidden)
    x = synth.voronoi_images(B, n, n, seed=3)
    net = deepinv.Net(phi, params, n, n, prec="bf16")
    net.reserve(B)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, M), device="cuda")
    xh = torch.empty((B, N), device="cuda")
    for _ in range(2):
        net.measure(xd, out=yd)
        net.forward(yd, out=xh)
    torch.cuda.synchronize()
    net.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.deep_steps):
        net.measure(xd, out=yd)
        net.forward(yd, out=xh)
    e1.record(stream)
    torch.cuda.synchronize()
    st = net.profile_read()
    net.profile(False)
    ms = e0.elapsed_time(e1) / args.deep_steps
    hid_ms = st["hidden"][0] / max(1, st["hidden"][1])
    out["inference"] = {"workload": "sense+recover 64x64, M/N=0.10 (M=%d), batch %d, %d conv layers" % (M, B, 3 + hidden),
                        "images_per_s": B / (ms / 1000.0), "ms_per_step": ms,
                        "hidden_ms_per_layer": hid_ms / hidden,
                        "hidden_tflops": 2.0 * 32 * 32 * 121 * B * N * hidden / (hid_ms / 1000.0) / 1e12,
                        "stage_ms": {k: v[0] / max(1, v[1]) for k, v in st.items()}}
    net.close()
    del yd, xh
    # training
    B = 256
    M = synth.m_for_ratio(0.25, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    x = synth.voronoi_images(B, n, n, seed=7)
    net = deepinv.Net(phi, params, n, n, prec="bf16", train_fc=True)
    net.reserve(B)
    xd = torch.from_numpy(x).cuda()
    yd = net.measure(xd)
    xh = torch.empty((B, N), device="cuda")
    saved = net.new_saved(B)
    grads = net.grad_buffers()

    lr = [0.0]

    def step():
        net.forward(yd, out=xh, saved=saved)
        loss, dW, db, dWfc = net.backward(yd, xd, saved, grads=grads)
        if not lr[0]:
            lr[0] = 1e-3 / float(loss)       # step relative to the first loss (He init, five layers)
        net.sgd_momentum(dW, db, dWfc, lr=lr[0], mu=0.9)
        return loss

    first = float(step())
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.deep_steps):
        loss = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.deep_steps
    out["training"] = {"workload": "training step 64x64, M/N=0.25 (M=%d), batch %d, %d conv layers, bf16 compute, "
                                   "fp32 masters, FC trained" % (M, B, 3 + hidden),
                       "images_per_s": B / (ms / 1000.0), "ms_per_step": ms, "lr": lr[0],
                       "loss_first": first, "loss_last": float(loss)}
    net.close()
    return out


SERVE_SIZES = (32, 64, 128)
SERVE_RATIOS = (0.05, 0.10, 0.25)
SERVE_MAX_BATCH = 256   # requests per batch at most; batches take what has queued


def serving_bench(args):
    """Mixed-size serving: 9 resident bf16 networks (32/64/128 squared x M/N 0.05/0.10/0.25),
    Poisson arrivals (seed 4) of single recoveries drawn uniformly over the 9 classes,
    a continuous-batching server (4 streams, batches <= 64, 40 GB budget); per offered
    rate: latency p50/p99 (scheduled arrival -> result in host memory) and images/s."""
    import numpy as np
    from paper_1701_03891_gb300 import deepinv, synth
    nets, pools = [], []
    for si, n in enumerate(SERVE_SIZES):
        N = n * n
        for ri, r in enumerate(SERVE_RATIOS):
            M = synth.m_for_ratio(r, N)
            phi = synth.gaussian_phi(M, N, seed=100 + 3 * si + ri)
            net = deepinv.Net(phi, synth.he_params(seed=1), n, n, prec="bf16")
            x = synth.voronoi_images(16, n, n, seed=200 + 3 * si + ri)
            y = (x.astype(np.float64) @ phi.astype(np.float64).T).astype(np.float32)
            nets.append(net)
            pools.append((np.ascontiguousarray(y), N))
    srv = deepinv.Server(hbm_budget_bytes=40 << 30, max_streams=4, max_batch=SERVE_MAX_BATCH)
    for net in nets:
        srv.add(net)
    # warm-up: every network runs a few batches first (the kernels' first launches
    # load their code), outside the measured sweep
    warm = (deepinv.Request * (len(nets) * 4))()
    wbuf = [np.empty((4, pools[c][1]), np.float32) for c in range(len(nets))]
    for c in range(len(nets)):
        for i in range(4):
            warm[4 * c + i] = deepinv.Request(c, pools[c][0][i].ctypes.data, wbuf[c][i].ctypes.data, 4 * c + i)
    res = (deepinv.Result * 64)()
    rc, got = srv.serve_raw(warm, 0, len(warm), res, 64, 0)
    while got < len(warm):
        rc, n_out = srv.serve_raw(warm, 0, 0, res, 64, 100000)
        got += n_out
    rng = np.random.default_rng(4)

    def measure(rate, seconds):
        n_req = int(min(400000, max(500, rate * seconds)))
        cls = rng.integers(0, len(nets), n_req)
        arrive = np.cumsum(rng.exponential(1.0 / rate, n_req))
        # results land in a ring of 64 host buffers per class (values are not checked here)
        ring = [np.empty((64, pools[c][1]), np.float32) for c in range(len(nets))]
        reqs = (deepinv.Request * n_req)()
        for i, c in enumerate(cls):
            y, _ = pools[c]
            reqs[i] = deepinv.Request(int(c), y[i % y.shape[0]].ctypes.data, ring[c][i % 64].ctypes.data, i)
        res = (deepinv.Result * 4096)()
        lag = np.zeros(n_req)
        lat = np.zeros(n_req)
        batch = np.zeros(n_req)
        done = 0
        sent = 0
        t0 = time.perf_counter()
        while done < n_req:
            now = time.perf_counter() - t0
            k = int(np.searchsorted(arrive, now, side="right")) - sent
            if k > 0:
                lag[sent:sent + k] = now - arrive[sent:sent + k]
            rc, n_out = srv.serve_raw(reqs, sent, max(0, k), res, 4096, 0)
            sent += max(0, k)
            for j in range(n_out):
                r = res[j]
                lat[r.tag] = r.latency_us * 1e-6
                batch[r.tag] = r.batch
            done += n_out
            if n_out == 0 and sent == n_req:
                time.sleep(20e-6)
        t_end = time.perf_counter() - t0
        total = lat + lag
        return {"offered_rps": rate, "requests": n_req,
                "images_per_s": n_req / t_end,
                "p50_ms": float(np.percentile(total, 50) * 1e3),
                "p99_ms": float(np.percentile(total, 99) * 1e3),
                "mean_batch": float(batch.mean())}

    rates = [float(v) for v in args.serve_rates.split(",") if v]
    # a short stream at the first rate first, not reported: the first seconds after
    # the set-up carry one-time costs (host threads and the GPU waking from idle)
    if rates:
        measure(rates[0], 0.1)
    points = [measure(rate, args.serve_seconds) for rate in rates]
    st = srv.stats()
    srv.close()
    for net in nets:
        net.close()
    # saturation: the highest throughput served, and the first offered rate the
    # server could not keep up with (served < 90 % of offered)
    sat = max(p["images_per_s"] for p in points) if points else None
    behind = [p["offered_rps"] for p in points if p["images_per_s"] < 0.9 * p["offered_rps"]]
    return {"workload": "9 bf16 networks: %s x M/N %s; Poisson arrivals, uniform over classes; "
                        "4 streams, batches <= %d, 40 GB budget" % ("/".join("%d^2" % n for n in SERVE_SIZES),
                                                                   "/".join(str(r) for r in SERVE_RATIOS),
                                                                   SERVE_MAX_BATCH),
            "latency": "scheduled arrival -> result in the request's host buffer",
            "points": points, "saturation_images_per_s": sat,
            "first_offered_rps_not_kept_up": behind[0] if behind else None,
            "max_in_flight": st["max_in_flight"], "batches": st["batches"],
            "peak_workspace_gb": st["peak_workspace_bytes"] / 2**30}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1701_03891_gb300 import synth
    oracle.build()
    # rank 0 has the host to itself (a launcher sets OMP_NUM_THREADS=1 for its workers)
    oracle.set_num_threads(os.cpu_count() or 1)
    n = args.size
    N = n * n
    M = synth.m_for_ratio(args.ratio, N)
    phi = synth.gaussian_phi(M, N, seed=0)
    params = synth.he_params(seed=1)
    x = synth.voronoi_images(max(1, args.steps + args.warmup), n, n, seed=3)
    for i in range(args.warmup):
        oracle.forward(oracle.measure(phi, x[i:i + 1]), params, n, n, phi=phi)
    t0 = time.perf_counter()
    for i in range(args.steps):
        j = args.warmup + i
        oracle.forward(oracle.measure(phi, x[j:j + 1]), params, n, n, phi=phi)
    dt = time.perf_counter() - t0
    val = args.steps / dt
    cfg = config(args, n, M, 1)
    cfg["workload"] += "; reference = FP64 CPU oracle, one image per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "images/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Voronoi images standing in for ImageNet 64x64 crops)",
            "config": cfg,
            "cpu_baseline": {"value": val, "unit": "images/s", "cores": oracle.num_threads(), "cpu": host_cpu(),
                             "kind": "oracle", "sample": "one image of the batch per step, %d steps" % args.steps},
            "e2e": {"value": val, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1701_03891_gb300 import build as libbuild, deepinv
    libbuild.build()
    n, N, M, phi, params, x = workload(args, rank)
    B = args.batch
    pk = peaks()

    net = deepinv.Net(phi, params, n, n, prec="bf16")
    net.set_conv1_rows(args.conv1_rows)
    net.reserve(B)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, M), device="cuda")
    xh = torch.empty((B, N), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        net.measure(xd, out=yd)
        net.forward(yd, out=xh)

    # the clock sampler starts before the warm-up, so that nvidia-smi's own start-up
    # (driver queries that can stall this process's CUDA calls) is over before the
    # timed region; it samples until the timed region ends
    clocks = Clocks(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    net.profile(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = deepinv.launch_count()
    host_issue = []
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        h0 = time.perf_counter()
        step()
        host_issue.append(time.perf_counter() - h0)
        evs[k][1].record(stream)
    w_issued = time.perf_counter() - w0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - w0
    launches = deepinv.launch_count() - launches0
    clk = clocks.stop()
    stages = net.profile_read()
    net.profile(False)
    step_times = sorted(a.elapsed_time(b) for a, b in evs)
    dev_ms = sum(step_times)
    dev_ms, value = aggregate(dev_ms, B, args.steps, world, dist, device="cuda")
    ms_per_step = dev_ms / args.steps
    step_stats = {"median": step_times[len(step_times) // 2], "min": step_times[0], "max": step_times[-1],
                  "note": "this rank's per-step CUDA-event times (ms)"}

    stage_ms = {k: v[0] / max(1, v[1]) for k, v in stages.items()}
    roof = roofline(stage_ms, B, n, M, pk, clk)

    bf16_out = xh.cpu().numpy()
    # float32 CUDA-core path on the same batch
    netf = deepinv.Net(phi, params, n, n, prec="f32")
    netf.reserve(B)
    yf = torch.empty((B, M), device="cuda")
    xf = torch.empty((B, N), device="cuda")
    netf.measure(xd, out=yf)
    netf.forward(yf, out=xf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.fp32_steps):
        netf.measure(xd, out=yf)
        netf.forward(yf, out=xf)
    e1.record(stream)
    torch.cuda.synchronize()
    f32_ms = e0.elapsed_time(e1) / args.fp32_steps
    f32_out = xf.cpu().numpy()
    rel = np.linalg.norm(bf16_out - f32_out, axis=1) / np.linalg.norm(f32_out, axis=1)
    del netf, yf, xf

    # end to end through the host-memory entry points: every step copies its batch
    # from pinned host memory and its x^ back; the submit / wait pair keeps two
    # batches in flight, so a batch's copies overlap its neighbours' compute
    xh_host = [torch.from_numpy(x).pin_memory() for _ in range(2)]
    out_host = [torch.empty((B, N), dtype=torch.float32).pin_memory() for _ in range(2)]
    for _ in range(2):
        net.sense_recover_host(xh_host[0], out_host[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = None
    for k in range(args.e2e_steps):
        t = net.sense_recover_host_submit(xh_host[k % 2], out_host[k % 2])
        if prev is not None:
            net.host_wait(prev)
        prev = t
    net.host_wait(prev)
    e2e_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        net.sense_recover_host(xh_host[0], out_host[0])
    sync_s = time.perf_counter() - t0
    e2e = {"value": world * B * args.e2e_steps / e2e_s, "unit": "images/s",
           "h2d_bytes_per_step": B * N * 4, "d2h_bytes_per_step": B * N * 4,
           "call": "deepinv_sense_recover_host_submit + deepinv_host_wait, two batches in flight "
                   "(pinned x in, pinned x^ out)",
           "sync_value": world * B * args.e2e_steps / sync_s,
           "sync_call": "deepinv_sense_recover_host, one batch at a time"}

    # the sections below run after the headline was measured: a failure in one
    # is recorded in its place in the line instead of losing the measurement
    serving = None
    if rank == 0 and not args.no_serving:
        serving = optional("serving", serving_bench, args)
    large = None
    if rank == 0 and not args.no_large:
        large = optional("large_256", large_bench, args)
    train = None
    if rank == 0 and not args.no_train:
        train = optional("train_64", train_bench, args)
    deep = None
    if rank == 0 and not args.no_deep:
        deep = optional("deep_64", deep_bench, args)
    ratios = None
    if rank == 0 and not args.no_ratios:
        ratios = optional("ratios_64", ratios_bench, args)
    fused = None
    if rank == 0 and not args.no_fused:
        fused = optional("fused12", fused_bench, args)

    evaluation = None
    if rank == 0 and args.eval:
        from paper_1701_03891_gb300 import evaluate
        evaluation = optional("eval_32", lambda: {
            "workload": "32x32 Voronoi images, 512 training / 64 test, 6000 SGD-momentum steps of 64 "
                        "(bf16, FC = Phi^T), step 1e-3 / first loss",
            "points": evaluate.sweep(32, ratios=(0.05, 0.10, 0.25), snrs=(None, 20.0)),
            "depth": evaluate.depth_sweep(32, 0.10, hiddens=(0, 1, 2)),
            "convergence_64": evaluate.train_and_evaluate(64, 0.10, steps=6000, curve_every=1000)})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = optional("cpu_baseline", cpu_baseline, args, phi, params, x, n, bf16_out)

    status = deepinv.device_status()
    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "step_ms": step_stats,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded Voronoi images standing in for ImageNet 64x64 crops; He-init weights)",
            "config": config(args, n, M, world),
            "roofline": roof, "stage_ms": stage_ms,
            "fp32": {"value": world * B / (f32_ms / 1000.0), "unit": "images/s", "ms_per_step": f32_ms,
                     "bf16_over_fp32": (world * B / (ms_per_step / 1000.0)) / (world * B / (f32_ms / 1000.0)),
                     "bf16_vs_fp32_max_rel_l2": float(rel.max())},
            "e2e": e2e, "serving": serving, "large_256": large, "train_64": train, "deep_64": deep,
            "fused12": fused, "ratios_64": ratios,
            "eval_32": evaluation,
            "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": launches,
            "gpu_launches_note": "the library's own kernel launches in the timed region, counted by "
                                 "deepinv_launch_count (the L2-flush fill is torch's and not counted)",
            "wall_s_timed_region": wall,
            "host": {"issue_ms_per_step": {"median": 1e3 * sorted(host_issue)[len(host_issue) // 2],
                                           "max": 1e3 * max(host_issue)},
                     "issue_s_all_steps": w_issued,
                     "note": "host time to issue each step's calls (argument checks + launches); the "
                             "wall time of the timed region also holds the L2-flush fills and the final "
                             "synchronisation"},
            "device_status": status}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def optional(name, fn, *a):
    """One of the line's extra sections; an exception in it is reported (stderr,
    and an "error" entry in its place) instead of ending the run."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 -- any failure of an extra section
        print("bench: section %s failed: %r" % (name, e), file=sys.stderr, flush=True)
        return {"error": "%s: %s" % (type(e).__name__, e)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
