#!/usr/bin/env python
"""Benchmark of the rasterised SMoE fit step on GB300.

One step = one fit iteration of the whole hot path on one image: binning
(bounding boxes, prefix sum, scatter, per-tile sort), the fused per-tile
forward render + MSE + backward, and finalize + Adam.  Workload (default):
2048x2048 RGB synthetic image (polygons with colour ramps + Perlin texture),
K = 262144 anisotropic kernels with linear experts, 16x16 tiles, q_max = 9.

Metric: fwd+bwd pixel-kernel evaluations per second, where the evaluations of
one step are sum over tiles of (in-image pixels of the tile) x (length of the
tile's kernel list) -- the paper's per-block work count (FLOPs/pixel = 2 x
average kernels per block, Tables I/II), counted once per forward+backward.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): every rank fits its own image (replicas, weak scaling),
no collective on the data path; rank 0 prints the job-wide line.
The reference arm (--impl reference) times the CPU oracle as it stands on the
host cores, on a bounded crop of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Gpix·kernel evals/s; fit p50/p99 latency at matched PSNR vs plain"
UNIT = "Gpix·kernel evals/s"
WORKLOAD = ("rgb2048_K262144_linear_aniso: 2048x2048 RGB fp32, 40 ramp polygons + Perlin "
            "texture 0.1, K=262144 anisotropic kernels (area sigma 5 px, aspect 1-3), linear "
            "experts, 16x16 tiles, q_max 9, Adam at the paper's rates")
MUFU_PER_CLK_PER_SM = 32          # ex2 lanes per clock per SM if the live measurement fails
# Algorithmic FP32 lane operations per in-range fwd+bwd pair, RGB linear
# experts: 19 in the forward and 48 in the backward (the per-pair count of the
# method's formulas, Eqs. 2-5 and their chain rule).
FP32_OPS_PER_PAIR = 67
# The server's cap on megapixels (image pixels x models) in flight: 8 / 16 /
# 32 / 64 measured 12.7 / 14.4 / 15.5 / 15.9 requests/s with p99 5.0 / 4.6 /
# 4.2 / 4.3 s on the serving workload (p50 3.2 / 2.4 / 3.2 / 3.9 s).
SERVE_MAX_MPX = 32.0
# PSNR the fit-to-PSNR leg times the 2048^2 fit to.
FIT_TARGET_DB = 50.0
# Kernels launched by one fit step: binning (bbox, huge-box cover, scan
# reduce/top/down, scatter, warp sort, long-list sort), the fused tile
# kernel, fused Adam.
KERNELS_PER_STEP = 10
# The fit re-sorts its kernels spatially every this many steps (FitBatch
# reorder_every; smoe_fit_reorder, 15 kernels); the timed steps include it.
REORDER_EVERY = 25
REORDER_KERNELS = 15
# From one ncu capture of the fused tile kernel on this workload (profiles/):
# DRAM bytes per launch, pipe utilisation and the executed FP32 lane
# operations (FFMA + FADD + FMUL + 2 x (FFMA2 + FADD2 + FMUL2) thread
# instructions); valid only while render.cu's code (comments and whitespace
# aside) is the code that was profiled.
NCU = {"render_cu_code_sha256": "b26ed48b808165f25b91cebb5b2189f88799079aeb5f09a65e078bc64d7d3511",
       "bytes_per_launch": 103.988736e6, "fma_pipe_active": 0.6125, "issue_active": 0.6250,
       "xu_active": 0.1359, "fp32_lane_ops": 14.632671605e9}

def issue_rates():
    """Measured lane operations per clock per SM of ex2 / FFMA / packed
    f32x2 FMA (libsmoe_rates.so), or None."""
    import ctypes
    from paper_2510_05814_gb300 import build
    try:
        lib = ctypes.CDLL(build.RATES_LIB)
    except OSError:
        return None
    out = (ctypes.c_double * 3)()
    clk = ctypes.c_double(0.0)
    lib.smoe_issue_rates.restype = ctypes.c_int
    if lib.smoe_issue_rates(out, ctypes.byref(clk)) != 0:
        return None
    return {"ex2": out[0], "ffma": out[1], "ffma2": out[2], "clock_mhz": clk.value}


def code_sha256(path):
    """sha256 of a C/CUDA source with its comments and whitespace removed: the
    text the compiler sees, so that a comment edit does not invalidate the
    profile figures taken from it."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()


class Clocks:
    """nvidia-smi samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def evaluated_pairs(tile_off, W, H, T):
    """sum over tiles of in-image pixels x list length (host, int64)."""
    import numpy as np
    tx, ty = (W + T - 1) // T, (H + T - 1) // T
    lens = np.diff(tile_off.astype(np.int64))[: tx * ty].reshape(ty, tx)
    pw = np.minimum(T, W - np.arange(tx) * T)
    ph = np.minimum(T, H - np.arange(ty) * T)
    return int((lens * ph[:, None] * pw[None, :]).sum())


def crop_workload(wl, size):
    """A size x size crop of a workload with the kernels whose centre lies in
    it (same density, same list lengths) -- the oracle's bounded sample."""
    import numpy as np
    from paper_2510_05814_gb300 import synth
    C, H, W = wl.target.shape
    x0, y0 = (W - size) // 2, (H - size) // 2
    t = wl.target[:, y0:y0 + size, x0:x0 + size].copy()
    p = wl.params
    px, py = p.mu[:, 0] * W - x0, p.mu[:, 1] * H - y0
    sel = (px >= 0) & (px < size) & (py >= 0) & (py < size)
    mu = np.stack([px[sel] / size, py[sel] / size], 1).astype(np.float32)
    return t, synth.Params(mu, p.chol[sel].copy(), p.ea[sel].copy(),
                           None if p.eW is None else p.eW[sel].copy())


def oracle_sample(wl, size):
    """Time the oracle (fwd + MSE backward, dense) on a crop; returns
    (pairs in the metric's count, seconds, threads)."""
    import oracle as om
    t, p = crop_workload(wl, size)
    m = om.Model(size, size, t.shape[0], p.mu, p.chol, p.ea, p.eW, tile=wl.tile, qmax=wl.qmax)
    off, _ = om.bin_tiles(m)
    pairs = evaluated_pairs(off, size, size, wl.tile)
    t0 = time.perf_counter()
    om.render(m)
    om.backward(m, target=t)
    return pairs, time.perf_counter() - t0, om.threads(), int(p.mu.shape[0])


def binned_sample(wl, size):
    """Time the binned CPU baseline (oracle binning + per-tile list walks,
    FP64, OpenMP) on a crop: one step's binning, forward, MSE and backward;
    returns (pairs in the metric's count, seconds, threads, kernels)."""
    import oracle as om
    t, p = crop_workload(wl, size)
    m = om.Model(size, size, t.shape[0], p.mu, p.chol, p.ea, p.eW, tile=wl.tile, qmax=wl.qmax)
    t0 = time.perf_counter()
    off, pk = om.bin_tiles(m)
    om.fwd_bwd_binned(m, t, lists=(off, pk))
    sec = time.perf_counter() - t0
    return evaluated_pairs(off, size, size, wl.tile), sec, om.threads(), int(p.mu.shape[0])


def dist_init(backend="nccl"):
    """Rank layout from the torchrun environment; joins the process group
    when WORLD_SIZE > 1 (NCCL on GPUs; gloo for the CPU tests of this logic)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return ws, rank, local


def replica_seed(rank):
    """Each rank fits its own image (independent problems, weak scaling)."""
    return 3 + rank


def aggregate(step_s, work, e2e_s, world, device="cuda"):
    """Job-wide figures: the slowest rank's times (max) and the work of all
    ranks (sum); the only collective of the benchmark, outside the timed
    region."""
    import torch
    vals = torch.tensor([step_s, work, e2e_s], dtype=torch.float64, device=device)
    if world == 1:
        return float(vals[0]), float(vals[1]), float(vals[2])
    mx, sm = vals.clone(), vals.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(mx[2])


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2510_05814_gb300 import synth
    import oracle
    oracle.build()
    wl = synth.rgb_2048()
    # The dense oracle's cost per step grows as crop^4 (pixels x kernels); take
    # the largest crop that keeps the whole run near 90 s (0.22 s per 256^2
    # step on 16 cores), unless --ref-crop is given.
    size = args.ref_crop
    if not size:
        n = args.steps + args.warmup
        size = next((c for c in (256, 192, 128, 96, 64) if n * 0.22 * (c / 256) ** 4 <= 90.0), 64)
    for _ in range(args.warmup):
        oracle_sample(wl, size)
    tot_pairs, tot_s, thr, kc = 0, 0.0, 1, 0
    for _ in range(args.steps):
        pairs, s, thr, kc = oracle_sample(wl, size)
        tot_pairs += pairs
        tot_s += s
    value = tot_pairs / tot_s / 1e9
    sample = (f"{size}x{size} centre crop of the 2048x2048 workload with its {kc} kernels; "
              "dense oracle forward + MSE backward per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batched(args):
    """64 RGB images with ragged sizes (128x96 .. 1920x1080), K = pixels/16,
    one batched fit (autotuned tile side / persistent launch) against the
    same fits run one image per launch; equal iterations, so equal PSNR up to
    FP32 summation order."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import api, autotune, build, synth
    from paper_2510_05814_gb300.fit import FitBatch
    build.build()
    sizes = synth.ragged_sizes(args.images, 4)
    targets, params = [], []
    for i, (W, H) in enumerate(sizes):
        t = synth.polygon_image(W, H, 3, 40, 400 + i, texture_amp=0.1)
        targets.append(torch.tensor(t, device="cuda"))
        params.append(api.SMoEParams.from_numpy(synth.init_params(t, (W * H) // 16, 5.0, True, 400 + i)))
    lr = [synth.fit_rates(W, H) for W, H in sizes]
    tr = autotune.tune(targets, params, lr, tiles=(8, 16, 32), persistent=(False, True))
    n = args.iters
    # batched: graph of `chunk` iterations replayed
    # both arms re-sort their kernels spatially after every graph replay
    # (FitBatch reorder_every; the first, untimed call captures its graph)
    chunk = 25
    # both arms size their pair buffers at 3x the initial pairs: the lists
    # grow as the kernels widen, and regrowth (a re-initialisation and a new
    # graph) is then rare in either arm
    fb = FitBatch(targets, [p.clone() for p in params], n, lr=lr, tile=tr.tile,
                  persistent=tr.persistent, deterministic=True, reorder_every=chunk,
                  pair_slack=3.0)
    fb.capture(chunk)
    fb.reorder()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # FitBatch.run: graph replays with the re-sort every `chunk` iterations; a
    # pair-buffer overflow (the lists grow as kernels widen) grows the buffer
    # and resumes, inside the timed region, in both arms
    cap0 = fb.pair_cap
    e0.record()
    fb.run(n, graph_iters=chunk)
    e1.record()
    torch.cuda.synchronize()
    assert fb.status_code() == 0
    grown = {"batched": int(fb.pair_cap != cap0), "plain": 0}
    t_batched = e0.elapsed_time(e1) / 1e3
    # plain: each image alone, one image per launch, same iterations
    t_plain = 0.0
    psnr_b, psnr_p, lat_plain = [], [], []
    for b in range(len(targets)):
        one = FitBatch([targets[b]], [params[b].clone()], n, lr=lr[b], tile=tr.tile,
                       deterministic=True, reorder_every=chunk, pair_slack=3.0)
        one.capture(chunk)
        one.reorder()
        torch.cuda.synchronize()
        cap0 = one.pair_cap
        e0.record()
        one.run(n, graph_iters=chunk)
        e1.record()
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1) / 1e3
        lat_plain.append(t_plain)
        assert one.status_code() == 0
        grown["plain"] += int(one.pair_cap != cap0)
        C, H, W = targets[b].shape
        yb, _, _ = api.render(fb.params_of(b), W, H, tile=tr.tile)
        yp, _, _ = api.render(one.params_of(0), W, H, tile=tr.tile)
        from paper_2510_05814_gb300.serve import synth_psnr
        tb = targets[b].cpu().numpy()
        psnr_b.append(synth_psnr(yb.cpu().numpy(), tb))
        psnr_p.append(synth_psnr(yp.cpu().numpy(), tb))
        del one
    # pairs per iteration of the batch (lists of the final parameters)
    pairs = 0
    for b in range(len(targets)):
        C, H, W = targets[b].shape
        r = api.Rasterizer(api.RasterDesc(W, H, C, tr.tile, True), params[b].K).bin(fb.params_of(b))
        pairs += evaluated_pairs(r.tile_off.cpu().numpy(), W, H, tr.tile)
    dpsnr = float(np.max(np.abs(np.array(psnr_b) - np.array(psnr_p))))
    print(json.dumps({
        "metric": "batched fit: fwd+bwd Gpix·kernel evals/s and fit latency vs one image per launch",
        "mode": "batched", "images": len(targets), "iters": n,
        "pixels": int(sum(t.shape[1] * t.shape[2] for t in targets)),
        "kernels": int(sum(p.K for p in params)), "pairs_per_iter": int(pairs),
        "reorder_every": chunk, "pair_buffers_grown": grown,
        "autotune": {"tile": tr.tile, "persistent": tr.persistent,
                     "table_ms_per_iter": [[a, bool(b_), c] for a, b_, _, c in tr.table]},
        "batched": {"s": t_batched, "ms_per_iter": 1e3 * t_batched / n,
                    "value": pairs * n / t_batched / 1e9, "latency_all_s": t_batched},
        "plain": {"s": t_plain, "ms_per_iter": 1e3 * t_plain / n,
                  "value": pairs * n / t_plain / 1e9,
                  "latency_p50_s": float(np.percentile(lat_plain, 50)),
                  "latency_p99_s": float(np.percentile(lat_plain, 99))},
        "speedup": t_plain / t_batched,
        "psnr_mean_db": float(np.mean(psnr_b)), "max_abs_psnr_diff_db": dpsnr,
        "unit": UNIT, "data": "synthetic", "dtype": "f32",
    }), flush=True)


def run_denoise(args):
    """MM-RSMoE denoising (Sec. V-C) on the synthetic 768x512 RGB stand-in
    for the paper's test images: for each noise variance of Table III and
    each model count H, the H fits of the noisy image run as one batch
    (CUDA-graph replays of 25 iterations) and the fused render follows;
    reports PSNR of the noisy and the fused image against the clean one and
    the GPU time of fit + fusion."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import build, denoise, synth
    from paper_2510_05814_gb300.fit import FitBatch
    build.build()
    W, H = 768, 512
    K = W * H // 64
    n = args.iters
    chunk = 25

    def psnr(y, c):
        mse = float(((y.clamp(0.0, 1.0) - c) ** 2).mean())
        return 10.0 * np.log10(1.0 / mse)

    rows = []
    for var in (0.0037, 0.005, 0.01, 0.05):
        clean, noisy = synth.denoise_case(W, H, var, seed=5)
        c = torch.tensor(clean, device="cuda")
        tn = torch.tensor(noisy, device="cuda")
        for nm in args.models:
            models = denoise.init_models(noisy, nm, K, 5.0, True, seed=500)
            fb = FitBatch([tn] * nm, models, n, lr=synth.fit_rates(W, H), tile=16)
            fb.capture(chunk)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            for _ in range(n // chunk):
                fb.graph.replay()
            e[1].record()
            y = fb.render_mean()
            e[2].record()
            torch.cuda.synchronize()
            assert fb.status_code() == 0
            rows.append({"noise_var": var, "models": nm, "psnr_noisy_db": psnr(tn, c),
                         "psnr_db": psnr(y, c), "fit_s": e[0].elapsed_time(e[1]) / 1e3,
                         "fuse_ms": e[1].elapsed_time(e[2]),
                         "ms_per_iter": e[0].elapsed_time(e[1]) / n})
            del fb, models, y
    print(json.dumps({
        "metric": "MM-RSMoE denoising: PSNR of the fused image and GPU time of H fits + fusion",
        "mode": "denoise", "image": f"{W}x{H}x3 synthetic (30 ramp polygons + Perlin 0.1, "
                                    f"clipped to [0,1]) + N(0, var) noise",
        "kernels_per_model": K, "iters": n, "lr": list(synth.fit_rates(W, H)), "tile": 16,
        "rows": rows, "data": "synthetic", "dtype": "f32",
    }), flush=True)


def run_quality(args):
    """Fit quality and speed on the paper-shaped workloads: the 128x128 grey
    image (K = 256, constant experts, 100 iterations at lr 1e-2) and the
    512x512 RGB image (K = 16384, linear experts, 2000 and 10000 iterations
    at the paper's rates) as softmax-gated R-SMoE (Eq. 4) and with learned gate
    weights pi_k; then softmax gates against the unnormalised RBF sum of
    Eq. 1 (the Gaussian-splatting regression the paper compares against)
    with constant experts at equal kernel counts.  PSNR against the target; iterations/s from CUDA events
    over graph replays of 25 iterations."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import api, build, synth
    from paper_2510_05814_gb300.fit import FitBatch
    build.build()

    def psnr(y, t):
        mse = float(((y.clamp(0.0, 1.0) - t) ** 2).mean())
        return 10.0 * np.log10(1.0 / mse)

    def one(name, target, params, iters, lr, rbf=False, pi=False):
        C, H, W = target.shape
        t = torch.tensor(target, device="cuda")
        if pi:
            params = synth.Params(params.mu, params.chol, params.ea, params.eW,
                                  np.zeros(params.K, np.float32))
        p = api.SMoEParams.from_numpy(params)
        fb = FitBatch([t], [p], iters, lr=lr, tile=16, rbf=rbf)
        chunk = 25 if iters % 25 == 0 else 1
        fb.capture(chunk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        # graph replays; a pair-buffer overflow (the lists grow as kernels
        # widen) grows the buffer and resumes, inside the timed region
        fb.run(iters, graph_iters=chunk, check_every=max(chunk, iters // 4))
        e1.record()
        torch.cuda.synchronize()
        y, inv, _ = api.render(fb.params_of(0), W, H, tile=16, rbf=rbf)
        s = e0.elapsed_time(e1) / 1e3
        return {"run": name, "image": f"{W}x{H}x{C}", "K": params.K, "iters": iters,
                "gate": "rbf (Eq. 1)" if rbf else ("softmax, learned pi" if pi else "softmax"),
                "lr": list(lr), "psnr_db": psnr(y, t),
                "uncovered_px": float((inv == 0).float().mean()),   # D = 0: y = 0, no gradient
                "iters_per_s": iters / s, "s": s}

    rows = []
    g = synth.plain_gray_128()
    # workload 1 gives one rate, 1e-2, for every group; its centre rate is
    # read in pixels like the paper's (synth.fit_rates)
    lr1 = (1e-2 / 128, 1e-2 / 128, 1e-2, 1e-2, 1e-2)
    rows.append(one("config 1: grey 128^2", g.target, g.params, 100, lr1))
    c2 = synth.rgb_512()
    lr2 = synth.fit_rates(512, 512)
    rows.append(one("config 2: RGB 512^2", c2.target, c2.params, 2000, lr2))
    rows.append(one("config 2, learned pi", c2.target, c2.params, 2000,
                    synth.fit_rates(512, 512, lr_pi=1e-2), pi=True))
    rows.append(one("config 2, 10000 iterations", c2.target, c2.params, 10000, lr2))
    # Sparsity comparison of Sec. II / VII: constant experts (the colours of a
    # Gaussian-splatting model), softmax gates against the RBF sum at equal
    # kernel counts, the paper's protocol of 10000 Adam iterations at its
    # rates.  The RBF colours start at target x spacing^2 / (2 pi sigma^2),
    # the inverse of the kernels' mean overlap on the grid, so that both
    # start near the target.
    for K in (4096, 16384):
        pk = synth.init_params(c2.target, K, 5.0, False, 2)
        overlap = (512 * 512 / K) / (2 * np.pi * 25.0)
        pr = synth.Params(pk.mu, pk.chol, (pk.ea * min(1.0, overlap)).astype(np.float32), None)
        rows.append(one(f"sparsity K={K}, SMoE", c2.target, pk, 10000, lr2))
        rows.append(one(f"sparsity K={K}, RBF", c2.target, pr, 10000, lr2, rbf=True))
    print(json.dumps({"metric": "fit PSNR and iterations/s on the paper-shaped workloads",
                      "mode": "quality", "rows": rows, "data": "synthetic", "dtype": "f32"}),
          flush=True)


def run_serve(args):
    """Poisson arrivals (50 req/s): fit requests (ragged sizes, half of them
    denoising with N(0, 0.05) noise as MM-RSMoE with --mm-models models,
    `iters` Adam steps) and render requests (a fitted model at 1-4x);
    continuous batching vs one request at a time."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import build, serve
    build.build()
    sizes = None
    if args.fit_size:
        W, H = (int(v) for v in args.fit_size.lower().split("x"))
        sizes = [(W, H)]
    reqs = serve.poisson_workload(args.fits, args.renders, args.rate, iters=args.iters,
                                  sizes=sizes, mm_models=args.mm_models)
    srv = serve.Server(args.budget_gb * (1 << 30), chunk=25,
                       max_pixels=int(args.max_mpx * 1e6) if args.max_mpx else None)
    t0 = time.perf_counter()
    res_b = srv.run(reqs, realtime=True)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_p = serve.serve_plain(reqs, realtime=True)
    t_p = time.perf_counter() - t0
    byid = lambda rs: {r.rid: r for r in rs}
    rb, rp = byid(res_b), byid(res_p)
    fits = [r.rid for r in reqs if isinstance(r, serve.FitRequest)]
    dpsnr = max(abs(rb[i].psnr - rp[i].psnr) for i in fits)
    split = lambda rs, k: [r for r in rs if r.kind == k]
    print(json.dumps({
        "metric": "serving: fit/render request latency p50/p99 and throughput, continuous "
                  "batching vs one request at a time", "mode": "serve",
        "mm_models_per_denoising_request": args.mm_models,
        "fit_size": args.fit_size or "ragged 128x96 .. 1920x1080",
        "max_mpx_in_flight": args.max_mpx or None,
        "requests": len(reqs), "fits": len(fits), "rate_per_s": args.rate, "iters": args.iters,
        "batched": {"wall_s": t_b, "req_per_s": len(reqs) / t_b,
                    "all": serve.latency_stats(res_b), "fit": serve.latency_stats(split(res_b, "fit")),
                    "render": serve.latency_stats(split(res_b, "render"))},
        "plain": {"wall_s": t_p, "req_per_s": len(reqs) / t_p,
                  "all": serve.latency_stats(res_p), "fit": serve.latency_stats(split(res_p, "fit")),
                  "render": serve.latency_stats(split(res_p, "render"))},
        "max_abs_psnr_diff_db": float(dpsnr),
        "psnr_mean_db": float(np.mean([rb[i].psnr for i in fits])),
        "data": "synthetic", "dtype": "f32",
    }), flush=True)


def _ragged_one(W, H, i):
    """One image of the batched leg and its initial kernels (runs in a
    spawned host process)."""
    from paper_2510_05814_gb300 import synth
    t = synth.polygon_image(W, H, 3, 40, 400 + i, texture_amp=0.1)
    return t, synth.init_params(t, (W * H) // 16, 5.0, True, 400 + i)


def _workload_2048(seed):
    from paper_2510_05814_gb300 import synth
    return synth.rgb_2048(seed=seed)


def host_inputs(seed, n_ragged):
    """The seeded inputs of the default run, drawn on the host cores in a
    spawned process pool before this process touches the GPU: the 2048^2
    workload and, with n_ragged > 0, the batched leg's ragged images."""
    import multiprocessing as mp
    from paper_2510_05814_gb300 import synth
    sizes = synth.ragged_sizes(n_ragged, 4) if n_ragged else []
    ctx = mp.get_context("spawn")
    procs = max(1, min(len(sizes) + 1, os.cpu_count() or 1))
    with ctx.Pool(procs) as pool:
        wl = pool.apply_async(_workload_2048, (seed,))
        imgs = pool.starmap(_ragged_one, [(W, H, i) for i, (W, H) in enumerate(sizes)])
        wl = wl.get()
    return wl, sizes, imgs


def psnr_of_mse(mse):
    import numpy as np
    mse = np.asarray(mse, np.float64)
    return 10.0 * np.log10(1.0 / np.maximum(mse, 1e-300))


def fit_to_psnr_leg(wl, params0, iters, target_db, chunk=25, late_n=20):
    """A whole fit of the 2048^2 workload from its initial kernels, the way a
    caller runs it (FitBatch.run with CUDA-graph replays of `chunk`
    iterations and the spatial re-sort every 25): CUDA events after every
    chunk give the fit's device time at each point of its loss history
    (the MSE of every iteration, before its update).  Returns the wall time,
    the time to the first iteration whose MSE reaches `target_db` PSNR, and
    the PSNR of the final model rendered and clamped to [0, 1].  Then, outside
    the fit's timing, `late_n` more iterations run phase by phase (L2 flushed
    before each): the step's phases at the end of a fit, where the kernels
    have stretched and the lists grown."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import api, synth
    from paper_2510_05814_gb300.fit import FitBatch
    C, H, W = wl.target.shape
    tgt = torch.tensor(wl.target, device="cuda")
    cap = None
    for _attempt in range(4):
        fb = FitBatch([tgt], [params0.clone()], iters + late_n, lr=synth.fit_rates(W, H),
                      tile=wl.tile, qmax=wl.qmax, hist=iters + late_n,
                      reorder_every=REORDER_EVERY, pair_cap=cap)
        fb.capture(chunk)
        n_chunks = iters // chunk
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_chunks + 1)]
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        ev[0].record()
        for c in range(n_chunks):
            fb.graph.replay()
            fb.reorder()
            ev[c + 1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - h0
        if fb.status_code() == 0:
            break
        cap = 2 * fb.pair_cap                     # the lists outgrew the buffer: rerun larger
    assert fb.status_code() == 0
    t_at = np.array([ev[0].elapsed_time(e) / 1e3 for e in ev[1:]])
    ps = psnr_of_mse(fb.losses()[0][: n_chunks * chunk])
    hit = np.nonzero(ps >= target_db)[0]
    t_hit = float(t_at[hit[0] // chunk]) if len(hit) else None
    y, inv, _ = api.render(fb.params_of(0), W, H, tile=wl.tile, qmax=wl.qmax)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.smoe_sq_error(y, tgt, out, clamp=True)
    final = float(psnr_of_mse(out.item() / y.numel()))
    late = None
    if late_n:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        pev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(late_n)]
        for e in pev:
            flush.zero_()
            e[0].record()
            fb.phase(0)
            e[1].record()
            fb.phase(1)
            e[2].record()
            fb.phase(2)
            e[3].record()
        torch.cuda.synchronize()
        assert fb.status_code() == 0
        med = lambda a, b: statistics.median(e[a].elapsed_time(e[b]) for e in pev)
        late = {"after_iter": n_chunks * chunk, "bin": med(0, 1), "fused_tiles": med(1, 2),
                "adam": med(2, 3), "steps": late_n,
                "how": "the fit's next iterations, launched phase by phase (no graph), CUDA "
                       "events between the phases, L2 flushed before each; median"}
    marks = [0, 100, 300, 1000, 2000, 5000, n_chunks * chunk - 1]
    return {"iters": n_chunks * chunk, "lr": list(synth.fit_rates(W, H)),
            "device_s": float(t_at[-1]), "wall_s": wall,
            "iters_per_s": n_chunks * chunk / float(t_at[-1]),
            "target_psnr_db": target_db, "s_to_target": t_hit,
            "iters_to_target": int(hit[0]) + 1 if len(hit) else None,
            "psnr_final_db": final, "psnr_max_db": float(ps.max()), "late_phases_ms": late,
            "uncovered_px": float((inv == 0).float().mean()),
            "psnr_db_at": {int(i): round(float(ps[i]), 3) for i in marks if i < len(ps)},
            "how": f"fresh fit from the initial kernels, graph replays of {chunk} iterations, "
                   f"re-sort every {REORDER_EVERY}; PSNR per iteration from the fit's own MSE "
                   "(before that iteration's update); final PSNR on the render clamped to [0,1]"}


def batched_leg(sizes, imgs, iters, chunk=25):
    """The ragged batch of 64 images (128x96 .. 1920x1080, K = pixels/16)
    fitted as one batch (one launch per phase per iteration over the ragged
    tile table, graph replays) against the same fits run one image per
    launch, one after another.  Deterministic accumulation, so every image's
    fit is the same bit for bit in both arms (equal PSNR).  All requests are
    present at t = 0: a batched image's latency is the batch's time; a plain
    image's latency is the time until its own fit ends."""
    import numpy as np
    import torch
    from paper_2510_05814_gb300 import api, synth
    from paper_2510_05814_gb300.fit import FitBatch
    T = 16
    targets = [torch.tensor(t, device="cuda") for t, _ in imgs]
    params = [api.SMoEParams.from_numpy(p) for _, p in imgs]
    lrs = [synth.fit_rates(W, H) for W, H in sizes]
    pairs = 0
    for (W, H), p in zip(sizes, params):
        r = api.Rasterizer(api.RasterDesc(W, H, 3, T, True), p.K).bin(p)
        pairs += evaluated_pairs(r.tile_off.cpu().numpy(), W, H, T)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fb = FitBatch(targets, [p.clone() for p in params], iters, lr=lrs, tile=T,
                  deterministic=True, hist=iters, pair_slack=3.0)
    fb.capture(chunk)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(iters // chunk):
        fb.graph.replay()
    e1.record()
    torch.cuda.synchronize()
    assert fb.status_code() == 0
    t_b = e0.elapsed_time(e1) / 1e3
    mse_b = fb.losses()[:, iters - 1]
    del fb
    t_p, lat_p, mse_p = 0.0, [], []
    for b in range(len(targets)):
        one = FitBatch([targets[b]], [params[b].clone()], iters, lr=lrs[b], tile=T,
                       deterministic=True, hist=iters, pair_slack=3.0)
        one.capture(chunk)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(iters // chunk):
            one.graph.replay()
        e1.record()
        torch.cuda.synchronize()
        assert one.status_code() == 0
        t_p += e0.elapsed_time(e1) / 1e3
        lat_p.append(t_p)
        mse_p.append(one.losses()[0][iters - 1])
        del one
    dpsnr = float(np.max(np.abs(psnr_of_mse(mse_b) - psnr_of_mse(np.array(mse_p)))))
    pct = lambda xs, q: float(np.percentile(xs, q))
    return {"images": len(targets), "iters": iters, "tile": T, "launch": "grid, deterministic",
            "pixels": int(sum(W * H for W, H in sizes)), "kernels": int(sum(p.K for p in params)),
            "pairs_per_iter": int(pairs),
            "batched": {"s": t_b, "value": pairs * iters / t_b / 1e9,
                        "latency_p50_s": t_b, "latency_p99_s": t_b},
            "plain": {"s": t_p, "value": pairs * iters / t_p / 1e9,
                      "latency_p50_s": pct(lat_p, 50), "latency_p99_s": pct(lat_p, 99)},
            "throughput_ratio": t_p / t_b,
            "p99_latency_ratio": pct(lat_p, 99) / t_b,
            "max_abs_psnr_diff_db": dpsnr,
            "psnr_mean_db": float(np.mean(psnr_of_mse(mse_b))),
            "unit": UNIT,
            "how": f"{iters} iterations as graph replays of {chunk}; requests all at t = 0; "
                   "plain images run one after another in the given order"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-crop", type=int, default=512)
    ap.add_argument("--ref-crop", type=int, default=0,
                    help="reference arm crop side (0: sized so the run takes about 90 s)")
    ap.add_argument("--binned-crop", type=int, default=1024)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--fit-iters", type=int, default=10000,
                    help="iterations of the fit-to-PSNR leg (0: skip)")
    ap.add_argument("--fit-target-db", type=float, default=FIT_TARGET_DB)
    ap.add_argument("--batched-images", type=int, default=64,
                    help="images of the batched-vs-plain leg (0: skip)")
    ap.add_argument("--batched-iters", type=int, default=25)
    ap.add_argument("--serve-fits", type=int, default=12,
                    help="fit requests of the serving leg (as many renders; 0: skip)")
    ap.add_argument("--serve-iters", type=int, default=200)
    ap.add_argument("--mode", default="fit",
                    choices=["fit", "batched", "serve", "denoise", "quality"],
                    help="fit: the 2048^2 fit step (default); batched: 64 ragged images; "
                         "serve: Poisson request stream; denoise: MM-RSMoE; quality: PSNR "
                         "and iterations/s of configs 1-2, learned pi and the RBF mode")
    ap.add_argument("--models", type=int, nargs="+", default=[1, 8, 16, 64],
                    help="denoise: model counts H")
    ap.add_argument("--images", type=int, default=64)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--fits", type=int, default=40)
    ap.add_argument("--renders", type=int, default=40)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--max-mpx", type=float, default=SERVE_MAX_MPX,
                    help="serve: cap on megapixels (x models) in flight (0: HBM budget only)")
    ap.add_argument("--fit-size", default=None,
                    help="serve: every fit request at this WxH (e.g. 2048x2048) instead of the "
                         "ragged sizes")
    ap.add_argument("--mm-models", type=int, default=4,
                    help="serve: MM-RSMoE models per denoising request")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        args.iters = args.iters or 1000
        return run_batched(args)
    if args.mode == "serve":
        args.iters = args.iters or 500
        return run_serve(args)
    if args.mode == "quality":
        return run_quality(args)
    if args.mode == "denoise":
        args.iters = args.iters or 2000
        return run_denoise(args)
    return run_fit(args)


def serving_leg(rimgs, n_fit, iters, mm_models=4, rate=50.0):
    """Continuous batching against one request at a time on a short Poisson
    stream: n_fit fit requests on the batched leg's ragged images (half of
    them denoising, N(0, 0.05) added, as MM-RSMoE with mm_models models) and
    as many render requests at 1-4x; the server admits by a 150 GB budget and
    SERVE_MAX_MPX megapixels in flight (paper_2510_05814_gb300.serve)."""
    import numpy as np
    from paper_2510_05814_gb300 import serve
    reqs = serve.poisson_workload(n_fit, n_fit, rate, iters=iters, mm_models=mm_models,
                                  images=[t for t, _ in rimgs[:n_fit]])
    srv = serve.Server(150 * (1 << 30), chunk=25, max_pixels=int(SERVE_MAX_MPX * 1e6))
    t0 = time.perf_counter()
    res_b = srv.run(reqs, realtime=True)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_p = serve.serve_plain(reqs, realtime=True)
    t_p = time.perf_counter() - t0
    byid = lambda rs: {r.rid: r for r in rs}
    rb, rp = byid(res_b), byid(res_p)
    fits = [r.rid for r in reqs if isinstance(r, serve.FitRequest)]
    sb, sp = serve.latency_stats(res_b), serve.latency_stats(res_p)
    return {"requests": len(reqs), "fits": len(fits), "iters": iters, "rate_per_s": rate,
            "mm_models_per_denoising_request": mm_models,
            "batched": {"wall_s": t_b, "req_per_s": len(reqs) / t_b, **sb},
            "plain": {"wall_s": t_p, "req_per_s": len(reqs) / t_p, **sp},
            "throughput_ratio": t_p / t_b, "p99_latency_ratio": sp["p99_s"] / sb["p99_s"],
            "max_abs_psnr_diff_db": float(max(abs(rb[i].psnr - rp[i].psnr) for i in fits)),
            "psnr_mean_db": float(np.mean([rb[i].psnr for i in fits])),
            "how": "Poisson arrivals; the fit requests use the batched leg's first images; "
                   "latency = result on the host - arrival; continuous batching vs one "
                   "request at a time, one image per launch"}


def cpu_legs(wl, args):
    """The oracle timed on the host cores (the CPU baseline) and the labelled
    binned CPU baseline, each on a bounded crop of the workload."""
    pairs_c, s_c, thr, kc = oracle_sample(wl, args.cpu_crop)
    cpu = {"value": pairs_c / s_c / 1e9, "unit": UNIT, "cores": thr, "kind": "oracle",
           "sample": f"{args.cpu_crop}x{args.cpu_crop} centre crop of the workload with its "
                     f"{kc} kernels; one dense forward + MSE backward ({s_c:.1f} s)"}
    pairs_b, s_b, thr_b, kb = binned_sample(wl, args.binned_crop)
    cpu_binned = {"value": pairs_b / s_b / 1e9, "unit": UNIT, "cores": thr_b,
                  "kind": "binned oracle (CPU baseline, labelled)",
                  "sample": f"{args.binned_crop}x{args.binned_crop} centre crop with its {kb} "
                            f"kernels; binning + per-tile forward, MSE, backward in FP64 "
                            f"({s_b:.1f} s)"}
    return cpu, cpu_binned


def roofline_fields(inrange, listed, tile_s, rates, sms, fallback_mhz, ncu):
    """The line's roofline objects for the fused tile kernel: `roofline` (the
    FP32 pipe on the method's in-range work), `roofline_ex2` (in-range and
    listed pairs) and `fp32_executed` (ncu-counted work, or None).
    inrange / listed: pairs of one launch; tile_s: its mean CUDA-event time;
    rates: the live issue-rate measurements (dicts with ex2, ffma and
    clock_mhz), possibly empty; ncu: the profiled figures or None."""
    clk = statistics.mean(r["clock_mhz"] for r in rates) if rates else fallback_mhz
    mufu = statistics.mean(r["ex2"] for r in rates) if rates else MUFU_PER_CLK_PER_SM
    ffma = statistics.mean(r["ffma"] for r in rates) if rates else 128.0
    ex2_peak = mufu * sms * clk * 1e6                              # ex2 / s
    fma_peak = ffma * sms * clk * 1e6                              # FP32 lane-ops / s
    fma_alg = FP32_OPS_PER_PAIR * inrange                          # per launch
    basis = (f"{sms} SMs x {clk:.0f} MHz (SM clock measured live by libsmoe_rates before "
             "and after the timed region)" if rates else f"{sms} SMs x {clk:.0f} MHz (fallback)")
    ex2 = lambda pairs: {"achieved": 2.0 * pairs / tile_s / 1e9, "peak": ex2_peak / 1e9,
                         "unit": "Gex2/s", "frac": 2.0 * pairs / tile_s / ex2_peak}
    out = {
        "roofline": {"bound": "alu", "kernel": "k_fit_tile (fused fwd+MSE+bwd)",
                     "achieved": fma_alg / tile_s / 1e12, "peak": fma_peak / 1e12,
                     "unit": "T FP32 lane-ops/s", "frac": fma_alg / tile_s / fma_peak,
                     "traffic": ncu["bytes_per_launch"] if ncu else None,
                     "per_unit": {"unit": "in-range (q <= q_max) fwd+bwd pixel-kernel pair",
                                  "fp32_lane_ops": FP32_OPS_PER_PAIR,
                                  "units_per_launch": int(inrange),
                                  "launch_ms": tile_s * 1e3},
                     "peak_basis": f"{ffma:.1f} FFMA lanes/clk/SM (libsmoe_rates, live) x "
                                   + basis,
                     "issue_rates_per_clk_per_sm": list(rates)},
        "roofline_ex2": {
            "in_range": dict(ex2(inrange), basis="2 ex2 per in-range fwd+bwd pair"),
            "listed": dict(ex2(listed), basis="2 ex2 per listed pair (sum over tiles of pixels "
                                              "x list length): the metric's pair count"),
            "peak_basis": f"{mufu:.1f} ex2 lanes/clk/SM (libsmoe_rates, live) x " + basis},
        "fp32_executed": None,
    }
    if ncu and ncu.get("fp32_lane_ops"):
        out["fp32_executed"] = {
            "lane_ops_per_launch": ncu["fp32_lane_ops"],
            "per_in_range_pair": ncu["fp32_lane_ops"] / inrange,
            "achieved": ncu["fp32_lane_ops"] / tile_s / 1e12, "unit": "T FP32 lane-ops/s",
            "frac": ncu["fp32_lane_ops"] / tile_s / fma_peak,
            "source": "ncu sass thread-instruction counts of one launch (FFMA + FADD + "
                      "FMUL + 2 x (FFMA2 + FADD2 + FMUL2)), profiles/",
            "pipes": {k: ncu[k] for k in ("fma_pipe_active", "issue_active", "xu_active")}}
    return out


def run_fit(args):
    import numpy as np
    # host inputs first: the pool is spawned before this process uses the GPU
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    n_ragged = args.batched_images if (world == 1 and args.batched_images) else 0
    if world == 1:
        wl, rsizes, rimgs = host_inputs(replica_seed(rank), n_ragged)
    else:
        from paper_2510_05814_gb300 import synth
        wl, rsizes, rimgs = synth.rgb_2048(seed=replica_seed(rank)), [], []

    import torch
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_2510_05814_gb300 import build, synth
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2510_05814_gb300 import api
    from paper_2510_05814_gb300.fit import FitBatch

    C, H, W = wl.target.shape
    T = wl.tile
    tgt = torch.tensor(wl.target, device="cuda")
    params0 = api.SMoEParams.from_numpy(wl.params)
    params = params0.clone()
    lr = synth.fit_rates(W, H)
    n_phase = min(args.steps, 200)               # eager steps timed phase by phase
    total_iters = args.warmup + 2 * args.steps + n_phase + 5
    fb = FitBatch([tgt], [params], total_iters, lr=lr, tile=T, qmax=wl.qmax,
                  hist=total_iters, reorder_every=REORDER_EVERY)
    desc = api.RasterDesc(W, H, C, T, True, wl.qmax, 1.0)

    def pairs_now():
        r = api.Rasterizer(desc, params.K, pair_cap=fb.pair_cap).bin(fb.params_of(0))
        return (evaluated_pairs(r.tile_off.cpu().numpy(), W, H, T), int(r.n_pairs.item()),
                r.count_inrange())

    for _ in range(args.warmup):
        fb.launch(1)
    torch.cuda.synchronize()
    assert fb.status_code() == 0
    pairs0, lists0, inrange0 = pairs_now()
    rates0 = issue_rates()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # The step as FitBatch.run(graph_iters=...) runs it: one CUDA-graph replay
    # of a whole fit iteration (its 10 kernels), L2 flushed before each step.
    graph = fb.capture(1)
    graph.replay()                              # one untimed replay
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_phase)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for s in range(args.steps):
            flush.zero_()                       # L2 flush outside the timed region
            ev[s][0].record(stream)
            graph.replay()
            if (s + 1) % REORDER_EVERY == 0:    # the periodic spatial re-sort, timed with its step
                fb.reorder()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    rates1 = issue_rates()
    if world > 1:
        torch.distributed.barrier()
    # the same step launched phase by phase (eager), for the breakdown
    rev = []
    for s in range(n_phase):
        flush.zero_()
        e = pev[s]
        e[0].record(stream)
        fb.phase(0)
        e[1].record(stream)
        fb.phase(1)
        e[2].record(stream)
        fb.phase(2)
        e[3].record(stream)
        if (s + 1) % REORDER_EVERY == 0:
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            fb.reorder()
            r1.record(stream)
            rev.append((r0, r1))
    torch.cuda.synchronize()
    st = fb.status_code()
    assert st == 0, f"fit status {st}"
    bin_ms = [e[0].elapsed_time(e[1]) for e in pev]
    tile_ms = [e[1].elapsed_time(e[2]) for e in pev]
    adam_ms = [e[2].elapsed_time(e[3]) for e in pev]
    eager_ms = [e[0].elapsed_time(e[3]) for e in pev]
    reorder_ms = [a.elapsed_time(b) for a, b in rev]
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    pairs1, lists1, inrange1 = pairs_now()
    pairs_step = 0.5 * (pairs0 + pairs1)
    inrange_step = 0.5 * (inrange0 + inrange1)
    tot_s = sum(step_ms) / 1e3

    # End to end through the public API, as a caller resumes a fit: inside
    # the timed region the target goes host -> device once (pinned memory),
    # the steps run as graph replays (with the periodic re-sort), and the
    # fitted parameters come back to pinned host memory in the caller's
    # kernel order (params_of into preallocated buffers).
    host_t = torch.empty_like(tgt, device="cpu").pin_memory()
    host_t.copy_(tgt.cpu())
    gathered = params.zeros_like()
    host_p = [torch.empty_like(t, device="cpu").pin_memory() for t in gathered.tensors()]
    step_graph = fb.capture(1)
    fb.params_of(0, out=gathered)               # warm the gather path outside the region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fb.targets[0].copy_(host_t, non_blocking=True)
    for s in range(args.steps):
        step_graph.replay()
        if (s + 1) % REORDER_EVERY == 0:
            fb.reorder()
    fb.params_of(0, out=gathered)
    for h, d in zip(host_p, gathered.tensors()):
        h.copy_(d, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    assert fb.status_code() == 0
    h2d = int(tgt.numel() * 4)
    d2h = int(sum(t.numel() for t in gathered.tensors()) * 4)
    del fb, graph, step_graph

    # super-resolution render of the initial model at 2x (4096 x 4096)
    sr_desc = api.RasterDesc(2 * W, 2 * H, C, T, True, wl.qmax, 2.0)
    sr = api.Rasterizer(sr_desc, params.K, pair_cap=8 * lists1).bin(params)
    y_sr, inv_sr = sr.render()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    f0.record(stream)
    sr.bin(params, check_capacity=False)
    sr.render(y_sr, inv_sr)
    f1.record(stream)
    torch.cuda.synchronize()
    sr_ms = f0.elapsed_time(f1)
    sr_pairs = evaluated_pairs(sr.tile_off.cpu().numpy(), 2 * W, 2 * H, T)
    del sr, y_sr, inv_sr

    # irregular-raster resampling at 10x magnification: a 205 x 205 crop of
    # the model on a jittered 10x raster (4.2 M points)
    g10 = (np.arange(2050) + 0.5) / 10.0
    pts = np.stack(np.meshgrid(900.0 + g10, 900.0 + g10), -1).reshape(-1, 2)
    pts += np.random.default_rng(11).uniform(-0.04, 0.04, pts.shape)
    pts = torch.tensor(pts, dtype=torch.float32, device="cuda")
    rp = api.Rasterizer(desc, params.K, pair_cap=2 * lists1).bin(params)
    yp, ip = rp.render_points(pts)
    torch.cuda.synchronize()
    f0.record(stream)
    rp.render_points(pts, yp, ip)
    f1.record(stream)
    torch.cuda.synchronize()
    pts_ms = f0.elapsed_time(f1)
    del rp, yp, ip

    # job-wide aggregation (max time over ranks, summed work)
    tot_s, work, e2e_s = aggregate(tot_s, pairs_step * args.steps, e2e_s, world)
    value = work / tot_s / 1e9
    e2e_value = work / e2e_s / 1e9

    def leg(fn, *a):
        """An auxiliary measurement: its failure is reported in its key and
        does not cost the line its headline figures."""
        try:
            return fn(*a)
        except Exception as exc:              # noqa: BLE001
            return {"error": f"{type(exc).__name__}: {exc}"}

    fit_leg = batched = serving = None
    if rank == 0 and world == 1 and args.fit_iters:
        fit_leg = leg(fit_to_psnr_leg, wl, params0, args.fit_iters, args.fit_target_db)
    if rank == 0 and world == 1 and rsizes:
        batched = leg(batched_leg, rsizes, rimgs, args.batched_iters)
        if args.serve_fits:
            serving = leg(serving_leg, rimgs, args.serve_fits, args.serve_iters)

    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    rl = [r for r in (rates0, rates1) if r]
    tile_s = statistics.mean(tile_ms) / 1e3
    ncu = None
    if NCU["render_cu_code_sha256"] and NCU["render_cu_code_sha256"] == code_sha256(
            os.path.join(ROOT, "paper_2510_05814_gb300", "csrc", "render.cu")):
        ncu = NCU
    roof = roofline_fields(inrange_step, pairs_step, tile_s, rl, sms,
                           clocks.get("sm_mhz") or 2070.0, ncu)

    cpu = cpu_binned = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r = leg(cpu_legs, wl, args)
        cpu, cpu_binned = (r, None) if isinstance(r, dict) else r

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "image": f"{W}x{H}x{C}", "K": params.K, "tile": T,
                       "lr": list(lr),
                       "l2": "flushed (256 MiB write, untimed) before every timed step",
                       "launch": "one CUDA-graph replay of the whole fit iteration per step "
                                 "(the FitBatch.run(graph_iters=...) path)",
                       "reorder_every": REORDER_EVERY,
                       "parallelism": f"replicas x{world}",
                       "pairs_per_step": int(pairs_step), "list_pairs": int(lists1),
                       "in_range_pairs_per_step": int(inrange_step)},
            # the binding resource of the fused tile kernel: the FP32 pipe, on
            # the method's work (pairs inside the cutoff); ex2 and the executed work beside it
            **roof,
            "value_fwd_bwd_only": pairs_step / tile_s / 1e9,
            # pairs with q <= q_max (the ones that contribute) per second of the
            # fused tile kernel, and their share of the listed pairs
            "in_range": {"Gpairs_per_s": inrange_step / tile_s / 1e9,
                         "fraction_of_listed": inrange_step / pairs_step},
            "phases_ms": {"bin": statistics.mean(bin_ms), "fused_tiles": statistics.mean(tile_ms),
                          "adam": statistics.mean(adam_ms), "eager_step": statistics.mean(eager_ms),
                          "reorder_per_call": statistics.mean(reorder_ms) if reorder_ms else None,
                          "steps": n_phase,
                          "how": "the same step launched phase by phase (no graph), "
                                 "CUDA events between the phases"},
            "fit_iters_per_s": args.steps / tot_s,
            # the fit wall-time at 2048^2: a fresh fit to the stated PSNR, and the
            # PSNR the paper's 10000 iterations reach
            "fit_wall_s_to_psnr": None if fit_leg is None or "error" in fit_leg else {
                "target_psnr_db": fit_leg["target_psnr_db"], "s": fit_leg["s_to_target"],
                "iters": fit_leg["iters_to_target"], "fit_s": fit_leg["device_s"],
                "fit_iters": fit_leg["iters"], "psnr_final_db": fit_leg["psnr_final_db"]},
            "fit_to_psnr": fit_leg,
            "batched_vs_plain": batched,
            "serving": serving,
            "sr_render_2x": {"ms": sr_ms, "pairs": sr_pairs, "out": f"{2 * W}x{2 * H}",
                             "Gpairs_per_s": sr_pairs / sr_ms / 1e6,
                             "model": "the initial kernels"},
            "resample_points_10x": {"points": int(pts.shape[0]), "ms": pts_ms,
                                    "Gpoints_per_s": pts.shape[0] / pts_ms / 1e6,
                                    "raster": "jittered 10x raster over a 205x205 crop"},
            "cpu_baseline": cpu,
            "cpu_baseline_binned": cpu_binned,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps,
                    "h2d_bytes": h2d, "d2h_bytes": d2h,
                    "copies": "the target host -> device once (pinned), the fitted parameters "
                              "(14 floats per kernel, caller's order) device -> host once, "
                              "both inside the timed region",
                    "launch": "one CUDA-graph replay per step (FitBatch.capture), the periodic "
                              "re-sort, params_of for the caller's order",
                    "l2": "not flushed: steps back to back, as a caller runs them"},
            "gpu_launches": KERNELS_PER_STEP * args.steps
                            + REORDER_KERNELS * (args.steps // REORDER_EVERY),
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
