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
FP32_OPS_PER_PAIR = 67            # algorithmic FP32 lane ops per fwd+bwd pair, RGB linear
# Kernels launched by one fit step: binning (bbox, scan reduce/top/down,
# scatter, warp sort, long-list sort), the fused tile kernel, fused Adam.
KERNELS_PER_STEP = 9
# The fit re-sorts its kernels spatially every this many steps (FitBatch
# reorder_every; smoe_fit_reorder, 15 kernels); the timed steps include it.
REORDER_EVERY = 25
REORDER_KERNELS = 15
# From one ncu capture of the fused tile kernel on this workload (profiles/):
# DRAM bytes per launch and pipe utilisation; valid only while render.cu's
# code (comments and whitespace aside) is the code that was profiled.
NCU = {"render_cu_code_sha256": "023a846244615376ce0e0d757481649c77f809707901515cfd6718cc83e15ca3",
       "bytes_per_launch": 105.25824e6, "fma_pipe_active": 0.610, "issue_active": 0.600,
       "xu_active": 0.129}


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
    lr = synth.PAPER_LR
    tr = autotune.tune(targets, params, lr, tiles=(8, 16, 32), persistent=(False, True))
    n = args.iters
    # batched: graph of `chunk` iterations replayed
    # both arms re-sort their kernels spatially after every graph replay
    # (FitBatch reorder_every; the first, untimed call captures its graph)
    chunk = 25
    fb = FitBatch(targets, [p.clone() for p in params], n, lr=lr, tile=tr.tile,
                  persistent=tr.persistent, deterministic=True, reorder_every=chunk)
    fb.capture(chunk)
    fb.reorder()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n // chunk):
        fb.graph.replay()
        fb.reorder()
    e1.record()
    torch.cuda.synchronize()
    assert fb.status_code() == 0
    t_batched = e0.elapsed_time(e1) / 1e3
    # plain: each image alone, one image per launch, same iterations
    t_plain = 0.0
    psnr_b, psnr_p, lat_plain = [], [], []
    for b in range(len(targets)):
        one = FitBatch([targets[b]], [params[b].clone()], n, lr=lr, tile=tr.tile,
                       deterministic=True, reorder_every=chunk)
        one.capture(chunk)
        one.reorder()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n // chunk):
            one.graph.replay()
            one.reorder()
        e1.record()
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1) / 1e3
        lat_plain.append(t_plain)
        assert one.status_code() == 0
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
        "reorder_every": chunk,
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
            fb = FitBatch([tn] * nm, models, n, lr=synth.PAPER_LR, tile=16)
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
        "kernels_per_model": K, "iters": n, "lr": list(synth.PAPER_LR), "tile": 16,
        "rows": rows, "data": "synthetic", "dtype": "f32",
    }), flush=True)


def run_quality(args):
    """Fit quality and speed on the paper-shaped workloads: the 128x128 grey
    image (K = 256, constant experts, 100 iterations at lr 1e-2) and the
    512x512 RGB image (K = 16384, linear experts, 2000 iterations at the
    paper's rates) as softmax-gated R-SMoE (Eq. 4) and with learned gate
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
    rows.append(one("config 1: grey 128^2", g.target, g.params, 100, (1e-2,) * 5))
    c2 = synth.rgb_512()
    lr_pi = tuple(synth.PAPER_LR) + (1e-2,)
    rows.append(one("config 2: RGB 512^2", c2.target, c2.params, 2000, synth.PAPER_LR))
    rows.append(one("config 2, learned pi", c2.target, c2.params, 2000, lr_pi, pi=True))
    # Sparsity comparison of Sec. II / VII: constant experts (the colours of a
    # Gaussian-splatting model), softmax gates against the RBF sum at equal
    # kernel counts, the paper's protocol of 10000 Adam iterations.  The RBF
    # colours start at target x spacing^2 / (2 pi sigma^2), the inverse of the
    # kernels' mean overlap on the grid, so that both start near the target.
    # The rates: the paper's, and ten times its L / expert rates with a tenth
    # of its centre rate (under the per-pixel cutoff, pixels that no kernel
    # reaches get y = 0 and no gradient; the faster shape rates leave fewer).
    fast = (1e-3, 1e-6, 1e-2, 1e-2, 1e-2)
    for K in (4096, 16384):
        pk = synth.init_params(c2.target, K, 5.0, False, 2)
        overlap = (512 * 512 / K) / (2 * np.pi * 25.0)
        pr = synth.Params(pk.mu, pk.chol, (pk.ea * min(1.0, overlap)).astype(np.float32), None)
        for lr in (synth.PAPER_LR, fast):
            rows.append(one(f"sparsity K={K}, SMoE", c2.target, pk, 10000, lr))
            rows.append(one(f"sparsity K={K}, RBF", c2.target, pr, 10000, lr, rbf=True))
    rows.append(one("config 2, fast rates", c2.target, c2.params, 10000, fast))
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
    reqs = serve.poisson_workload(args.fits, args.renders, args.rate, iters=args.iters,
                                  sizes=None, mm_models=args.mm_models)
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
    ap.add_argument("--max-mpx", type=float, default=16.0,
                    help="serve: cap on megapixels (x models) in flight (0: HBM budget only)")
    ap.add_argument("--mm-models", type=int, default=4,
                    help="serve: MM-RSMoE models per denoising request")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        args.iters = args.iters or 200
        return run_batched(args)
    if args.mode == "serve":
        args.iters = args.iters or 500
        return run_serve(args)
    if args.mode == "quality":
        return run_quality(args)
    if args.mode == "denoise":
        args.iters = args.iters or 2000
        return run_denoise(args)

    import numpy as np
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

    wl = synth.rgb_2048(seed=replica_seed(rank))
    C, H, W = wl.target.shape
    T = wl.tile
    tgt = torch.tensor(wl.target, device="cuda")
    params = api.SMoEParams.from_numpy(wl.params)
    n_phase = min(args.steps, 200)               # eager steps timed phase by phase
    total_iters = args.warmup + 2 * args.steps + n_phase + 5
    fb = FitBatch([tgt], [params], total_iters, lr=synth.PAPER_LR, tile=T, qmax=wl.qmax,
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
    rates = issue_rates()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # The step as FitBatch.run(graph_iters=...) runs it: one CUDA-graph replay
    # of a whole fit iteration (its 9 kernels), L2 flushed before each step.
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

    # end to end through the public API with host buffers: per step the
    # target goes host->device from pinned memory and the loss comes back.
    # The copies run on their own stream into a double buffer, so step s+1's
    # target moves while step s computes; every copy is inside the timed
    # region (the first one starts after e0, the last loss lands before e1).
    host_t = torch.empty_like(tgt, device="cpu").pin_memory()
    host_t.copy_(tgt.cpu())
    host_loss = torch.zeros(1, dtype=torch.float64).pin_memory()
    bufs = [fb.targets[0], torch.empty_like(tgt)]
    cstream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    # one captured iteration per target buffer (the target pointer is part of
    # the captured launches), captured before the timed region
    step_graph = []
    for buf in bufs:
        fb.set_target(0, buf)
        step_graph.append(fb.capture(1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    cstream.wait_event(e0)
    with torch.cuda.stream(cstream):
        bufs[0].copy_(host_t, non_blocking=True)
        ready[0].record(cstream)
    for s in range(args.steps):
        cur, nxt = s % 2, 1 - s % 2
        if s + 1 < args.steps:
            if s >= 1:
                cstream.wait_event(freed[nxt])        # step s-1 is done with that buffer
            with torch.cuda.stream(cstream):
                bufs[nxt].copy_(host_t, non_blocking=True)
                ready[nxt].record(cstream)
        stream.wait_event(ready[cur])
        it = int(args.warmup + 1 + args.steps + n_phase + s)
        step_graph[cur].replay()
        if (s + 1) % REORDER_EVERY == 0:
            fb.reorder()
        freed[cur].record(stream)
        host_loss.copy_(fb.loss[0, it:it + 1], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    fb.set_target(0, bufs[0])
    assert fb.status_code() == 0

    # super-resolution render of the current model at 2x (4096 x 4096)
    sr_desc = api.RasterDesc(2 * W, 2 * H, C, T, True, wl.qmax, 2.0)
    sr = api.Rasterizer(sr_desc, params.K, pair_cap=4 * fb.pair_cap).bin(fb.params_of(0))
    y_sr, inv_sr = sr.render()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    f0.record(stream)
    sr.bin(fb.params_of(0), check_capacity=False)
    sr.render(y_sr, inv_sr)
    f1.record(stream)
    torch.cuda.synchronize()
    sr_ms = f0.elapsed_time(f1)
    sr_pairs = evaluated_pairs(sr.tile_off.cpu().numpy(), 2 * W, 2 * H, T)

    # irregular-raster resampling at 10x magnification: a 205 x 205 crop of
    # the current model on a jittered 10x raster (4.2 M points)
    g10 = (np.arange(2050) + 0.5) / 10.0
    pts = np.stack(np.meshgrid(900.0 + g10, 900.0 + g10), -1).reshape(-1, 2)
    pts += np.random.default_rng(11).uniform(-0.04, 0.04, pts.shape)
    pts = torch.tensor(pts, dtype=torch.float32, device="cuda")
    rp = api.Rasterizer(desc, params.K, pair_cap=fb.pair_cap).bin(fb.params_of(0))
    yp, ip = rp.render_points(pts)
    torch.cuda.synchronize()
    f0.record(stream)
    rp.render_points(pts, yp, ip)
    f1.record(stream)
    torch.cuda.synchronize()
    pts_ms = f0.elapsed_time(f1)

    # job-wide aggregation (max time over ranks, summed work)
    tot_s, work, e2e_s = aggregate(tot_s, pairs_step * args.steps, e2e_s, world)
    value = work / tot_s / 1e9
    e2e_value = work / e2e_s / 1e9

    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = clocks.get("sm_max_mhz")
    if not sm_max and os.path.exists(peaks_path):
        sm_max = json.load(open(peaks_path)).get("sm_max_mhz")
    sm_max = sm_max or 2070.0
    sm_load = clocks.get("sm_mhz") or sm_max                      # median SM clock under load
    mufu = rates["ex2"] if rates else MUFU_PER_CLK_PER_SM
    ex2_peak = mufu * sms * sm_load * 1e6                          # ex2 / s
    tile_s = statistics.mean(tile_ms) / 1e3
    ex2_achieved = 2.0 * pairs_step / tile_s                       # fwd + bwd: 2 ex2 / pair
    # FP32 roofline on the pairs that contribute (q <= q_max): the algorithmic
    # FP32 lane operations of one fwd+bwd pair, RGB linear, against the
    # measured FFMA lane rate (listed pairs would exceed 1: culled pairs cost
    # the kernel next to nothing)
    ffma = rates["ffma"] if rates else 128.0
    fma_peak = ffma * sms * sm_load * 1e6
    fma_achieved = FP32_OPS_PER_PAIR * inrange_step / tile_s
    ncu = None
    if NCU["render_cu_code_sha256"] and NCU["render_cu_code_sha256"] == code_sha256(
            os.path.join(ROOT, "paper_2510_05814_gb300", "csrc", "render.cu")):
        ncu = NCU
    traffic = ncu["bytes_per_launch"] if ncu else None

    cpu = cpu_binned = None
    if rank == 0 and world == 1 and not args.no_cpu:
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

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "image": f"{W}x{H}x{C}", "K": params.K, "tile": T,
                       "l2": "flushed (256 MiB write, untimed) before every timed step",
                       "launch": "one CUDA-graph replay of the whole fit iteration per step "
                                 "(the FitBatch.run(graph_iters=...) path)",
                       "reorder_every": REORDER_EVERY,
                       "parallelism": f"replicas x{world}",
                       "pairs_per_step": int(pairs_step), "list_pairs": int(lists1),
                       "in_range_pairs_per_step": int(inrange_step)},
            "roofline": {"bound": "alu", "kernel": "k_fit_tile (fused fwd+MSE+bwd)",
                         "achieved": ex2_achieved / 1e9, "peak": ex2_peak / 1e9,
                         "unit": "Gex2/s", "frac": ex2_achieved / ex2_peak,
                         "traffic": traffic,
                         "peak_basis": (f"{mufu:.1f} ex2 lanes/clk/SM "
                                        f"({'measured live, libsmoe_rates' if rates else 'fallback'})"
                                        f" x {sms} SMs x {sm_load:.0f} MHz (median under load); "
                                        "2 ex2 per listed fwd+bwd pair"),
                         "issue_rates_per_clk_per_sm": rates,
                         "ncu_pipes": None if ncu is None else {
                             "fma_pipe_active": ncu["fma_pipe_active"],
                             "issue_active": ncu["issue_active"],
                             "xu_active": ncu["xu_active"]}},
            "roofline_fma": {"bound": "alu", "kernel": "k_fit_tile (fused fwd+MSE+bwd)",
                             "achieved": fma_achieved / 1e12, "peak": fma_peak / 1e12,
                             "unit": "T FP32 lane-ops/s", "frac": fma_achieved / fma_peak,
                             "basis": (f"{FP32_OPS_PER_PAIR} FP32 lane operations per in-range "
                                       "fwd+bwd pair (19 forward + 48 backward, RGB linear) x "
                                       "in-range pairs / fused-kernel time; peak "
                                       f"{ffma:.1f} FFMA lanes/clk/SM x {sms} SMs x "
                                       f"{sm_load:.0f} MHz")},
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
            "sr_render_2x": {"ms": sr_ms, "pairs": sr_pairs, "out": f"{2 * W}x{2 * H}",
                             "Gpairs_per_s": sr_pairs / sr_ms / 1e6},
            "resample_points_10x": {"points": int(pts.shape[0]), "ms": pts_ms,
                                    "Gpoints_per_s": pts.shape[0] / pts_ms / 1e6,
                                    "raster": "jittered 10x raster over a 205x205 crop"},
            "cpu_baseline": cpu,
            "cpu_baseline_binned": cpu_binned,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tgt.numel() * 4),
                    "d2h_bytes_per_step": 8,
                    "copies": "pinned host target -> device each step on a copy stream "
                              "(double buffer, overlapping the previous step); loss -> host",
                    "launch": "one CUDA-graph replay per step, one graph per target buffer "
                              "(FitBatch.capture after set_target)",
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
