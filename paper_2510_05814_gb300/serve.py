"""Serving loop for rasterised SMoE: fit requests (regression of an image,
including denoising of noisy inputs) and render requests (a fitted model
resampled at 1-4x, the native super-resolution of the method), with
continuous batching.

- Fit requests are admitted while the device-memory budget allows; every
  admitted fit is a slot of ONE batched fit (one set of launches per
  iteration over the ragged tile table of all slots).  When slots join or
  leave, the batch is re-formed; each continuing slot keeps its parameters,
  Adam moments and step count on the device.
- Iterations run in chunks on the fit stream (a CUDA graph per batch
  composition and chunk length); slots leave at chunk boundaries when their
  run is complete, their final render is copied to the host and the fitted
  model stays resident for render requests.
- Render requests run on a second stream, so they overlap the fit chunks.
- Fits run in the deterministic accumulation mode by default: an image's
  result is then bit-identical whatever else shares the batch.
- A denoising request may ask for MM-RSMoE (Sec. V-C): its `models` models,
  started from lattices shifted by the window offsets, are slots of the same
  batch; the result is the per-pixel mean of their renders (Eq. 11), and a
  later render request resamples that fused model at its scale.

`serve_plain` runs the same requests one at a time, one image per launch,
in arrival order: the baseline the batched server is compared with.
Latency = time the result is on the host - arrival time.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import denoise, synth
from .api import Rasterizer, RasterDesc, SMoEParams, render_mean
from .fit import FitBatch


@dataclass
class FitRequest:
    rid: int
    image: np.ndarray                  # C x H x W float32 (host)
    iters: int = 500
    pixels_per_kernel: int = 16
    sigma: float = 5.0
    denoise: bool = False              # the image carries noise (result = fitted render)
    arrival: float = 0.0
    seed: int = 0
    models: int = 1                    # > 1: MM-RSMoE with that many models (Sec. V-C)


@dataclass
class RenderRequest:
    rid: int
    model: int                         # rid of a finished fit (resident model)
    scale: float = 1.0
    arrival: float = 0.0


@dataclass
class Result:
    rid: int
    kind: str
    arrival: float
    finish: float
    output: np.ndarray | None = None
    psnr: float | None = None
    losses: np.ndarray | None = None

    @property
    def latency(self):
        return self.finish - self.arrival


def fit_bytes(C, H, W, K):
    """Device bytes a fit slot holds: parameters + two Adam moments + target +
    its share of the fit workspace (records, sums, boxes, lists)."""
    n_param = K * (5 + 3 * C)
    pairs = 40 * K          # ~13 (tile, kernel) pairs per kernel at T = 16, 3x headroom
    return 4 * (3 * n_param + C * H * W) + K * (64 + 64 + 16) + 12 * pairs


def render_bytes(C, H, W, K, scale):
    Ho, Wo = int(round(H * scale)), int(round(W * scale))
    return 4 * (C + 1) * Ho * Wo + K * 96 + 12 * 10 * K * int(np.ceil(scale * scale))


@dataclass
class _Slot:
    req: FitRequest
    target: torch.Tensor
    params: SMoEParams
    m: SMoEParams
    v: SMoEParams
    done: int = 0
    nbytes: int = 0
    pairs: int = 0
    losses: list = field(default_factory=list)
    member: int = 0                    # index of the model inside an MM-RSMoE request


class Server:
    """Continuous-batching server on one GPU (see the module docstring)."""

    def __init__(self, hbm_budget, tile=16, lr=None, chunk=25, graphs=True,
                 persistent=False, qmax=9.0, deterministic=True, max_pixels=None):
        """max_pixels: cap on the pixels in flight (image pixels x models over
        the admitted fits); beyond the point where one batch fills the GPU,
        more concurrency only stretches every request's iterations, so the
        cap keeps the queue FIFO and the median latency down.  None: only
        the HBM budget limits admission."""
        self.deterministic = deterministic
        self.max_pixels = max_pixels
        self.px_used = 0
        self.budget = int(hbm_budget)
        self.tile, self.lr, self.chunk = tile, lr, chunk
        self.graphs, self.persistent, self.qmax = graphs, persistent, qmax
        self.fit_stream = torch.cuda.Stream()
        self.render_stream = torch.cuda.Stream()
        self.models = {}                 # rid -> (SMoEParams, (C, H, W))
        self.used = 0
        self.batch = None
        self.graph_key = None
        self.events = []                 # (t, what) trace

    # -- slots
    def _make_slots(self, r: FitRequest):
        """One slot per model of the request (r.models > 1: the MM-RSMoE set,
        lattices shifted by the window offsets; all share the target)."""
        C, H, W = r.image.shape
        K = max(1, (H * W) // r.pixels_per_kernel)
        slots = []
        with torch.cuda.stream(self.fit_stream):
            tgt = torch.tensor(r.image, device="cuda")
            for h, p in enumerate(denoise.init_models(r.image, r.models, K, r.sigma, True,
                                                      seed=r.seed)):
                s = _Slot(r, tgt, p, p.zeros_like(), p.zeros_like(), member=h)
                rr = Rasterizer(RasterDesc(W, H, C, self.tile, True, self.qmax), K).bin(p)
                s.pairs = int(rr.n_pairs.item())
                s.nbytes = fit_bytes(C, H, W, K)
                slots.append(s)
        return slots

    def _form_batch(self, slots, slack=3.0):
        cap = int(slack * sum(s.pairs for s in slots)) + 4096
        with torch.cuda.stream(self.fit_stream):
            self.batch = FitBatch([s.target for s in slots], [s.params for s in slots],
                                  [s.req.iters for s in slots], lr=self.lr, tile=self.tile,
                                  qmax=self.qmax, persistent=self.persistent,
                                  moments=[(s.m, s.v) for s in slots],
                                  steps=[s.done for s in slots],
                                  hist=max(s.req.iters for s in slots), pair_cap=cap,
                                  deterministic=self.deterministic)
        self.graph_key = None

    def _run_chunk(self, slots, n):
        fb = self.batch
        with torch.cuda.stream(self.fit_stream):
            if self.graphs:
                if self.graph_key != n:
                    fb.capture(n)
                    self.graph_key = n
                fb.graph.replay()
            else:
                fb.launch(n)
            ev = torch.cuda.Event()
            ev.record()
        return ev

    def _finish_fit(self, group, now):
        """Result of a request whose slots (one, or its MM-RSMoE models in
        member order) have all finished: the render, or the fused render."""
        s = group[0]
        C, H, W = s.target.shape
        with torch.cuda.stream(self.fit_stream):
            losses = np.mean([np.asarray(g.losses) for g in group], axis=0)
            if len(group) == 1:
                r = Rasterizer(RasterDesc(W, H, C, self.tile, True, self.qmax),
                               s.params.K).bin(s.params)
                y, _ = r.render()
            else:
                y = render_mean([g.params for g in group], W, H, self.tile, self.qmax)
            out = y.cpu().numpy()
        psnr = synth_psnr(out, s.req.image)
        self.models[s.req.rid] = ([g.params for g in group], (C, H, W))
        return Result(s.req.rid, "fit", s.req.arrival, now(), out, psnr, losses)

    def _start_render(self, q: RenderRequest):
        models, (C, H, W) = self.models[q.model]
        Ho, Wo = int(round(H * q.scale)), int(round(W * q.scale))
        if len(models) > 1:                  # a fused MM-RSMoE model (synchronous)
            with torch.cuda.stream(self.render_stream):
                y = render_mean(models, Wo, Ho, self.tile, self.qmax, q.scale)
                host = y.cpu()
                ev = torch.cuda.Event()
                ev.record()
            return (q, None, host, ev)
        params = models[0]
        with torch.cuda.stream(self.render_stream):
            r = Rasterizer(RasterDesc(Wo, Ho, C, self.tile, True, self.qmax, q.scale), params.K,
                           pair_cap=int(12 * params.K * max(1.0, q.scale * q.scale)))
            r.bin(params, check_capacity=False)      # checked when the render completes
            y, _ = r.render()
            host = torch.empty(y.shape, dtype=torch.float32, pin_memory=True)
            host.copy_(y, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record()
        return (q, r, host, ev)

    # -- the loop
    def run(self, requests, realtime=True):
        """Serve `requests` (FitRequest / RenderRequest with arrival times in
        seconds from the start); returns the results in completion order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        fits_q, renders_q = collections.deque(), collections.deque()
        slots, inflight, results = [], [], []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or fits_q or renders_q or slots or inflight:
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                r = pending.popleft()
                (fits_q if isinstance(r, FitRequest) else renders_q).append(r)
            # admit fits while the budget allows (FIFO)
            changed = False
            while fits_q:
                r = fits_q[0]
                C, H, W = r.image.shape
                need = r.models * fit_bytes(C, H, W, max(1, (H * W) // r.pixels_per_kernel))
                px = r.models * H * W
                if self.used + need > self.budget and (slots or inflight):
                    break
                if self.max_pixels and self.px_used + px > self.max_pixels and slots:
                    break
                fits_q.popleft()
                for s in self._make_slots(r):
                    self.used += s.nbytes
                    slots.append(s)
                self.px_used += px
                changed = True
                self.events.append((now(), f"admit fit {r.rid}"))
            # start renders whose model is resident
            for _ in range(len(renders_q)):
                q = renders_q.popleft()
                if q.model in self.models:
                    inflight.append(self._start_render(q))
                    self.events.append((now(), f"start render {q.rid}"))
                else:
                    renders_q.append(q)
            # one chunk of iterations for all slots
            if slots:
                if changed or self.batch is None:
                    self._form_batch(slots)
                n = min(self.chunk, min(s.req.iters - s.done for s in slots))
                ev = self._run_chunk(slots, n)
                ev.synchronize()
                fb = self.batch
                st = fb.status_code()
                steps = fb.step.cpu().numpy()
                loss = fb.loss.cpu().numpy()
                for b, s in enumerate(slots):
                    s.losses.extend(loss[b, s.done:int(steps[b])].tolist())
                    s.done = int(steps[b])
                if st == 2:           # the pair buffer overflowed: re-form larger, go on
                    for s in slots:
                        s.pairs = int(s.pairs * 1.5) + 1024
                    self._form_batch(slots)
                    continue
                if st != 0:
                    raise RuntimeError(f"fit status {st}")
                keep, finished = [], collections.OrderedDict()
                for s in slots:
                    if s.done >= s.req.iters:
                        finished.setdefault(s.req.rid, []).append(s)
                        self.used -= s.nbytes
                    else:
                        keep.append(s)
                for rid, group in finished.items():
                    results.append(self._finish_fit(sorted(group, key=lambda g: g.member), now))
                    r0 = group[0].req
                    self.px_used -= r0.models * r0.image.shape[1] * r0.image.shape[2]
                    self.events.append((now(), f"finish fit {rid}"))
                if len(keep) != len(slots):
                    slots = keep
                    self.batch = None
            # completed renders
            still = []
            for (q, r, host, ev) in inflight:
                if ev.query():
                    if r is not None and int(r.status.item()) != 0:
                        # pair buffer too small: redo, growing it
                        with torch.cuda.stream(self.render_stream):
                            r.bin(self.models[q.model][0][0])
                            y, _ = r.render()
                            host = y.cpu()
                    results.append(Result(q.rid, "render", q.arrival, now(), host.numpy()))
                    self.events.append((now(), f"finish render {q.rid}"))
                else:
                    still.append((q, r, host, ev))
            inflight = still
            if not slots and not inflight and pending and realtime:
                wait = pending[0].arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        return results


def serve_plain(requests, tile=16, lr=None, qmax=9.0, realtime=True, graphs=True,
                deterministic=True):
    """Baseline: one request at a time in arrival order, one image per launch."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    models, results = {}, []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for r in reqs:
        if realtime:
            wait = r.arrival - now()
            if wait > 0:
                time.sleep(wait)
        if isinstance(r, FitRequest):
            C, H, W = r.image.shape
            K = max(1, (H * W) // r.pixels_per_kernel)
            tgt = torch.tensor(r.image, device="cuda")
            ps, losses = [], []
            for p in denoise.init_models(r.image, r.models, K, r.sigma, True, seed=r.seed):
                fb = FitBatch([tgt], [p], r.iters, lr=lr, tile=tile, qmax=qmax,
                              deterministic=deterministic, pair_slack=3.0)
                # graph replays of 25 iterations; a pair-buffer overflow (the
                # lists grow as kernels widen) grows the buffer and resumes
                fb.run(r.iters, graph_iters=min(25, r.iters) if graphs else None,
                       check_every=r.iters)
                st = fb.status_code()
                if st != 0:
                    raise RuntimeError(f"fit status {st}")
                ps.append(p)
                losses.append(fb.losses()[0])
            if len(ps) == 1:
                rr = Rasterizer(RasterDesc(W, H, C, tile, True, qmax), K).bin(ps[0])
                y, _ = rr.render()
            else:
                y = render_mean(ps, W, H, tile, qmax)
            out = y.cpu().numpy()
            models[r.rid] = (ps, (C, H, W))
            results.append(Result(r.rid, "fit", r.arrival, now(), out, synth_psnr(out, r.image),
                                  np.mean(losses, axis=0)))
        else:
            ps, (C, H, W) = models[r.model]
            Ho, Wo = int(round(H * r.scale)), int(round(W * r.scale))
            if len(ps) == 1:
                rr = Rasterizer(RasterDesc(Wo, Ho, C, tile, True, qmax, r.scale),
                                ps[0].K).bin(ps[0])
                y, _ = rr.render()
            else:
                y = render_mean(ps, Wo, Ho, tile, qmax, r.scale)
            results.append(Result(r.rid, "render", r.arrival, now(), y.cpu().numpy()))
    return results


def synth_psnr(y, t):
    d = np.clip(y.astype(np.float64), 0.0, 1.0) - t.astype(np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return {"n": int(len(lat)), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean())}


def poisson_workload(n_fit, n_render, rate, seed=5, iters=500, sizes=None, noise_var=0.05,
                     render_scales=(1.0, 4.0), mm_models=1, images=None):
    """Fit requests with sizes from `sizes` (default: the ragged size
    distribution, 128x96 .. 1920x1080), half of them denoising requests with
    N(0, noise_var) added (MM-RSMoE with `mm_models` models when > 1);
    render requests on earlier fits at scales drawn from U[render_scales];
    Poisson arrivals at `rate` per second.  `images`: (C, H, W) images to use
    for the fit requests in turn instead of drawing new ones."""
    rng = np.random.default_rng(seed)
    sizes = sizes or synth.ragged_sizes(n_fit, seed)
    n = n_fit + n_render
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    kinds = np.array(["fit"] * n_fit + ["render"] * n_render)
    kinds[0] = "fit"
    rest = kinds[1:].copy()
    rng.shuffle(rest)
    kinds[1:] = rest
    reqs, fit_ids, fi = [], [], 0
    for i, (a, k) in enumerate(zip(arrivals, kinds)):
        if k == "fit" or not fit_ids:
            if images is not None:
                img = np.array(images[fi % len(images)], np.float32)
            else:
                W, H = sizes[fi % len(sizes)]
                img = synth.polygon_image(W, H, 3, 12, seed * 1000 + i, texture_amp=0.1)
            fi += 1
            den = (len(fit_ids) % 2) == 1
            if den:
                img = (img + rng.normal(0.0, np.sqrt(noise_var), img.shape)).astype(np.float32)
            reqs.append(FitRequest(i, img, iters, denoise=den, arrival=float(a), seed=i,
                                   models=mm_models if den else 1))
            fit_ids.append(i)
        else:
            reqs.append(RenderRequest(i, int(rng.choice(fit_ids)),
                                      float(rng.uniform(*render_scales)), float(a)))
    return reqs
