"""Autotuner for batched fits: tile side, persistent launch, and how many
kernels one batched launch may hold (larger batches are split into groups
that run one after the other).

Every candidate fits the same model (the truncated SMoE does not depend on
the tile size; only the lists do), so the choice is made on measured time
per iteration alone: each candidate runs a few warm-up and timed iterations
on clones of the initial parameters, timed with CUDA events on the current
stream."""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import torch

from .fit import FitBatch


@dataclass
class TuneResult:
    tile: int
    persistent: bool
    max_kernels: int | None
    ms_per_iter: float
    table: list = field(default_factory=list)   # (tile, persistent, max_kernels, ms)


def groups_by_kernels(Ks, max_kernels):
    """Consecutive groups of images with at most max_kernels kernels each
    (an image larger than the limit gets a group of its own); no images, no
    groups."""
    if not Ks:
        return []
    if not max_kernels:
        return [list(range(len(Ks)))]
    out, cur, n = [], [], 0
    for i, k in enumerate(Ks):
        if cur and n + k > max_kernels:
            out.append(cur)
            cur, n = [], 0
        cur.append(i)
        n += k
    if cur:
        out.append(cur)
    return out


def _time(batches, warmup, iters):
    for fb in batches:
        fb.launch(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        for fb in batches:
            fb.launch(1)
    e1.record()
    torch.cuda.synchronize()
    for fb in batches:
        st = fb.status_code()
        if st != 0:
            raise RuntimeError(f"autotune candidate failed with status {st}")
    return e0.elapsed_time(e1) / iters


def tune(targets, params, lr, tiles=(8, 16, 32), persistent=(False, True),
         max_kernels=(None,), warmup=2, iters=6, **fit_kw) -> TuneResult:
    """Time every candidate and return the fastest (with the full table)."""
    Ks = [p.K for p in params]
    table = []
    for T, pers, mk in itertools.product(tiles, persistent, max_kernels):
        batches = []
        for grp in groups_by_kernels(Ks, mk):
            batches.append(FitBatch([targets[i] for i in grp], [params[i].clone() for i in grp],
                                    warmup + iters, lr=lr, tile=T, persistent=pers, **fit_kw))
        ms = _time(batches, warmup, iters)
        table.append((T, pers, mk, ms))
        del batches
    best = min(table, key=lambda r: r[3])
    return TuneResult(best[0], best[1], best[2], best[3], table)
