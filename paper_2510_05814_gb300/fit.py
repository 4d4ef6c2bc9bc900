"""Fit driver over smoe_fit: one image or a ragged batch of images, each
iteration = binning, one fused forward/MSE/backward launch over the ragged
tile table of all images, one fused finalize + Adam launch.  Iterations can
be captured in a CUDA graph and replayed; the pair buffer grows (and the run
continues) if an iteration overflows it."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import SmoeError, check
from .api import RasterDesc, Rasterizer, SMoEParams, _ptr, _stream, smoe_get_status


class FitBatch:
    """B images fitted together.

    targets: list of (C,H,W) float32 CUDA tensors; params: list of SMoEParams
    (each image's own tensors, updated in place); iters: per-image run length
    (int or list); lr = (mu0, mu1, chol, ea, eW[, pi]) or one tuple per image
    (pi: the rate of the gate weights log pi_k, for parameters that carry them;
    default: synth.fit_rates of each image, the paper's rates with the centre
    rate in pixels);
    rbf: fit the unnormalised RBF sum of Eq. 1 instead of the softmax gates;
    persistent: run the fused tile kernel as one persistent grid;
    deterministic: per-pair gradient partials added in a fixed order (a fit
    is then bit-reproducible and independent of the rest of the batch);
    reorder_every: in run(), re-sort each image's kernels into tile-major
    order of their centres every that many iterations (smoe_fit_reorder: the
    fit moves the centres and the binning is faster when consecutive kernels
    are neighbours).  The batch's parameter tensors then hold the kernels in
    that order; params_of() returns them in the caller's order."""

    def __init__(self, targets, params, iters, lr=None, tile=16,
                 qmax=9.0, b1=0.9, b2=0.999, eps=1e-8, hist=None, pair_slack=1.5,
                 persistent=False, pair_cap=None, moments=None, steps=None,
                 deterministic=False, device="cuda", rbf=False, reorder_every=None):
        """moments: optional list of (m, v) SMoEParams per image and steps an
        optional list of iterations already done: a run that continues in a
        re-formed batch keeps its Adam state and schedule position."""
        assert len(targets) == len(params) and len(targets) > 0
        self.B = len(targets)
        self.device = device
        self.C = params[0].C
        self.linear = params[0].linear
        self.tile, self.qmax = tile, qmax
        self.b1, self.b2, self.eps = b1, b2, eps
        self.persistent = bool(persistent)
        self.rbf = bool(rbf)
        self.deterministic = bool(deterministic)
        self.targets = [t.contiguous() for t in targets]
        self.iters = [iters] * self.B if np.isscalar(iters) else list(iters)
        if lr is None:
            from .synth import fit_rates
            self.lr = [fit_rates(t.shape[2], t.shape[1]) for t in self.targets]
        else:
            self.lr = [lr] * self.B if np.isscalar(lr[0]) else list(lr)
        self.params = list(params)
        self.Ks = [p.K for p in params]
        if moments is None:
            self.m = [p.zeros_like() for p in params]
            self.v = [p.zeros_like() for p in params]
        else:
            self.m = [mv[0] for mv in moments]
            self.v = [mv[1] for mv in moments]
        self.step = torch.tensor(list(steps) if steps is not None else [0] * self.B,
                                 dtype=torch.int32, device=device)
        self._continue = moments is not None
        self.reorder_every = int(reorder_every) if reorder_every else None
        self.k_off = [int(x) for x in np.concatenate([[0], np.cumsum(self.Ks)[:-1]])]
        # slot -> kernel index in the caller's order (global over the batch)
        self.order = (torch.arange(sum(self.Ks), dtype=torch.int32, device=device)
                      if self.reorder_every else None)
        self._since_reorder = 0
        self._reorder_graph = None
        self.hist = int(hist if hist is not None else max(self.iters))
        self.loss = torch.zeros(self.B, max(self.hist, 1), dtype=torch.float64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.graph = None
        if pair_cap is None:
            # Pair capacity: bin each image once with its initial parameters.
            total = 0
            for b in range(self.B):
                t = self.targets[b]
                desc = RasterDesc(t.shape[2], t.shape[1], self.C, tile, self.linear, qmax, 1.0)
                r = Rasterizer(desc, self.Ks[b]).bin(self.params[b])
                total += int(r.n_pairs.item())
            pair_cap = int(total * pair_slack) + 4096
        self.pair_cap = int(pair_cap)
        self._setup(reset=not self._continue)

    # -- C structs
    def _structs(self):
        imgs = (_lib.FitImage * self.B)()
        for b in range(self.B):
            t = self.targets[b]
            lr = self.lr[b]
            imgs[b] = _lib.FitImage(t.shape[2], t.shape[1], _ptr(t), self.params[b].c(),
                                    self.m[b].c(), self.v[b].c(), int(self.iters[b]), lr[0],
                                    lr[1], lr[2], lr[3], lr[4], lr[5] if len(lr) > 5 else 0.0)
        batch = _lib.FitBatch(self.B, self.C, self.tile, int(self.linear), self.qmax, self.b1,
                              self.b2, self.eps, _ptr(self.step), _ptr(self.loss), self.hist,
                              int(self.persistent), int(self.deterministic), int(self.rbf))
        return batch, imgs

    def _setup(self, reset):
        lib = _lib.load()
        self._batch, self._imgs = self._structs()
        n = ctypes.c_size_t(0)
        check(lib.smoe_fit_workspace_size(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                          ctypes.byref(n)), "smoe_fit_workspace_size")
        raw = torch.empty(n.value + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        self.ws = raw[off:off + n.value]
        if not reset:
            # an overflowed iteration stopped at binning: it added no loss and
            # took no step, so only the status is cleared
            self.status.zero_()
        check(lib.smoe_fit_init(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                _ptr(self.ws), self.ws.numel(), int(reset), _ptr(self.status),
                                _stream(None)), "smoe_fit_init")
        self.graph = None
        self._reorder_graph = None

    def params_of(self, b, out=None, stream=None):
        """Image b's parameters in the caller's kernel order: the batch's own
        tensors, or (after reordering) a copy scattered back through the
        order map by smoe_scatter_params (into ``out`` when given, an
        SMoEParams of the same shape, else into new tensors)."""
        if self.order is None:
            if out is not None:
                for d, s_ in zip(out.tensors(), self.params[b].tensors()):
                    d.copy_(s_)
                return out
            return self.params[b]
        src = self.params[b]
        dst = src.zeros_like() if out is None else out
        if src.K:
            idx = self.order[self.k_off[b]:self.k_off[b] + src.K]
            check(_lib.load().smoe_scatter_params(ctypes.byref(src.c()), _ptr(idx), self.k_off[b],
                                                  self.C, ctypes.byref(dst.c()), _stream(stream)),
                  "smoe_scatter_params")
        return dst

    def _reorder_call(self, stream=None):
        check(_lib.load().smoe_fit_reorder(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                           _ptr(self.ws), self.ws.numel(),
                                           _ptr(self.order) if self.order is not None else None,
                                           _ptr(self.status), _stream(stream)),
              "smoe_fit_reorder")

    def reorder(self, stream=None):
        """Re-sort every image's kernels into tile-major order of their centres
        (smoe_fit_reorder); parameters and Adam moments move together.  On
        the current stream it replays a captured CUDA graph of the call (its
        launches are many and short)."""
        if stream is not None:
            self._reorder_call(stream)
        else:
            if self._reorder_graph is None:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._reorder_call()
                self._reorder_graph = g
            self._reorder_graph.replay()
        self._since_reorder = 0

    def set_target(self, b, target):
        """Point image b at another target tensor of the same shape (for
        example the other half of a double buffer that a copy stream fills).
        A single-image batch only rewrites the host-side struct; a batch of
        several images re-uploads its image table (smoe_fit_init, which
        synchronises)."""
        t = self.targets[b]
        assert target.shape == t.shape and target.dtype == t.dtype and target.is_contiguous()
        self.targets[b] = target
        if self.B == 1:
            self._imgs[b].target = _ptr(target)
        else:
            self._setup(reset=False)

    def launch(self, n_iters=1, stream=None):
        """Enqueue n_iters iterations (no host synchronisation)."""
        check(_lib.load().smoe_fit(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                   _ptr(self.ws), self.ws.numel(), n_iters, _ptr(self.status),
                                   _stream(stream)), "smoe_fit")

    def phase(self, phase, stream=None):
        """Enqueue one phase (0 bin, 1 fused tiles, 2 Adam) of one iteration."""
        check(_lib.load().smoe_fit_phase(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                         _ptr(self.ws), self.ws.numel(), phase,
                                         _ptr(self.status), _stream(stream)), "smoe_fit_phase")

    def gradients(self, stream=None, with_pi=None):
        """The gradients this iteration would apply (smoe_fit_gradients):
        bins, runs the fused forward / MSE / backward launch and reads out
        every kernel's finalized dL/dtheta without stepping Adam.  Returns one
        SMoEParams per image, rows in the batch's kernel order (the caller's
        order unless the batch has been re-sorted; see params_of).  with_pi:
        also return dL/dlogpi (default: when the parameters carry logpi)."""
        K = sum(self.Ks)
        if with_pi is None:
            with_pi = self.params[0].logpi is not None
        g = SMoEParams.zeros(K, self.C, self.linear, device=self.device, pi=with_pi)
        check(_lib.load().smoe_fit_gradients(ctypes.byref(self._batch), self._imgs, self.pair_cap,
                                             _ptr(self.ws), self.ws.numel(), ctypes.byref(g.c()),
                                             _ptr(self.status), _stream(stream)),
              "smoe_fit_gradients")
        out = []
        for b in range(self.B):
            a, n = self.k_off[b], self.Ks[b]
            out.append(SMoEParams(*(None if t is None else t[a:a + n] for t in g.slots())))
        return out

    def capture(self, n_iters=1):
        """Capture n_iters iterations into a CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.launch(0)          # warm the library's launch path outside capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch(n_iters)
        self.graph, self.graph_iters = g, n_iters
        return g

    def status_code(self):
        return smoe_get_status(self.status)

    def _launch_iters(self, n, graph_iters):
        """Enqueue n iterations: replays of the graph of graph_iters
        iterations (captured on first use), the rest launched directly."""
        if not graph_iters:
            self.launch(n)
            return
        if self.graph is None or self.graph_iters != graph_iters:
            self.capture(graph_iters)
        reps = n // graph_iters
        for _ in range(reps):
            self.graph.replay()
        if n - reps * graph_iters:
            self.launch(n - reps * graph_iters)

    def run(self, n_iters, graph_iters=None, check_every=None):
        """Run n_iters iterations; with graph_iters, as replays of a captured
        graph of that many iterations.  The status is checked (one host
        synchronisation) after every `check_every` iterations (default: at
        the end); the spatial re-sort runs every reorder_every iterations in
        between, without a synchronisation.  A pair-buffer overflow stops the
        batch at that iteration's binning (every later kernel, the re-sort
        included, sees the status and does nothing): the buffer grows and the
        run resumes from the iteration that overflowed."""
        done = 0
        check_every = check_every or n_iters
        while done < n_iters:
            chunk = min(check_every, n_iters - done)
            before = self.step.clone()
            since0 = self._since_reorder
            left = chunk
            while left > 0:
                seg = left
                if self.reorder_every:
                    seg = min(seg, self.reorder_every - self._since_reorder)
                self._launch_iters(seg, graph_iters)
                left -= seg
                if self.reorder_every:
                    self._since_reorder += seg
                    if self._since_reorder >= self.reorder_every:
                        self.reorder()
            st = self.status_code()
            if st == _lib.SMOE_ERR_CAPACITY:
                # Grow the pair buffer and continue where the run stopped.
                progressed = int((self.step - before).max().item())
                self.pair_cap = int(self.pair_cap * 1.5) + 4096
                self._setup(reset=False)
                done += progressed
                if self.reorder_every:
                    # the re-sorts up to the overflow ran, the later ones did nothing
                    self._since_reorder = (since0 + progressed) % self.reorder_every
                continue
            if st != _lib.SMOE_OK:
                raise SmoeError(st, "smoe_fit")
            done += chunk
        return self

    def render_mean(self, out=None, stream=None):
        """Multi-model fusion (Sec. V-C, Eq. 11): the per-pixel mean of the
        renders of the batch's B models, all images of one size.  Bins the
        current parameters (growing the pair buffer if they overflow it) and
        returns a (C, H, W) tensor."""
        t = self.targets[0]
        if any(x.shape != t.shape for x in self.targets):
            raise ValueError("render_mean needs images of one size")
        out = torch.empty_like(t) if out is None else out
        assert out.shape == t.shape and out.dtype == torch.float32 and out.is_contiguous()
        while True:
            check(_lib.load().smoe_fit_render_mean(ctypes.byref(self._batch), self._imgs,
                                                   self.pair_cap, _ptr(self.ws), self.ws.numel(),
                                                   _ptr(out), _ptr(self.status),
                                                   _stream(stream)), "smoe_fit_render_mean")
            st = self.status_code()
            if st == _lib.SMOE_ERR_CAPACITY:
                self.pair_cap = int(self.pair_cap * 1.5) + 4096
                self._setup(reset=False)
                continue
            if st != _lib.SMOE_OK:
                raise SmoeError(st, "smoe_fit_render_mean")
            return out

    def losses(self):
        return self.loss.cpu().numpy()
