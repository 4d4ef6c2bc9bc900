"""Python binding of libsmoe.so: the C-ABI calls under the same names, taking
torch CUDA tensors (argument marshalling only -- every step runs in the
library's kernels), plus small helpers that own workspaces and lists."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import SmoeError, check


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


@dataclass(frozen=True)
class RasterDesc:
    """A raster: W x H pixels, C channels, tile side, expert type, cutoff,
    resampling scale (L' = L/s, eW' = eW/s) and gate mode (rbf: the
    unnormalised sum of Eq. 1 instead of the softmax gates of Eq. 4)."""
    W: int
    H: int
    C: int
    tile: int = 16
    linear: bool = True
    qmax: float = 9.0
    scale: float = 1.0
    rbf: bool = False

    def c(self):
        return _lib.Desc(self.W, self.H, self.C, self.tile, int(self.linear), self.qmax, self.scale,
                         int(self.rbf))

    @property
    def n_tiles(self):
        return ((self.W + self.tile - 1) // self.tile) * ((self.H + self.tile - 1) // self.tile)


class SMoEParams:
    """Kernel parameters as FP32 CUDA tensors (SoA): mu (K,2) normalised,
    chol (K,3) = (a,b,c), ea (K,C), eW (K,C,2) or None, logpi (K,) gate
    weights log pi_k (Eq. 4) or None for pi = 1."""

    def __init__(self, mu, chol, ea, eW=None, logpi=None):
        self.mu, self.chol, self.ea, self.eW, self.logpi = mu, chol, ea, eW, logpi

    @classmethod
    def from_numpy(cls, p, device="cuda"):
        f = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a, np.float32),
                                                              device=device)
        return cls(f(p.mu), f(p.chol), f(p.ea), f(p.eW), f(getattr(p, "logpi", None)))

    @classmethod
    def zeros(cls, K, C, linear, device="cuda", pi=False):
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        return cls(z(K, 2), z(K, 3), z(K, C), z(K, C, 2) if linear else None,
                   z(K) if pi else None)

    def zeros_like(self):
        return SMoEParams(*(None if t is None else torch.zeros_like(t) for t in self.slots()))

    def clone(self):
        return SMoEParams(*(None if t is None else t.clone() for t in self.slots()))

    def slots(self):
        """(mu, chol, ea, eW, logpi), None for an absent group."""
        return (self.mu, self.chol, self.ea, self.eW, self.logpi)

    def tensors(self):
        """The groups present, in slot order."""
        return tuple(t for t in self.slots() if t is not None)

    @property
    def K(self):
        return int(self.mu.shape[0])

    @property
    def C(self):
        return int(self.ea.shape[1])

    @property
    def linear(self):
        return self.eW is not None

    def c(self):
        return _lib.Params(self.K, _ptr(self.mu), _ptr(self.chol), _ptr(self.ea), _ptr(self.eW),
                           _ptr(self.logpi))

    def numpy(self):
        """Host copies of the present groups, in slot order."""
        return tuple(t.detach().cpu().numpy() for t in self.tensors())


# ---------------------------------------------------------------------------
# the C-ABI calls
# ---------------------------------------------------------------------------

def smoe_version() -> int:
    return int(_lib.load().smoe_version())


def smoe_workspace_size(desc: RasterDesc, K: int, pair_cap: int) -> int:
    n = ctypes.c_size_t(0)
    check(_lib.load().smoe_workspace_size(ctypes.byref(desc.c()), K, pair_cap, ctypes.byref(n)),
          "smoe_workspace_size")
    return int(n.value)


def smoe_bin(desc, params: SMoEParams, ws, tile_off, pair_k, n_pairs, status, stream=None):
    d, p = desc.c(), params.c()
    check(_lib.load().smoe_bin(ctypes.byref(d), ctypes.byref(p), _ptr(ws), ws.numel(),
                               _ptr(tile_off), _ptr(pair_k), pair_k.numel(), _ptr(n_pairs),
                               _ptr(status), _stream(stream)), "smoe_bin")


def smoe_render(desc, K, ws, tile_off, pair_k, y, inv_d=None, status=None, stream=None):
    d = desc.c()
    check(_lib.load().smoe_render(ctypes.byref(d), K, _ptr(ws), ws.numel(), _ptr(tile_off),
                                  _ptr(pair_k), _ptr(y), _ptr(inv_d), _ptr(status),
                                  _stream(stream)), "smoe_render")


def smoe_render_backward(desc, params, ws, tile_off, pair_k, y, inv_d, gy, target, grad,
                         status=None, stream=None):
    d, p, g = desc.c(), params.c(), grad.c()
    check(_lib.load().smoe_render_backward(ctypes.byref(d), ctypes.byref(p), _ptr(ws), ws.numel(),
                                           _ptr(tile_off), _ptr(pair_k), _ptr(y), _ptr(inv_d),
                                           _ptr(gy), _ptr(target), ctypes.byref(g), _ptr(status),
                                           _stream(stream)), "smoe_render_backward")


def smoe_adam_step(p, g, m, v, lr, b1=0.9, b2=0.999, eps=1e-8, step=1, stream=None):
    """lr = (mu, chol, ea, eW[, logpi])."""
    lr5 = list(lr) + [0.0] * (5 - len(lr))
    lr4 = (ctypes.c_float * 5)(*[float(x) for x in lr5[:5]])
    pc, gc, mc, vc = p.c(), g.c(), m.c(), v.c()
    check(_lib.load().smoe_adam_step(ctypes.byref(pc), ctypes.byref(gc), ctypes.byref(mc),
                                     ctypes.byref(vc), p.C, lr4, float(b1), float(b2),
                                     float(eps), step, _stream(stream)), "smoe_adam_step")


def smoe_sq_error(y, target, out, clamp=True, stream=None):
    check(_lib.load().smoe_sq_error(_ptr(y), _ptr(target), y.numel(), int(clamp), _ptr(out),
                                    _stream(stream)), "smoe_sq_error")


def smoe_get_status(status, stream=None) -> int:
    return int(_lib.load().smoe_get_status(_ptr(status), _stream(stream)))


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class Rasterizer:
    """Owns the workspace, the tile lists and the status word of one raster.

    ``bin`` builds the lists (growing the pair buffer when the pair count
    exceeds it, which costs one host synchronisation), ``render`` and
    ``backward`` run the tile kernels on them."""

    def __init__(self, desc: RasterDesc, K: int, pair_cap: int | None = None, device="cuda"):
        self.desc, self.K, self.device = desc, K, device
        self.tile_off = torch.zeros(desc.n_tiles + 1, dtype=torch.int32, device=device)
        self.n_pairs = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self._alloc(pair_cap if pair_cap is not None else max(1024, 8 * K))

    def _alloc(self, cap):
        self.pair_cap = int(cap)
        self.pair_k = torch.zeros(max(self.pair_cap, 1), dtype=torch.int32, device=self.device)
        n = smoe_workspace_size(self.desc, self.K, self.pair_cap)
        self.ws = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws = self.ws[off:off + n]

    def bin(self, params: SMoEParams, check_capacity=True, stream=None):
        assert params.K == self.K
        self.status.zero_()
        smoe_bin(self.desc, params, self.ws, self.tile_off, self.pair_k, self.n_pairs, self.status,
                 stream)
        if check_capacity:
            st = smoe_get_status(self.status, stream)
            if st == _lib.SMOE_ERR_CAPACITY:
                need = int(self.n_pairs.item())
                self._alloc(int(need * 1.25) + 1024)
                self.status.zero_()
                smoe_bin(self.desc, params, self.ws, self.tile_off, self.pair_k, self.n_pairs,
                         self.status, stream)
                st = smoe_get_status(self.status, stream)
            if st != _lib.SMOE_OK:
                raise SmoeError(st, "smoe_bin")
        return self

    def render(self, y=None, inv_d=None, stream=None):
        d = self.desc
        if y is None:
            y = torch.empty(d.C, d.H, d.W, dtype=torch.float32, device=self.device)
        if inv_d is None:
            inv_d = torch.empty(d.H, d.W, dtype=torch.float32, device=self.device)
        smoe_render(d, self.K, self.ws, self.tile_off, self.pair_k, y, inv_d, self.status, stream)
        return y, inv_d

    def backward(self, params, y, inv_d, gy=None, target=None, grad=None, stream=None):
        if grad is None:
            grad = params.zeros_like()
        smoe_render_backward(self.desc, params, self.ws, self.tile_off, self.pair_k, y, inv_d, gy,
                             target, grad, self.status, stream)
        return grad

    def render_points(self, xy, y=None, inv_d=None, stream=None):
        """y(x) at the (n, 2) float32 CUDA points ``xy`` (pixel units of this
        raster); returns (y (C, n), inv_d (n,))."""
        d = self.desc
        xy = xy.contiguous()
        assert xy.dtype == torch.float32 and xy.dim() == 2 and xy.shape[1] == 2
        n = xy.shape[0]
        if y is None:
            y = torch.empty(d.C, n, dtype=torch.float32, device=self.device)
        if inv_d is None:
            inv_d = torch.empty(n, dtype=torch.float32, device=self.device)
        lib = _lib.load()
        nb = ctypes.c_size_t(0)
        check(lib.smoe_points_workspace_size(ctypes.byref(d.c()), n, ctypes.byref(nb)),
              "smoe_points_workspace_size")
        if getattr(self, "_pws", None) is None or self._pws.numel() < nb.value:
            raw = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
            off = (-raw.data_ptr()) % 256
            self._pws = raw[off:off + nb.value]
        check(lib.smoe_render_points(ctypes.byref(d.c()), self.K, _ptr(self.ws), self.ws.numel(),
                                     _ptr(self.tile_off), _ptr(self.pair_k), n, _ptr(xy),
                                     _ptr(self._pws), self._pws.numel(), _ptr(y), _ptr(inv_d),
                                     _ptr(self.status), _stream(stream)), "smoe_render_points")
        return y, inv_d

    def count_inrange(self, stream=None):
        """Number of listed (pixel, kernel) pairs with q <= q_max (synchronises)."""
        out = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(_lib.load().smoe_count_inrange(ctypes.byref(self.desc.c()), self.K, _ptr(self.ws),
                                             self.ws.numel(), _ptr(self.tile_off),
                                             _ptr(self.pair_k), _ptr(out), _ptr(self.status),
                                             _stream(stream)), "smoe_count_inrange")
        return int(out.item())

    def lists(self):
        """(tile_off, pair_k) trimmed to the pair count, on the host."""
        off = self.tile_off.cpu().numpy()
        return off, self.pair_k[: int(off[-1])].cpu().numpy()


def sharpen(params: SMoEParams, factor: float, qmax: float = 9.0):
    """Native sharpening by kernel editing (Sec. II-B, smoe_sharpen): a model
    whose kernel bandwidths are divided by ``factor`` (L' = factor L, on the
    GPU; mu and the experts are shared with ``params``) and the cutoff that
    keeps each kernel's support, q_max' = q_max factor^2, both from the
    library.  Returns (sharpened params, q_max').  Raises ValueError where
    the library refuses the factor (q_max' beyond the FP32 range of the
    gates)."""
    chol = torch.empty_like(params.chol)
    q2 = ctypes.c_float(0.0)
    code = _lib.load().smoe_sharpen(_ptr(params.chol), _ptr(chol), params.K, float(factor),
                                    float(qmax), ctypes.byref(q2), _stream(None))
    if code == _lib.SMOE_ERR_ARG:
        raise ValueError(f"smoe_sharpen refused factor {factor} at q_max {qmax}")
    check(code, "smoe_sharpen")
    return SMoEParams(params.mu, chol, params.ea, params.eW), float(q2.value)


def render(params: SMoEParams, W, H, tile=16, qmax=9.0, scale=1.0, sharpen_factor=None,
           rbf=False):
    """Bin and render ``params`` on a W x H raster (``scale`` times the fitted
    raster, optionally sharpened; rbf: the sum of Eq. 1); returns
    (y, inv_d, rasterizer)."""
    if sharpen_factor is not None and sharpen_factor != 1.0:
        params, qmax = sharpen(params, sharpen_factor, qmax)
    desc = RasterDesc(W, H, params.C, tile, params.linear, qmax, scale, rbf)
    r = Rasterizer(desc, params.K).bin(params)
    y, inv_d = r.render()
    return y, inv_d, r


def render_mean(models, W, H, tile=16, qmax=9.0, scale=1.0, rbf=False, pair_cap=None,
                stream=None):
    """Multi-model fusion (Sec. V-C, Eq. 11) of separate models (a list of
    SMoEParams) on a W x H raster at `scale`: the per-pixel mean of their
    renders, one binning pass and one averaging launch.  Returns (C, H, W)."""
    lib = _lib.load()
    Hm = len(models)
    d = RasterDesc(W, H, models[0].C, tile, models[0].linear, qmax, scale, rbf).c()
    arr = (_lib.Params * Hm)(*[m.c() for m in models])
    K = sum(m.K for m in models)
    cap = int(pair_cap if pair_cap is not None else 12 * K * max(1.0, scale * scale) + 4096)
    y = torch.empty(models[0].C, H, W, dtype=torch.float32, device=models[0].mu.device)
    status = torch.zeros(1, dtype=torch.int32, device=y.device)
    while True:
        n = ctypes.c_size_t(0)
        check(lib.smoe_render_mean_workspace_size(ctypes.byref(d), arr, Hm, cap, ctypes.byref(n)),
              "smoe_render_mean_workspace_size")
        raw = torch.empty(n.value + 256, dtype=torch.uint8, device=y.device)
        off = (-raw.data_ptr()) % 256
        ws = raw[off:off + n.value]
        status.zero_()
        check(lib.smoe_render_mean(ctypes.byref(d), arr, Hm, _ptr(ws), ws.numel(), cap, _ptr(y),
                                   _ptr(status), _stream(stream)), "smoe_render_mean")
        st = smoe_get_status(status, stream)
        if st == _lib.SMOE_ERR_CAPACITY:
            cap = 2 * cap
            continue
        if st != _lib.SMOE_OK:
            raise SmoeError(st, "smoe_render_mean")
        return y


def render_points(params: SMoEParams, W, H, xy, tile=16, qmax=9.0, sharpen_factor=None,
                  rbf=False):
    """Resample the model fitted on a W x H raster at the (n, 2) points
    ``xy`` (pixel units of that raster): super-resolution on an irregular
    raster.  Returns (y (C, n), inv_d (n,), rasterizer)."""
    if sharpen_factor is not None and sharpen_factor != 1.0:
        params, qmax = sharpen(params, sharpen_factor, qmax)
    desc = RasterDesc(W, H, params.C, tile, params.linear, qmax, 1.0, rbf)
    r = Rasterizer(desc, params.K).bin(params)
    y, inv_d = r.render_points(xy)
    return y, inv_d, r


class SMoERender(torch.autograd.Function):
    """y = R-SMoE render of (mu, chol, ea, eW[, logpi]) on a raster (Eqs. 2-5;
    the RBF sum of Eq. 1 when desc.rbf), with the backward of the tile
    kernels.  Each forward keeps its own lists for its backward."""

    @staticmethod
    def forward(ctx, mu, chol, ea, eW, desc: RasterDesc, logpi=None):
        c = lambda t: None if t is None else t.detach().contiguous()
        p = SMoEParams(c(mu), c(chol), c(ea), c(eW), c(logpi))
        r = Rasterizer(desc, p.K).bin(p)
        y, inv_d = r.render()
        ctx.r, ctx.p = r, p
        ctx.save_for_backward(y, inv_d)
        return y

    @staticmethod
    def backward(ctx, gy):
        y, inv_d = ctx.saved_tensors
        g = ctx.r.backward(ctx.p, y, inv_d, gy=gy.contiguous())
        return g.mu, g.chol, g.ea, g.eW, None, g.logpi


def smoe_render_fn(mu, chol, ea, eW, desc: RasterDesc, logpi=None):
    return SMoERender.apply(mu, chol, ea, eW, desc, logpi)
