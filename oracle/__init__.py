"""CPU oracle for rasterised SMoE regression -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It wraps ``smoe_oracle.c`` (plain C, FP64 values, an
FP32 replica of the inclusion predicate and the bounding box) with ctypes and
numpy.  It shares no code with the CUDA library and never imports it.

Model (arXiv 2510.05814): steered Gaussian kernels (Eq. 2) with precision
P = L L^T, softmax gates (Eq. 4, pi = 1), constant or linear experts (Eq. 3),
per-block kernel subsets (Eq. 5) from a square bounding box whose side is the
major axis of the q_max ellipse (Sec. IV-B/C), Adam fit (Sec. VI-B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smoe_oracle.c")
_LIB = os.path.join(_HERE, "libsmoe_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of float expressions)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("C", ctypes.c_int32),
                ("T", ctypes.c_int32), ("linear", ctypes.c_int32),
                ("qmax", ctypes.c_float), ("scale", ctypes.c_float),
                ("K", ctypes.c_int64),
                ("mu", ctypes.c_void_p), ("chol", ctypes.c_void_p),
                ("ea", ctypes.c_void_p), ("eW", ctypes.c_void_p),
                ("rbf", ctypes.c_int32), ("logpi", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        # SMOE_ORACLE_LIB lets the mutation tests load a deliberately broken
        # copy of the oracle; normally the library is built from smoe_oracle.c.
        lib = ctypes.CDLL(os.environ.get("SMOE_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        MP = ctypes.POINTER(_Model)
        lib.om_included.argtypes = [MP, I64, ctypes.c_int32, ctypes.c_int32]
        lib.om_included.restype = ctypes.c_int
        lib.om_rect.argtypes = [MP, I64, P]
        lib.om_rect.restype = I64
        lib.om_bin.argtypes = [MP, I64, P, P, P, I64]
        lib.om_bin.restype = I64
        lib.om_render.argtypes = [MP, I64, P, P, P, P]
        lib.om_render.restype = None
        lib.om_render_points.argtypes = [MP, I64, P, P, P, P]
        lib.om_render_points.restype = None
        lib.om_backward.argtypes = [MP, P, P, I64, P, P, P, P, P, P, P, P, P, P, P]
        lib.om_backward.restype = None
        lib.om_adam.argtypes = [I64, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        lib.om_adam.restype = None
        lib.om_lr_mu.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                 ctypes.c_int32]
        lib.om_lr_mu.restype = ctypes.c_double
        lib.om_fit.argtypes = [MP, P, ctypes.c_int32, P, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, P, P, P, P, P, P]
        lib.om_fit.restype = None
        lib.om_fwd_bwd_binned.argtypes = [MP, P, P, P, P, P, P, P]
        lib.om_fwd_bwd_binned.restype = ctypes.c_double
        lib.om_threads.argtypes = []
        lib.om_threads.restype = ctypes.c_int32
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class Model:
    """A truncated SMoE model on a W x H raster (FP32 parameters, SoA).

    mu (K,2) normalised, chol (K,3) = (a,b,c) of L = [[a,0],[b,c]] with
    precision P = L L^T in pixel units of the fitted raster, ea (K,C),
    eW (K,C,2) or None for constant experts.  ``scale`` resamples the model on
    a raster ``scale`` times finer (L and eW divided by it).  ``logpi`` (K,)
    holds the gate weights log pi_k of Eq. 4 (None: pi = 1); ``rbf`` selects
    the unnormalised RBF / Gaussian-splatting sum of Eq. 1 (D = 1)."""
    W: int
    H: int
    C: int
    mu: np.ndarray
    chol: np.ndarray
    ea: np.ndarray
    eW: np.ndarray | None = None
    tile: int = 16
    qmax: float = 9.0
    scale: float = 1.0
    logpi: np.ndarray | None = None
    rbf: bool = False

    def __post_init__(self):
        f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
        self.mu = f32(self.mu).reshape(-1, 2)
        self.chol = f32(self.chol).reshape(-1, 3)
        self.ea = f32(self.ea).reshape(-1, self.C)
        if self.eW is not None:
            self.eW = f32(self.eW).reshape(-1, self.C, 2)
        if self.logpi is not None:
            self.logpi = f32(self.logpi).reshape(-1)

    @property
    def K(self) -> int:
        return int(self.mu.shape[0])

    @property
    def linear(self) -> bool:
        return self.eW is not None

    def _c(self) -> _Model:
        self._keep = (self.mu, self.chol, self.ea, self.eW, self.logpi)
        return _Model(self.W, self.H, self.C, self.tile, int(self.linear),
                      float(self.qmax), float(self.scale), self.K,
                      _ptr(self.mu), _ptr(self.chol), _ptr(self.ea), _ptr(self.eW),
                      int(self.rbf), _ptr(self.logpi))


def threads() -> int:
    return int(_load().om_threads())


def included(m: Model, k: int, i: int, j: int) -> bool:
    """FP32 truncation predicate q32 <= q_max for kernel k at pixel (i, j)."""
    c = m._c()
    return bool(_load().om_included(ctypes.byref(c), k, i, j))


def rect(m: Model, k: int):
    """Inclusive tile rectangle (tx0, ty0, tx1, ty1) of kernel k and its tile count."""
    r = np.zeros(4, np.int32)
    c = m._c()
    n = _load().om_rect(ctypes.byref(c), k, _ptr(r))
    return tuple(int(v) for v in r), int(n)


def bin_tiles(m: Model, tiles=None):
    """Per-tile kernel lists (Eq. 5): returns (tile_off int64[n+1], pair_k int32[P])."""
    lib = _load()
    c = m._c()
    sel = None if tiles is None else np.ascontiguousarray(tiles, dtype=np.int64)
    tx = (m.W + m.tile - 1) // m.tile
    ty = (m.H + m.tile - 1) // m.tile
    n = tx * ty if sel is None else len(sel)
    off = np.zeros(n + 1, np.int64)
    total = lib.om_bin(ctypes.byref(c), 0 if sel is None else len(sel), _ptr(sel), _ptr(off),
                       None, 0)
    pk = np.zeros(max(total, 1), np.int32)
    lib.om_bin(ctypes.byref(c), 0 if sel is None else len(sel), _ptr(sel), _ptr(off),
               _ptr(pk), total)
    return off, pk[:total]


def render(m: Model, pixels=None, with_scale=False):
    """FP64 render.  Returns (y, invd): y is (C,H,W) for a full render or
    (C,n) for the listed flat pixel indices; invd likewise (H,W) or (n,).
    with_scale=True also returns, in y's layout, sum_k w_k times the sum of the
    magnitudes of the terms of m_k (|a| + |W0 dx| + |W1 dy|): the scale of
    the rounding error of the gated sum."""
    lib = _load()
    c = m._c()
    sel = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    n = m.W * m.H if sel is None else len(sel)
    y = np.zeros((m.C, n), np.float64)
    invd = np.zeros(n, np.float64)
    absm = np.zeros((m.C, n), np.float64) if with_scale else None
    lib.om_render(ctypes.byref(c), n, _ptr(sel), _ptr(y), _ptr(invd), _ptr(absm))
    if sel is None:
        y, invd = y.reshape(m.C, m.H, m.W), invd.reshape(m.H, m.W)
        absm = None if absm is None else absm.reshape(m.C, m.H, m.W)
    return (y, invd, absm) if with_scale else (y, invd)


def render_points(m: Model, xy, with_scale=False):
    """FP64 resampling of the model at arbitrary points (Sec. II-B): xy is
    (n, 2) in the raster's pixel units (pixel (i, j) has centre (i+0.5,
    j+0.5)), taken as float32; a point outside [0,W) x [0,H) gets 0.
    Returns (y (C, n), invd (n,)) and, with with_scale, the term scale."""
    lib = _load()
    c = m._c()
    pts = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    n = len(pts)
    y = np.zeros((m.C, n), np.float64)
    invd = np.zeros(n, np.float64)
    absm = np.zeros((m.C, n), np.float64) if with_scale else None
    lib.om_render_points(ctypes.byref(c), n, _ptr(pts), _ptr(y), _ptr(invd), _ptr(absm))
    return (y, invd, absm) if with_scale else (y, invd)


def sharpen(m: Model, f: float) -> Model:
    """Native sharpening by kernel editing (Sec. II-B, Sec. VII-C): every
    kernel's bandwidth divided by the sharpening factor f, i.e. L' = f L
    (P' = f^2 P), each entry rounded to float once; the cutoff becomes
    q_max' = q_max f^2 (float32 products), so the set of included points
    stays that of the fitted model and only the gates get steeper."""
    f32 = np.float32(f)
    chol = (m.chol.astype(np.float32) * f32).astype(np.float32)
    qmax = float(np.float32(m.qmax) * (f32 * f32))
    return Model(m.W, m.H, m.C, m.mu.copy(), chol, m.ea.copy(),
                 None if m.eW is None else m.eW.copy(), tile=m.tile, qmax=qmax, scale=m.scale,
                 logpi=None if m.logpi is None else m.logpi.copy(), rbf=m.rbf)


def render_mean(models, pixels=None, with_scale=False):
    """Multi-model fusion (Sec. V-C, Eq. 11) in FP64: y_m = (1/H) sum_h y_h
    over the H models, each y_h exactly as `render` gives it (0 at a pixel
    where model h includes no kernel).  Layout as `render`'s y; with_scale
    also returns the mean over the models of `render`'s term-magnitude sum."""
    outs = [render(m, pixels, with_scale=True) for m in models]
    y = np.sum([o[0] for o in outs], axis=0) / len(models)
    if not with_scale:
        return y
    return y, np.sum([np.maximum(np.abs(o[0]), o[2]) for o in outs], axis=0) / len(models)


def mm_denoise(models, noisy, n_it, lr=(1e-2, 1e-5, 1e-3, 1e-3, 1e-3)):
    """MM-RSMoE denoising (Sec. V-C): each of the H models (the same kernel
    count, initial lattices shifted against each other) is fitted to the one
    noisy image by `fit`, then the H renders are fused by Eq. 11.  Updates
    the models in place; returns (y_m, per-model loss histories)."""
    losses = [fit(m, noisy, n_it, lr=lr) for m in models]
    return render_mean(models), losses


def backward(m: Model, gy=None, target=None, kernels=None, with_scale=False):
    """FP64 gradient of the loss w.r.t. (mu, chol, ea, eW) in API units, and
    w.r.t. logpi as a fifth entry when the model has gate weights.

    gy: upstream dL/dy (C,H,W) float64, or target (C,H,W) for the fused MSE
    loss sum((y-t)^2)/(C H W).  kernels: optional list of kernel ids.
    with_scale=True also returns, per element, the sum of the magnitudes of
    the terms that make up the gradient (the scale of FP cancellation)."""
    lib = _load()
    c = m._c()
    sel = None if kernels is None else np.ascontiguousarray(kernels, dtype=np.int64)
    n = m.K if sel is None else len(sel)

    def alloc():
        return [np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, m.C)),
                np.zeros((n, m.C, 2)) if m.linear else None,
                np.zeros(n) if m.logpi is not None else None]
    g, sc = alloc(), (alloc() if with_scale else [None] * 5)
    gy_ = None if gy is None else np.ascontiguousarray(gy, dtype=np.float64)
    t_ = None if target is None else np.ascontiguousarray(target, dtype=np.float32)
    if gy_ is None and t_ is None:
        raise ValueError("need gy or target")
    lib.om_backward(ctypes.byref(c), _ptr(gy_), _ptr(t_), 0 if sel is None else n, _ptr(sel),
                    *[_ptr(x) for x in g[:4]], *[_ptr(x) for x in sc[:4]], _ptr(g[4]),
                    _ptr(sc[4]))
    k = 5 if m.logpi is not None else 4
    return (tuple(g[:k]), tuple(sc[:k])) if with_scale else tuple(g[:k])


def fwd_bwd_binned(m: Model, target, lists=None):
    """The binned CPU baseline: forward, MSE and backward with each pixel
    visiting only its tile's list (om_bin's lists, computed here unless
    given).  Returns (mse, (g_mu, g_chol, g_ea, g_eW)); equals the dense
    render + backward up to the order of the FP64 sums."""
    lib = _load()
    c = m._c()
    off, pk = lists if lists is not None else bin_tiles(m)
    off = np.ascontiguousarray(off, dtype=np.int64)
    pk = np.ascontiguousarray(pk, dtype=np.int32)
    t_ = np.ascontiguousarray(target, dtype=np.float32)
    g = [np.zeros((m.K, 2)), np.zeros((m.K, 3)), np.zeros((m.K, m.C)),
         np.zeros((m.K, m.C, 2)) if m.linear else None]
    mse = lib.om_fwd_bwd_binned(ctypes.byref(c), _ptr(t_), _ptr(off), _ptr(pk),
                                *[_ptr(x) for x in g])
    return float(mse), tuple(g)


def adam(p, g, m_, v, lr, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """One FP64 Adam step in place (torch semantics)."""
    for a in (p, g, m_, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _load().om_adam(p.size, _ptr(p), _ptr(g), _ptr(m_), _ptr(v), lr, b1, b2, eps, step)


def lr_mu(lr0: float, lr1: float, it: int, n_it: int) -> float:
    return float(_load().om_lr_mu(lr0, lr1, it, n_it))


def fit(m: Model, target, n_it: int, lr=(1e-2, 1e-2, 1e-2, 1e-2, 1e-2),
        b1=0.9, b2=0.999, eps=1e-8):
    """FP64 Adam fit on the MSE (Sec. VI-B).  lr = (mu0, mu1, chol, ea, eW)
    and, for a model with gate weights, a sixth rate for logpi.
    Updates m's parameters in place; returns the loss history (n_it,)."""
    lib = _load()
    c = m._c()
    t_ = np.ascontiguousarray(target, dtype=np.float32)
    lr6 = list(lr) + [0.0] * (6 - len(lr))
    lr_ = np.ascontiguousarray(lr6[:6], dtype=np.float64)
    loss = np.zeros(n_it, np.float64)
    lib.om_fit(ctypes.byref(c), _ptr(t_), n_it, _ptr(lr_), b1, b2, eps, _ptr(m.mu),
               _ptr(m.chol), _ptr(m.ea), _ptr(m.eW), _ptr(m.logpi), _ptr(loss))
    return loss


def psnr(y, target) -> float:
    """PSNR in dB with peak 1 on y clamped to [0, 1], over all channels."""
    d = np.clip(np.asarray(y, np.float64), 0.0, 1.0) - np.asarray(target, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
