"""Seeded synthetic inputs: images and initial kernel sets.

This module holds no arithmetic of the regression method itself (no gate,
expert, binning, gradient or optimiser code).  It only draws inputs, and both
the CUDA path and the CPU oracle consume what it returns.  Numpy only.

Images stand in for the natural photographs of the paper's Kodak / DIV2K
workloads (neither is available here): flat-to-smooth regions separated by
sharp polygon edges, optionally with a band-limited gradient-noise texture
(Perlin's improved noise construction: a seeded permutation hash, random unit
gradients at lattice points, the 6t^5-15t^4+10t^3 fade) and additive Gaussian
noise whose *variance* is given.

Initial kernels follow the paper's initialisation (Sec. IV-A, Sec. VI-B):
round kernels spread over the image (a jittered grid), a fixed bandwidth in
pixels, constant or linear experts.  The precision factor is L = I / sigma.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------

def _star_polygon(rng, W, H):
    n = int(rng.integers(3, 9))
    cx, cy = rng.uniform(0, W), rng.uniform(0, H)
    R = rng.uniform(0.05, 0.35) * min(W, H)
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    rad = R * rng.uniform(0.5, 1.0, n)
    return np.stack([cx + rad * np.cos(ang), cy + rad * np.sin(ang)], 1), (cx, cy, R)


def _inside(poly, px, py):
    """Even-odd point-in-polygon test at the given pixel centres."""
    inside = np.zeros(px.shape, bool)
    n = len(poly)
    for e in range(n):
        x1, y1 = poly[e]
        x2, y2 = poly[(e + 1) % n]
        if y1 == y2:
            continue
        cross = (y1 > py) != (y2 > py)
        xint = (x2 - x1) * (py - y1) / (y2 - y1) + x1
        inside ^= cross & (px < xint)
    return inside


def _ramp(rng, C, px, py, cx, cy, R):
    th = rng.uniform(0, 2 * np.pi)
    d = ((px - cx) * np.cos(th) + (py - cy) * np.sin(th)) / (2.0 * R) + 0.5
    d = np.clip(d, 0.0, 1.0)
    v0 = rng.uniform(0, 1, C)
    v1 = rng.uniform(0, 1, C)
    return v0[:, None] + (v1 - v0)[:, None] * d[None, :]


def perlin(W, H, cell, rng):
    """2-D gradient noise in about [-1, 1] with lattice spacing ``cell`` px."""
    perm = rng.permutation(256)
    perm = np.concatenate([perm, perm])
    ang = rng.uniform(0, 2 * np.pi, 256)
    gx, gy = np.cos(ang), np.sin(ang)
    xs = (np.arange(W) + 0.5) / cell
    ys = (np.arange(H) + 0.5) / cell
    X, Y = np.meshgrid(xs, ys)
    xi, yi = np.floor(X).astype(np.int64), np.floor(Y).astype(np.int64)
    xf, yf = X - xi, Y - yi
    xi &= 255
    yi &= 255

    def grad(ix, iy, dx, dy):
        h = perm[perm[ix] + iy]
        return gx[h] * dx + gy[h] * dy

    fade = lambda t: t * t * t * (t * (t * 6 - 15) + 10)
    u, v = fade(xf), fade(yf)
    n00 = grad(xi, yi, xf, yf)
    n10 = grad((xi + 1) & 255, yi, xf - 1, yf)
    n01 = grad(xi, (yi + 1) & 255, xf, yf - 1)
    n11 = grad((xi + 1) & 255, (yi + 1) & 255, xf - 1, yf - 1)
    nx0 = n00 + u * (n10 - n00)
    nx1 = n01 + u * (n11 - n01)
    return (nx0 + v * (nx1 - nx0)) * math.sqrt(2.0)


def polygon_image(W, H, C, n_poly, seed, texture_amp=0.0, noise_var=0.0):
    """C x H x W float32 image: a ramp background, ``n_poly`` star polygons in
    painter's order each filled with a linear ramp, an optional Perlin texture
    of amplitude ``texture_amp`` and N(0, noise_var) noise (not clipped)."""
    rng = np.random.default_rng(seed)
    img = np.zeros((C, H, W), np.float64)
    PX, PY = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    bg = _ramp(rng, C, PX.ravel(), PY.ravel(), W / 2, H / 2, max(W, H) / 2)
    img[:] = bg.reshape(C, H, W)
    for _ in range(n_poly):
        poly, (cx, cy, R) = _star_polygon(rng, W, H)
        x0 = max(int(np.floor(poly[:, 0].min())), 0)
        x1 = min(int(np.ceil(poly[:, 0].max())) + 1, W)
        y0 = max(int(np.floor(poly[:, 1].min())), 0)
        y1 = min(int(np.ceil(poly[:, 1].max())) + 1, H)
        if x0 >= x1 or y0 >= y1:
            _ramp(rng, C, np.zeros(1), np.zeros(1), cx, cy, R)
            continue
        sx, sy = PX[y0:y1, x0:x1], PY[y0:y1, x0:x1]
        m = _inside(poly, sx, sy)
        vals = _ramp(rng, C, sx.ravel(), sy.ravel(), cx, cy, R).reshape(C, y1 - y0, x1 - x0)
        sub = img[:, y0:y1, x0:x1]
        sub[:, m] = vals[:, m]
    if texture_amp:
        for ch in range(C):
            img[ch] += texture_amp * perlin(W, H, 12.0, rng)
    if noise_var:
        img += rng.normal(0.0, math.sqrt(noise_var), img.shape)
    return img.astype(np.float32)


# --------------------------------------------------------------------------
# kernels
# --------------------------------------------------------------------------

def jittered_grid(gx, gy, seed):
    """gx*gy normalised centres, one per grid cell, jittered by U(-1/2, 1/2) cell."""
    rng = np.random.default_rng(seed)
    ix, iy = np.meshgrid(np.arange(gx), np.arange(gy))
    jx = rng.uniform(-0.5, 0.5, ix.shape)
    jy = rng.uniform(-0.5, 0.5, iy.shape)
    mu = np.stack([(ix + 0.5 + jx) / gx, (iy + 0.5 + jy) / gy], -1).reshape(-1, 2)
    return mu.astype(np.float32)


def grid_shape(K, W, H):
    """A gx x gy grid with gx*gy == K and gx/gy close to W/H."""
    best = None
    for gy in range(1, K + 1):
        if K % gy:
            continue
        gx = K // gy
        err = abs(math.log((gx / gy) / (W / H)))
        if best is None or err < best[0]:
            best = (err, gx, gy)
    return best[1], best[2]


def precision_factor(sig_u, sig_v, theta):
    """Lower-triangular L with L L^T = Sigma^-1 for a Gaussian with standard
    deviations sig_u, sig_v along axes rotated by theta (input generation)."""
    c, s = np.cos(theta), np.sin(theta)
    iu, iv = 1.0 / sig_u ** 2, 1.0 / sig_v ** 2
    p00 = c * c * iu + s * s * iv
    p01 = c * s * (iu - iv)
    p11 = s * s * iu + c * c * iv
    a = np.sqrt(p00)
    b = p01 / a
    cc = np.sqrt(np.maximum(p11 - b * b, 0.0))
    return np.stack([a, b, cc], -1)


@dataclass
class Params:
    mu: np.ndarray           # (K, 2) normalised
    chol: np.ndarray         # (K, 3)
    ea: np.ndarray           # (K, C)
    eW: np.ndarray | None    # (K, C, 2) or None
    logpi: np.ndarray | None = None   # (K,) gate weights log pi_k, or None (pi = 1)

    @property
    def K(self):
        return int(self.mu.shape[0])

    def copy(self):
        return Params(self.mu.copy(), self.chol.copy(), self.ea.copy(),
                      None if self.eW is None else self.eW.copy(),
                      None if self.logpi is None else self.logpi.copy())


def init_params(target, K, sigma, linear, seed, aniso=None, slope_std=0.0, offset=(0.0, 0.0)):
    """Initial kernel set for ``target`` (C,H,W): K kernels on a jittered grid,
    round with bandwidth ``sigma`` px (or, with aniso=(lo, hi), random
    orientation and aspect ratio in [lo, hi] at the same area), experts set to
    the target at the nearest pixel, slopes zero (or N(0, slope_std)).
    ``offset`` = (ox, oy) pixels shifts the whole grid (wrapping around the
    image), the shifted initial lattice of one model of a multi-model set."""
    C, H, W = target.shape
    gx, gy = grid_shape(K, W, H)
    mu = jittered_grid(gx, gy, seed)
    if offset[0] or offset[1]:
        mu = np.mod(mu.astype(np.float64) + np.array([offset[0] / W, offset[1] / H]), 1.0)
        mu = mu.astype(np.float32)
    rng = np.random.default_rng(seed + 7919)
    if aniso is None:
        chol = np.zeros((K, 3), np.float64)
        chol[:, 0] = 1.0 / sigma
        chol[:, 2] = 1.0 / sigma
    else:
        rho = rng.uniform(aniso[0], aniso[1], K)
        th = rng.uniform(0, np.pi, K)
        chol = precision_factor(sigma * np.sqrt(rho), sigma / np.sqrt(rho), th)
    ix = np.clip(np.floor(mu[:, 0] * W).astype(np.int64), 0, W - 1)
    iy = np.clip(np.floor(mu[:, 1] * H).astype(np.int64), 0, H - 1)
    ea = target[:, iy, ix].T.copy()
    eW = None
    if linear:
        eW = (rng.normal(0.0, slope_std, (K, C, 2)) if slope_std else np.zeros((K, C, 2)))
        eW = eW.astype(np.float32)
    return Params(mu.astype(np.float32), chol.astype(np.float32), ea.astype(np.float32), eW)


# --------------------------------------------------------------------------
# workload presets (sizes and distributions of the paper's regression tasks)
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    target: np.ndarray
    params: Params
    tile: int = 16
    qmax: float = 9.0
    iters: int = 100
    lr: tuple = (1e-2, 1e-2, 1e-2, 1e-2, 1e-2)   # mu0, mu1, chol, ea, eW
    extra: dict = field(default_factory=dict)


# The Adam rates printed in Sec. VI-B: centres 0.01 decaying exponentially to
# 0.00001, covariance factor 0.001, experts 0.001 (mu0, mu1, chol, ea, eW).
PAPER_LR = (1e-2, 1e-5, 1e-3, 1e-3, 1e-3)


def fit_rates(W, H, lr_pi=None):
    """The Sec. VI-B rates in the units of the fit API for a W x H image:
    the centre rates are read in pixels per step (0.01 px decaying to
    1e-5 px, the same on every raster size), and the API's centres are
    normalised (pixel = mu * (W, H)), so they are divided by the longer
    side; the Cholesky factor and the experts take the printed 0.001.
    lr_pi, when given, is appended as the rate of the gate weights."""
    s = 1.0 / max(W, H)
    lr = (PAPER_LR[0] * s, PAPER_LR[1] * s) + PAPER_LR[2:]
    return lr + (lr_pi,) if lr_pi is not None else lr


def plain_gray_128(seed=1):
    """128x128 grey image, 6 ramp polygons + N(0, 0.01); K=256 round kernels
    (sigma 8 px) on a 16x16 jittered grid, constant experts, 100 iterations at
    lr 1e-2, 16x16 tiles, q_max 9."""
    t = polygon_image(128, 128, 1, 6, seed, noise_var=0.01)
    p = init_params(t, 256, 8.0, False, seed)
    return Workload("gray128_K256_const", t, p, 16, 9.0, 100, (1e-2,) * 5)


def rgb_512(seed=2):
    """512x512 RGB, 40 polygons + Perlin texture (amplitude 0.1); K=16384
    sigma 5 px, linear experts, 2000 iterations at the paper's rates."""
    t = polygon_image(512, 512, 3, 40, seed, texture_amp=0.1)
    p = init_params(t, 16384, 5.0, True, seed)
    return Workload("rgb512_K16384_linear", t, p, 16, 9.0, 2000, PAPER_LR)


def rgb_2048(seed=3, aniso=(1.0, 3.0), slope_std=2e-3):
    """2048x2048 RGB of the same generator; K=262144 anisotropic kernels of
    area-equivalent sigma 5 px with linear experts."""
    t = polygon_image(2048, 2048, 3, 40, seed, texture_amp=0.1)
    p = init_params(t, 262144, 5.0, True, seed, aniso=aniso, slope_std=slope_std)
    return Workload("rgb2048_K262144_linear_aniso", t, p, 16, 9.0, 1, PAPER_LR)


def denoise_case(W=768, H=512, noise_var=0.01, seed=5):
    """Denoising input at the size of the paper's 768x512 RGB test images:
    a clean synthetic image (30 ramp polygons + Perlin texture 0.1, values
    clipped to [0, 1]) and the same image plus N(0, noise_var) noise (not
    clipped).  Returns (clean, noisy), each (3, H, W) float32."""
    clean = np.clip(polygon_image(W, H, 3, 30, seed, texture_amp=0.1), 0.0, 1.0)
    rng = np.random.default_rng(seed + 104729)
    noisy = clean + rng.normal(0.0, math.sqrt(noise_var), clean.shape)
    return clean.astype(np.float32), noisy.astype(np.float32)


def ragged_sizes(n=64, seed=4):
    """Log-uniform image sizes from 128x96 to 1920x1080: t ~ U(0, 1) with the
    first two draws set to the end points, W = round(128 * 15^t),
    H = round(96 * 11.25^t)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 1.0, n)
    t[:2] = (0.0, 1.0)[:n]
    W = np.rint(128 * 15.0 ** t).astype(int)
    H = np.rint(96 * 11.25 ** t).astype(int)
    return list(zip(W.tolist(), H.tolist()))
