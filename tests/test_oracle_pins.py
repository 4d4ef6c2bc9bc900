"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties one oracle function to a value the mathematics fixes: closed
forms (normalised-RBF / logistic special cases computed with scipy), library
routines (numpy eigen decomposition / inverse / Cholesky, torch float64
autograd, torch.optim.Adam), invariants of the method (gates sum to one, a
single kernel reproduces its expert, zero gradient at an exact fit) and brute
force on tiny inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.special

from paper_2510_05814_gb300 import synth


def rand_model(om, rng, W=24, H=20, C=3, K=12, linear=True, tile=8, qmax=9.0, sig=(2.0, 6.0)):
    """Random anisotropic kernels; L from numpy's Cholesky of inv(Sigma)."""
    mu = rng.uniform(0.0, 1.0, (K, 2))
    chol = np.zeros((K, 3))
    for k in range(K):
        s = rng.uniform(*sig, 2)
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        Sig = R @ np.diag(s ** 2) @ R.T
        L = np.linalg.cholesky(np.linalg.inv(Sig))
        chol[k] = (L[0, 0], L[1, 0], L[1, 1])
    ea = rng.uniform(0, 1, (K, C))
    eW = rng.normal(0, 0.05, (K, C, 2)) if linear else None
    return om.Model(W, H, C, mu, chol, ea, eW, tile=tile, qmax=qmax)


def kernel_px64(m, k, scale=1.0):
    """Centre (float32 product, the model's definition) and precision P=L L^T."""
    mx = np.float32(m.mu[k, 0]) * np.float32(m.W)
    my = np.float32(m.mu[k, 1]) * np.float32(m.H)
    a, b, c = (float(np.float32(v) / np.float32(scale)) for v in m.chol[k])
    L = np.array([[a, 0.0], [b, c]])
    return np.array([float(mx), float(my)]), L @ L.T


def q64(m, k, i, j, scale=1.0):
    c, P = kernel_px64(m, k, scale)
    d = np.array([i + 0.5, j + 0.5]) - c
    return float(d @ P @ d)


# ---------------------------------------------------------------- predicate

def test_predicate_agrees_with_fp64_quadratic_form(om):
    """Sec. IV truncation: away from the boundary the FP32 predicate equals
    (x-mu)^T L L^T (x-mu) <= q_max evaluated in FP64 with numpy matmul.  An
    anisotropic L catches L vs L^T, a dropped cross term or a wrong sign."""
    rng = np.random.default_rng(0)
    m = rand_model(om, rng, W=40, H=36, K=20)
    n_far = 0
    for k in range(m.K):
        for j in range(m.H):
            for i in range(m.W):
                q = q64(m, k, i, j)
                if abs(q - m.qmax) > 1e-3:
                    n_far += 1
                    assert om.included(m, k, i, j) == (q <= m.qmax), (k, i, j, q)
    assert n_far > 20000


def test_predicate_tie_is_included(om):
    """q == q_max exactly is included (the cutoff is q <= q_max).  With
    L = [[1/2, 0], [1/2, 1/2]] and a centre on a pixel centre, (dx, dy) =
    (6, 0) gives z = (3, 0) and (-6, 6) gives z = (0, 3): q = 9 exactly in
    binary; one pixel further out is excluded."""
    W = H = 64
    mu = np.array([[20.5 / 64, 30.5 / 64]])            # exact: centre (20.5, 30.5)
    m = om.Model(W, H, 1, mu, np.array([[0.5, 0.5, 0.5]]), np.array([[1.0]]))
    assert om.included(m, 0, 26, 30)                   # dx=6, dy=0 -> q=9
    assert not om.included(m, 0, 27, 30)               # dx=7 -> q=12.25
    assert om.included(m, 0, 14, 36)                   # dx=-6, dy=6 -> q=9
    assert not om.included(m, 0, 14, 37)               # dy=7 -> q=10.25
    assert q64(m, 0, 26, 30) == 9.0 and q64(m, 0, 14, 36) == 9.0


# ---------------------------------------------------------------- bounding box

def test_rect_hand_computed():
    """Isotropic sigma=4 px at (20, 20), q_max=9: r = 12 (1+2^-10), the box
    [7.988, 32.012]^2 covers 8x8 tiles 0..4 (Fig. 3b, square box)."""
    import oracle as om
    m = om.Model(64, 64, 1, np.array([[20 / 64, 20 / 64]]), np.array([[0.25, 0.0, 0.25]]),
                 np.array([[1.0]]), tile=8)
    assert om.rect(m, 0) == ((0, 0, 4, 4), 25)
    m.tile = 16
    assert om.rect(m, 0) == ((0, 0, 2, 2), 9)
    # far off-image: empty
    m2 = om.Model(64, 64, 1, np.array([[2.0, 0.5]]), np.array([[0.25, 0.0, 0.25]]),
                  np.array([[1.0]]), tile=8)
    assert om.rect(m2, 0)[1] == 0


def test_rect_contains_ellipse_and_is_tight(om):
    """The box side is the major axis of the q_max ellipse (Fig. 3b):
    half side = sqrt(q_max * max eig(Sigma)) from numpy.linalg.eigvalsh."""
    rng = np.random.default_rng(1)
    m = rand_model(om, rng, W=200, H=180, K=200, tile=8, sig=(0.5, 20.0))
    tx, ty = (m.W + 7) // 8, (m.H + 7) // 8
    for k in range(m.K):
        c, P = kernel_px64(m, k)
        r = math.sqrt(m.qmax * np.linalg.eigvalsh(np.linalg.inv(P)).max())
        (x0, y0, x1, y1), n = om.rect(m, k)
        lo = np.floor((c - r * (1 + 1e-6)) / 8)
        hi = np.floor((c + r * (1 + 2e-3)) / 8)
        lo2 = np.floor((c - r * (1 + 2e-3)) / 8)
        hi2 = np.floor((c + r * (1 - 1e-6)) / 8)
        # contains the exact box, and is within a 0.2% wider one
        assert x0 <= max(lo[0], 0) and y0 <= max(lo[1], 0)
        assert x1 >= min(hi2[0], tx - 1) and y1 >= min(hi2[1], ty - 1)
        assert x0 >= max(lo2[0], 0) and y0 >= max(lo2[1], 0)
        assert x1 <= min(hi[0], tx - 1) and y1 <= min(hi[1], ty - 1)
        assert n == (x1 - x0 + 1) * (y1 - y0 + 1)


def degenerate_model(om, W=40, H=33, tile=8):
    mu = [[0.5, 0.5], [0.5, 0.5], [0.5, 0.5], [0.3, 0.7], [1.4, 0.5], [-0.2, -0.2],
          [0.0, 0.0], [1.0, 1.0], [0.5, 0.5], [np.nan, 0.5], [0.25, 0.25], [0.6, 0.4],
          [0.125, 0.24242424]]
    chol = [[0.0, 0.3, 0.3],     # a = 0: band in x
            [0.3, 0.1, 0.0],     # c = 0: line band
            [1e-30, 0.0, 1e-30],  # det underflows
            [5.0, 0.0, 5.0],     # tiny kernel
            [0.2, 0.0, 0.2],     # off image right, reaches in
            [0.05, 0.0, 0.05],   # off image, huge
            [0.5, 0.0, 0.5],     # on the corner
            [0.5, 0.0, 0.5],
            [np.inf, 0.0, 0.3],  # non-finite
            [0.3, 0.0, 0.3],     # NaN centre
            [-0.3, 0.2, -0.4],   # negative diagonal (sign is free)
            [0.25, -0.9, 0.05],  # very elongated
            [1 / 3.0, 0.0, 1 / 3.0]]  # centre on a tile edge (5 px, 8 px)
    K = len(mu)
    return om.Model(W, H, 1, np.array(mu), np.array(chol), np.ones((K, 1)), tile=tile)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_binning_conservative_exhaustive(om, tile):
    """Every included (pixel, kernel) pair lies in a tile whose list holds the
    kernel (Eq. 5 must not drop a pair the truncated model keeps); lists are
    ascending and their sizes sum to the rectangles' tile counts."""
    rng = np.random.default_rng(2)
    models = [rand_model(om, rng, W=53, H=47, K=40, tile=tile, sig=(0.3, 12.0)),
              degenerate_model(om, tile=tile)]
    for m in models:
        off, pk = om.bin_tiles(m)
        tx = (m.W + tile - 1) // tile
        lists = [set(pk[off[t]:off[t + 1]].tolist()) for t in range(len(off) - 1)]
        for t in range(len(off) - 1):
            seg = pk[off[t]:off[t + 1]]
            assert np.all(np.diff(seg) > 0)
        assert off[-1] == sum(om.rect(m, k)[1] for k in range(m.K))
        for k in range(m.K):
            for j in range(m.H):
                for i in range(m.W):
                    if om.included(m, k, i, j):
                        assert k in lists[(j // tile) * tx + i // tile], (k, i, j)


def test_degenerate_rects(om):
    m = degenerate_model(om)
    tx, ty = 5, 5
    assert om.rect(m, 0) == ((0, 0, tx - 1, ty - 1), 25)   # a = 0 -> whole image
    assert om.rect(m, 1) == ((0, 0, tx - 1, ty - 1), 25)   # c = 0
    assert om.rect(m, 2) == ((0, 0, tx - 1, ty - 1), 25)   # det underflow
    assert om.rect(m, 8)[1] == 0                           # inf in L: nothing passes
    assert om.rect(m, 9)[1] == 0                           # NaN centre
    for k in (8, 9):
        assert not any(om.included(m, k, i, j) for i in range(m.W) for j in range(m.H))


def test_bin_selected_tiles_match_full(om):
    rng = np.random.default_rng(3)
    m = rand_model(om, rng, W=64, H=48, K=30, tile=16)
    off, pk = om.bin_tiles(m)
    sel = [5, 0, 11]
    off2, pk2 = om.bin_tiles(m, sel)
    for s, t in enumerate(sel):
        assert pk2[off2[s]:off2[s + 1]].tolist() == pk[off[t]:off[t + 1]].tolist()


# ---------------------------------------------------------------- render

def test_single_kernel_reproduces_expert(om):
    """Eq. 3/4 with one kernel: the gate is 1 where it is included, so y is its
    expert exactly (constant and linear m(x) = a + W (x - mu)); elsewhere the
    empty-pixel rule gives y = 0."""
    for linear in (False, True):
        m = om.Model(30, 26, 3, np.array([[0.41, 0.55]]), np.array([[0.21, -0.07, 0.15]]),
                     np.array([[0.2, 0.5, 0.9]]),
                     np.array([[[0.01, -0.02], [0.03, 0.0], [-0.01, 0.015]]]) if linear else None)
        y, invd = om.render(m)
        mx, my = float(np.float32(0.41) * np.float32(30)), float(np.float32(0.55) * np.float32(26))
        n_in = 0
        for j in range(m.H):
            for i in range(m.W):
                if om.included(m, 0, i, j):
                    n_in += 1
                    exp = m.ea[0].astype(np.float64).copy()
                    if linear:
                        exp += m.eW[0].astype(np.float64) @ np.array([i + 0.5 - mx, j + 0.5 - my])
                    np.testing.assert_allclose(y[:, j, i], exp, rtol=1e-14, atol=1e-15)
                    q = q64(m, 0, i, j)
                    assert invd[j, i] == pytest.approx(math.exp(0.5 * q), rel=1e-12)
                else:
                    assert np.all(y[:, j, i] == 0) and invd[j, i] == 0
        assert n_in > 100


def test_gates_sum_to_one_and_constant_image(om):
    """Softmax gates (Eq. 4) sum to 1 wherever any kernel is included: unit
    experts give y = 1; equal constant experts v give y = v (a constant image
    stays constant); uncovered pixels give 0."""
    rng = np.random.default_rng(4)
    m = rand_model(om, rng, W=40, H=30, K=15, linear=False, sig=(1.0, 4.0))
    covered = np.array([[any(om.included(m, k, i, j) for k in range(m.K)) for i in range(m.W)]
                        for j in range(m.H)])
    assert covered.any() and (~covered).any()
    m.ea[:] = 1.0
    y, _ = om.render(m)
    np.testing.assert_allclose(y[:, covered], 1.0, rtol=1e-14)
    assert np.all(y[:, ~covered] == 0)
    v = np.array([0.25, 0.6, 0.8], np.float32)
    m.ea[:] = v
    y, _ = om.render(m)
    for ch in range(3):
        np.testing.assert_allclose(y[ch][covered], v[ch], rtol=1e-13)


def test_no_cutoff_limit_is_normalised_rbf(om):
    """With q_max -> inf the truncated model is the global SMoE (Sec. III-B):
    y = sum_k softmax_k(-q_k/2) m_k, q_k = d^T inv(Sigma_k) d.  Expected values
    use scipy's softmax and numpy's inverse of Sigma (not L)."""
    rng = np.random.default_rng(5)
    K, W, H = 7, 16, 12
    mu = rng.uniform(0.1, 0.9, (K, 2))
    Sigs, chol = [], np.zeros((K, 3))
    for k in range(K):
        s = rng.uniform(2.0, 5.0, 2)
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        Sig = R @ np.diag(s ** 2) @ R.T
        L = np.linalg.cholesky(np.linalg.inv(Sig))
        chol[k] = (L[0, 0], L[1, 0], L[1, 1])
    chol = chol.astype(np.float32)
    for k in range(K):  # Sigma of the float parameters, via its inverse
        a, b, c = chol[k].astype(np.float64)
        Sigs.append(np.linalg.inv(np.array([[a * a, a * b], [a * b, b * b + c * c]])))
    ea = rng.uniform(0, 1, (K, 1))
    m = om.Model(W, H, 1, mu, chol, ea, tile=8, qmax=1e30)
    y, _ = om.render(m)
    centres = np.stack([np.float32(mu[:, 0]).astype(np.float32) * np.float32(W),
                        np.float32(mu[:, 1]).astype(np.float32) * np.float32(H)], 1).astype(np.float64)
    for j in range(H):
        for i in range(W):
            d = np.array([i + 0.5, j + 0.5]) - centres
            q = np.array([d[k] @ np.linalg.solve(Sigs[k], d[k]) for k in range(K)])
            w = scipy.special.softmax(-0.5 * q)
            assert y[0, j, i] == pytest.approx(float(w @ m.ea[:, 0]), rel=1e-10, abs=1e-12)


def test_two_kernel_logistic_closed_form(om):
    """Two constant experts: y = m2 + (m1 - m2) * expit((q2 - q1)/2) where both
    kernels are included (Eq. 4 for two gates is a logistic function)."""
    m = om.Model(32, 16, 1, np.array([[0.35, 0.5], [0.6, 0.45]]),
                 np.array([[0.2, 0.05, 0.18], [0.15, -0.04, 0.22]]), np.array([[0.1], [0.9]]))
    y, _ = om.render(m)
    n = 0
    for j in range(m.H):
        for i in range(m.W):
            if om.included(m, 0, i, j) and om.included(m, 1, i, j):
                n += 1
                q1, q2 = q64(m, 0, i, j), q64(m, 1, i, j)
                e = 0.9 + (0.1 - 0.9) * scipy.special.expit(0.5 * (q2 - q1))
                assert y[0, j, i] == pytest.approx(float(np.float32(0.9)) + (float(np.float32(0.1)) - float(np.float32(0.9))) * scipy.special.expit(0.5 * (q2 - q1)), rel=1e-12)
                assert abs(y[0, j, i] - e) < 1e-6
    assert n > 50


def test_brute_force_4x4_rational(om):
    """4x4 image, 3 kernels: gate ratios summed in exact rational arithmetic
    (exp values taken as doubles) agree with the oracle to FP64 rounding."""
    rng = np.random.default_rng(6)
    m = rand_model(om, rng, W=4, H=4, C=1, K=3, linear=False, tile=8, sig=(1.0, 3.0))
    y, _ = om.render(m)
    for j in range(4):
        for i in range(4):
            num, den = Fraction(0), Fraction(0)
            for k in range(3):
                if om.included(m, k, i, j):
                    e = Fraction(math.exp(-0.5 * q64(m, k, i, j)))
                    num += e * Fraction(float(m.ea[k, 0]))
                    den += e
            ref = float(num / den) if den else 0.0
            assert y[0, j, i] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_super_resolution_linear_expert(om):
    """Native super-resolution (Sec. II-B, VII-C): rendering at scale s samples
    the same continuous function.  One kernel with a linear expert rendered at
    s = 2 equals a + W (x'/2 - mu) at the included fine pixels."""
    mu = np.array([[0.5, 0.4]])
    m = om.Model(20, 20, 1, mu, np.array([[0.25, 0.0, 0.25]]), np.array([[0.3]]),
                 np.array([[[0.02, -0.01]]]))
    sr = om.Model(40, 40, 1, mu, m.chol, m.ea, m.eW, scale=2.0)
    y2, _ = om.render(sr)
    n = 0
    for j in range(40):
        for i in range(40):
            x = np.array([(i + 0.5) / 2, (j + 0.5) / 2])
            q = float(((x - np.array([10.0, 8.0])) ** 2).sum() * 0.0625)
            if abs(q - 9.0) < 1e-3:
                continue
            assert om.included(sr, 0, i, j) == (q <= 9.0)
            if q <= 9.0:
                n += 1
                ref = 0.3 + 0.02 * (x[0] - 10.0) - 0.01 * (x[1] - 8.0)
                assert y2[0, j, i] == pytest.approx(float(np.float32(0.3)) + float(np.float32(0.02)) * (x[0] - 10.0) + float(np.float32(-0.01)) * (x[1] - 8.0), rel=1e-12)
                assert abs(y2[0, j, i] - ref) < 1e-6
    assert n > 400


# ---------------------------------------------------------------- backward

def dense_torch_loss(m, mask, gy, scale=1.0, with_y=False):
    """The truncated model written densely in torch float64 (for autograd):
    softmax gates with weights pi = exp(logpi) (Eq. 4), or the RBF sum of
    Eq. 1 when m.rbf."""
    import torch
    mu = torch.tensor(m.mu, dtype=torch.float64, requires_grad=True)
    chol = torch.tensor(m.chol, dtype=torch.float64, requires_grad=True)
    ea = torch.tensor(m.ea, dtype=torch.float64, requires_grad=True)
    eW = torch.tensor(m.eW, dtype=torch.float64, requires_grad=True) if m.linear else None
    lp = (torch.tensor(m.logpi, dtype=torch.float64, requires_grad=True)
          if m.logpi is not None else None)
    jj, ii = torch.meshgrid(torch.arange(m.H, dtype=torch.float64),
                            torch.arange(m.W, dtype=torch.float64), indexing="ij")
    X = torch.stack([ii.reshape(-1) + 0.5, jj.reshape(-1) + 0.5], 1)          # (HW, 2)
    # The centre is the float product mu*W; its derivative w.r.t. mu is W.
    c_f = torch.tensor(np.stack([np.float32(m.mu[:, 0]) * np.float32(m.W),
                                 np.float32(m.mu[:, 1]) * np.float32(m.H)], 1), dtype=torch.float64)
    scale_wh = torch.tensor([m.W, m.H], dtype=torch.float64)
    centre = c_f + (mu - mu.detach()) * scale_wh
    # L' = L / s and eW' = eW / s are rounded to float (the model's
    # definition); their derivatives are 1/s.
    def fdiv(t):
        exact = t / scale
        rounded = torch.tensor((t.detach().numpy().astype(np.float32) / np.float32(scale)),
                               dtype=torch.float64)
        return exact + (rounded - exact).detach()
    Lf = fdiv(chol)
    d = X[:, None, :] - centre[None]                                             # (HW, K, 2)
    z0 = Lf[:, 0] * d[..., 0] + Lf[:, 1] * d[..., 1]
    z1 = Lf[:, 2] * d[..., 1]
    arg = -0.5 * (z0 * z0 + z1 * z1)
    if lp is not None:
        arg = arg + lp[None]
    e = torch.exp(arg) * torch.tensor(mask, dtype=torch.float64)
    mexp = ea[None].expand(X.shape[0], -1, -1)
    if m.linear:
        mexp = mexp + torch.einsum("kcd,pkd->pkc", fdiv(eW), d)
    D = e.sum(1)
    if m.rbf:
        y = (e[..., None] * mexp).sum(1)
    else:
        y = (e[..., None] * mexp).sum(1) / torch.where(D > 0, D, torch.ones_like(D))[:, None]
    loss = (y.T.reshape(m.C, m.H, m.W) * torch.tensor(gy)).sum()
    leaves = [mu, chol, ea] + ([eW] if m.linear else []) + ([lp] if lp is not None else [])
    grads = [g.numpy() for g in torch.autograd.grad(loss, leaves)]
    if with_y:
        return grads, y.detach().T.reshape(m.C, m.H, m.W).numpy()
    return grads


def inclusion_mask(om, m):
    return np.array([[om.included(m, k, p % m.W, p // m.W) for k in range(m.K)]
                     for p in range(m.W * m.H)], np.float64)


@pytest.mark.parametrize("linear,scale,pi,rbf", [(False, 1.0, False, False),
                                                  (True, 1.0, False, False),
                                                  (True, 1.5, False, False),
                                                  (True, 1.0, True, False),
                                                  (False, 1.0, True, True),
                                                  (True, 1.5, True, True)])
def test_backward_matches_torch_autograd(om, linear, scale, pi, rbf):
    """Analytic backward (the a.e. gradient of the truncated model) equals
    torch float64 autograd of the dense formula, for every parameter group:
    softmax gates with and without gate weights pi (Eq. 4), and the RBF sum
    of Eq. 1; the renders agree as well."""
    rng = np.random.default_rng(7)
    m = rand_model(om, rng, W=22, H=18, K=9, linear=linear, sig=(2.0, 5.0))
    m.W, m.H, m.scale = int(22 * scale), int(18 * scale), scale
    if pi:
        m.logpi = rng.normal(0, 0.7, m.K).astype(np.float32)
    m.rbf = rbf
    gy = rng.normal(0, 1, (m.C, m.H, m.W))
    mask = inclusion_mask(om, m)
    ref, y_ref = dense_torch_loss(m, mask, gy, scale, with_y=True)
    got = [g for g in om.backward(m, gy=gy) if g is not None]
    assert len(got) == len(ref)
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g, r, rtol=1e-9, atol=1e-12 * np.abs(r).max())
    np.testing.assert_allclose(om.render(m)[0], y_ref, rtol=1e-12, atol=1e-14)


def test_backward_fused_mse_and_selected_kernels(om):
    """The fused MSE upstream G = 2(y-t)/(CHW) equals passing that gy
    explicitly; a kernel subset returns the same rows."""
    rng = np.random.default_rng(8)
    m = rand_model(om, rng, W=20, H=16, K=10)
    t = rng.uniform(0, 1, (m.C, m.H, m.W)).astype(np.float32)
    y, _ = om.render(m)
    gy = 2.0 * (y - t.astype(np.float64)) / y.size
    a = om.backward(m, gy=gy)
    b = om.backward(m, target=t)
    sel = [7, 2, 9]
    c = om.backward(m, target=t, kernels=sel)
    for x, z, w in zip(a, b, c):
        np.testing.assert_allclose(z, x, rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(w, x[sel], rtol=1e-12, atol=1e-18)


def test_backward_term_scale_bounds_gradient(om):
    """The optional term-magnitude sums bound the gradients (triangle
    inequality) and equal them for a single all-positive term."""
    rng = np.random.default_rng(12)
    m = rand_model(om, rng, W=20, H=18, K=8)
    gy = rng.normal(0, 1, (m.C, m.H, m.W))
    g, s = om.backward(m, gy=gy, with_scale=True)
    for a, b in zip(g, s):
        assert np.all(np.abs(a) <= b * (1 + 1e-12) + 1e-300)
    g2, s2 = om.backward(m, gy=np.abs(gy), with_scale=True)
    np.testing.assert_allclose(np.abs(g2[2]), s2[2], rtol=1e-12)   # ea: terms g*|G| >= 0


def test_backward_central_differences(om):
    """Central differences of the oracle's own FP64 render agree with its
    analytic gradient on parameters whose inclusion pattern does not change."""
    rng = np.random.default_rng(9)
    m = rand_model(om, rng, W=18, H=16, K=6, sig=(2.5, 4.0))
    gy = rng.normal(0, 1, (m.C, m.H, m.W))
    g = om.backward(m, gy=gy)
    base = inclusion_mask(om, m)
    groups = [m.mu, m.chol, m.ea, m.eW]
    checked = 0
    for gi, arr in enumerate(groups):
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, min(flat.size, 12), replace=False):
            v0 = flat[idx]
            h = np.float32(2e-3 * max(1.0, abs(v0)) if gi != 0 else 2e-3)
            vals = []
            for sgn in (1, -1):
                flat[idx] = np.float32(v0 + sgn * h)
                if not np.array_equal(inclusion_mask(om, m), base):
                    vals = None
                    break
                vals.append(float((om.render(m)[0] * gy).sum()))
            real_h = (float(np.float32(v0 + h)) - float(np.float32(v0 - h))) / 2
            flat[idx] = v0
            if vals is None:
                continue
            fd = (vals[0] - vals[1]) / (2 * real_h)
            an = g[gi].reshape(-1)[idx]
            assert fd == pytest.approx(an, rel=2e-3, abs=2e-4 * np.abs(g[gi]).max()), (gi, idx)
            checked += 1
    assert checked >= 24


def test_zero_gradient_at_exact_fit(om):
    """If the target equals the model output the MSE gradient vanishes: equal
    constant experts 0.5 give y = 0.5 exactly where covered (0 elsewhere)."""
    rng = np.random.default_rng(10)
    m = rand_model(om, rng, W=24, H=20, K=10, linear=True)
    m.ea[:] = 0.5
    m.eW[:] = 0.0
    y, _ = om.render(m)
    assert set(np.unique(y)) <= {0.0, 0.5}
    g = om.backward(m, target=y.astype(np.float32))
    for x in g:
        assert np.all(x == 0.0)
    # a general model fitted exactly up to float rounding of the target
    m = rand_model(om, rng, W=24, H=20, K=10, linear=True)
    y, _ = om.render(m)
    g0 = om.backward(m, target=y.astype(np.float32))
    g1 = om.backward(m, target=(y + 0.05).astype(np.float32))
    for a, b in zip(g0, g1):
        assert np.abs(a).max() < 1e-5 * np.abs(b).max()


# ---------------------------------------------------------------- Adam / fit

def test_adam_matches_torch(om):
    """Adam (Sec. VI-B) equals torch.optim.Adam in float64 over several steps."""
    import torch
    rng = np.random.default_rng(11)
    p = rng.normal(0, 1, 50)
    m_, v = np.zeros(50), np.zeros(50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(0, 1, 50) * (10.0 ** rng.integers(-6, 2))
        om.adam(p, g.copy(), m_, v, 3e-3, 0.9, 0.999, 1e-8, step)
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_lr_schedule_closed_form(om):
    """mu learning rate decays exponentially from 1e-2 to 1e-5 (Sec. VI-B)."""
    assert om.lr_mu(1e-2, 1e-5, 0, 100) == pytest.approx(1e-2, rel=1e-15)
    assert om.lr_mu(1e-2, 1e-5, 99, 100) == pytest.approx(1e-5, rel=1e-12)
    assert om.lr_mu(1e-2, 1e-5, 33, 100) == pytest.approx(1e-2 * 1e-3 ** (33 / 99), rel=1e-12)
    assert om.lr_mu(1e-2, 1e-5, 0, 1) == pytest.approx(1e-2)


def test_fit_step_edge_figure2_toy(om):
    """Fig. 2 toy: a 21-sample step from 0.1 to 0.9 (a 21x1 image).  Two SMoE
    kernels fitted by Adam through the oracle reach a high PSNR on the clean
    step (the paper reports ~27 dB on a noisy one) and the loss decreases."""
    t = np.where(np.arange(21) < 10, 0.1, 0.9).astype(np.float32).reshape(1, 1, 21)
    mu = np.array([[6 / 21, 0.5], [15 / 21, 0.5]])
    chol = np.array([[0.25, 0.0, 0.25], [0.25, 0.0, 0.25]])
    m = om.Model(21, 1, 1, mu, chol, np.array([[0.3], [0.7]]), tile=8, qmax=1e30)
    loss = om.fit(m, t, 300, lr=(5e-3, 5e-3, 2e-2, 2e-2, 0.0))
    assert loss[-1] < loss[0] * 1e-2
    y, _ = om.render(m)
    assert om.psnr(y, t) > 27.0


def test_fit_decreases_loss_on_synthetic(om):
    wl = synth.plain_gray_128()
    # a small crop keeps the dense oracle fast
    t = wl.target[:, :48, :48].copy()
    p = synth.init_params(t, 36, 8.0 * 48 / 128, False, 1)
    m = om.Model(48, 48, 1, p.mu, p.chol, p.ea, tile=16)
    loss = om.fit(m, t, 20, lr=(1e-2,) * 5)
    assert loss[-1] < 0.8 * loss[0]
    assert np.all(np.isfinite(loss))


# ---------------------------------------------------------------- accounting

def test_flop_convention_from_tables():
    """Tables I/II print FLOPs per pixel next to the average kernels per block;
    the paper's convention is FLOPs/px = 2 x avg kernels/block (up to the
    rounding of the printed averages).  The benchmark reports pair counts in
    the same convention."""
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables_flops.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()[:2]])
    assert len(rows) >= 7
    for avg, flops in rows:
        assert abs(flops - 2 * avg) <= 2.0


# ---------------------------------------------------------------- multi-model fusion

def test_render_mean_of_constant_models(om):
    """Eq. 11 on models whose experts are one constant colour c_h each: the
    gates of a model sum to one, so model h renders exactly c_h wherever it
    includes a kernel and 0 elsewhere, and the fused image is the mean of
    those over all H models."""
    rng = np.random.default_rng(60)
    cols = [np.array([0.2, 0.4, 0.6]), np.array([0.9, 0.1, 0.5]), np.array([0.35, 0.8, 0.05])]
    models = []
    for h, c in enumerate(cols):
        m = rand_model(om, rng, W=24, H=20, C=3, K=6 + 3 * h, linear=False, sig=(1.0, 2.5))
        m.ea[:] = c
        models.append(m)
    y = om.render_mean(models)
    expect = np.zeros((3, 20, 24))
    covered_by = np.zeros((20, 24), int)
    for m, c in zip(models, cols):
        cov = om.render(m)[1] > 0
        covered_by += cov
        expect += c.astype(np.float32).astype(np.float64)[:, None, None] * cov   # FP32 experts
    expect /= len(models)
    assert np.any(covered_by < len(models))       # some pixels miss some models
    assert np.any(covered_by == len(models))
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-12)


def test_render_mean_error_is_at_most_the_mean_model_error(om):
    """Convexity of the squared error: the fused image's squared error to any
    target is at most the mean of the models' squared errors (equal only
    when the renders coincide), and fusing copies of one model, or one model
    alone, returns its render; the order of the models does not matter."""
    rng = np.random.default_rng(61)
    models = [rand_model(om, rng, W=20, H=16, C=3, K=9, linear=True) for _ in range(4)]
    t = rng.uniform(0, 1, (3, 16, 20))
    y = om.render_mean(models)
    singles = [om.render(m)[0] for m in models]
    err_fused = np.sum((y - t) ** 2)
    err_mean = np.mean([np.sum((s - t) ** 2) for s in singles])
    assert err_fused < err_mean
    np.testing.assert_allclose(om.render_mean(models[::-1]), y, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(om.render_mean([models[2]]), singles[2])
    np.testing.assert_allclose(om.render_mean([models[1]] * 3), singles[1], rtol=0, atol=1e-15)


def test_mm_denoise_fuses_fitted_models(om):
    """The MM-RSMoE pipeline on a small noisy image: every model's loss goes
    down and the fused image is the mean of the fitted models' renders."""
    clean, noisy = synth.denoise_case(24, 16, 0.01, seed=62)
    models = []
    for h, off in enumerate([(0, 0), (4, 0), (0, 4), (4, 4)]):
        p = synth.init_params(noisy, 12, 3.0, True, 62 + h, offset=off)
        models.append(om.Model(24, 16, 3, p.mu, p.chol, p.ea, p.eW, tile=8))
    y, losses = om.mm_denoise(models, noisy, 15, lr=(1e-2, 1e-3, 1e-2, 1e-2, 1e-2))
    for l in losses:
        assert l[-1] < l[0]
    np.testing.assert_allclose(y, np.mean([om.render(m)[0] for m in models], axis=0),
                               rtol=0, atol=1e-14)


# ---------------------------------------------------------------- resampling and sharpening

def qxy(m, k, x, y):
    """FP64 quadratic form of kernel k at the point (x, y) (numpy matmul)."""
    c, P = kernel_px64(m, k)
    d = np.array([x, y], np.float64) - c
    return float(d @ P @ d)


def test_points_at_pixel_centres_equal_render(om):
    rng = np.random.default_rng(70)
    m = rand_model(om, rng, W=26, H=19, C=3, K=14, linear=True)
    y, invd = om.render(m)
    xs = np.stack(np.meshgrid(np.arange(26) + 0.5, np.arange(19) + 0.5), -1).reshape(-1, 2)
    yp, ip = om.render_points(m, xs)
    np.testing.assert_array_equal(yp, y.reshape(3, -1))
    np.testing.assert_array_equal(ip, invd.reshape(-1))


def test_points_single_kernel_closed_form(om):
    """One kernel with a linear expert evaluated at random continuous points:
    y = ea + eW (x - mu) where the point is inside the cutoff (numpy FP64
    quadratic form), 0 outside; 1/D = exp(q/2).  Catches an x/y swap of the
    point coordinates or of the slopes."""
    m = om.Model(30, 22, 3, np.array([[0.37, 0.58]]), np.array([[0.23, -0.09, 0.17]]),
                 np.array([[0.2, 0.5, 0.9]]),
                 np.array([[[0.02, -0.03], [0.05, 0.01], [-0.01, 0.025]]]))
    rng = np.random.default_rng(71)
    pts = rng.uniform([0, 0], [30, 22], (400, 2)).astype(np.float32)
    y, invd = om.render_points(m, pts)
    c, _ = kernel_px64(m, 0)
    n_in = 0
    for p in range(len(pts)):
        q = qxy(m, 0, pts[p, 0], pts[p, 1])
        if abs(q - 9.0) < 1e-4:
            continue
        if q < 9.0:
            n_in += 1
            d = pts[p].astype(np.float64) - c
            np.testing.assert_allclose(y[:, p], m.ea[0] + m.eW[0].astype(np.float64) @ d,
                                       rtol=1e-13, atol=1e-15)
            assert invd[p] == pytest.approx(math.exp(0.5 * q), rel=1e-10)
        else:
            assert np.all(y[:, p] == 0) and invd[p] == 0
    assert n_in > 40


def test_points_outside_the_raster_are_zero(om):
    rng = np.random.default_rng(72)
    m = rand_model(om, rng, W=16, H=12, C=1, K=6, linear=False, sig=(6.0, 9.0))
    pts = np.array([[-0.01, 3.0], [16.0, 3.0], [3.0, 12.0], [3.0, -1e-6], [np.nan, 2.0],
                    [2.0, np.inf], [15.999, 11.999], [0.0, 0.0]], np.float32)
    y, invd = om.render_points(m, pts)
    assert np.all(y[:, :6] == 0) and np.all(invd[:6] == 0)
    assert np.all(invd[6:] > 0)


@pytest.mark.parametrize("f", [1.0, 1.7, 3.0])
def test_sharpen_two_kernel_logistic_closed_form(om, f):
    """Sharpening by f (L' = f L) turns the two-kernel gate into a logistic in
    f^2 (q2 - q1) / 2 with q from the unedited kernels; with q_max' = f^2 q_max
    every pixel included before stays included."""
    m = om.Model(32, 16, 1, np.array([[0.35, 0.5], [0.6, 0.45]]),
                 np.array([[0.2, 0.05, 0.18], [0.15, -0.04, 0.22]]), np.array([[0.1], [0.9]]))
    s = om.sharpen(m, f)
    y, _ = om.render(s)
    m1, m2 = float(np.float32(0.1)), float(np.float32(0.9))
    n = 0
    for j in range(m.H):
        for i in range(m.W):
            if om.included(m, 0, i, j) and om.included(m, 1, i, j):
                n += 1
                q1, q2 = q64(m, 0, i, j), q64(m, 1, i, j)
                ref = m2 + (m1 - m2) * scipy.special.expit(0.5 * f * f * (q2 - q1))
                # the edited L is rounded to float: relative error ~1e-7 in q
                assert y[0, j, i] == pytest.approx(ref, abs=1e-5 * max(1.0, f * f * abs(q2 - q1)))
    assert n > 50


def test_sharpen_keeps_the_support_and_flat_regions(om):
    """With q_max' = f^2 q_max the included (pixel, kernel) pairs are those of
    the fitted model (up to float rounding at the boundary), so equal
    constant experts still give a constant image wherever the model covered
    it (Sec. II-B: flat regions are preserved)."""
    rng = np.random.default_rng(73)
    m = rand_model(om, rng, W=36, H=28, C=3, K=16, linear=False, sig=(1.5, 4.0))
    s = om.sharpen(m, 2.5)
    same = total = 0
    for k in range(m.K):
        for j in range(m.H):
            for i in range(m.W):
                a, b = om.included(m, k, i, j), om.included(s, k, i, j)
                total += a or b
                same += a == b and a
    assert total > 500 and same >= total - 2
    v = np.array([0.3, 0.6, 0.9], np.float32)
    s.ea[:] = v
    y, invd = om.render(s)
    cov = invd > 0
    for ch in range(3):
        np.testing.assert_allclose(y[ch][cov], v[ch], rtol=1e-13)


def test_sharpen_large_factor_tends_to_hard_assignment(om):
    """As f grows the softmax gates tend to the indicator of the kernel with
    the smallest q (Mahalanobis-nearest): for every covered pixel
    |y - m_min| <= sum_{k != min} exp(-f^2 (q_k - q_min) / 2) |m_k - m_min|
    (the gate of k is at most e_k / e_min), which f = 4 makes tiny at most
    pixels.  (f^2 q_max = 144 keeps every included e_k inside the FP32 normal
    range, the limit the library enforces.)"""
    rng = np.random.default_rng(74)
    m = rand_model(om, rng, W=30, H=24, C=1, K=10, linear=False, sig=(3.0, 6.0))
    f = 4.0
    y, _ = om.render(om.sharpen(m, f))
    n_hard = 0
    for j in range(m.H):
        for i in range(m.W):
            ks = [k for k in range(m.K) if om.included(m, k, i, j)]
            if len(ks) < 2:
                continue
            q = sorted((q64(m, k, i, j), k) for k in ks)
            mmin = float(m.ea[q[0][1], 0])
            bound = sum(math.exp(-0.5 * f * f * (qk - q[0][0])) * abs(float(m.ea[k, 0]) - mmin)
                        for qk, k in q[1:])
            assert abs(y[0, j, i] - mmin) <= bound * (1 + 1e-6) + 1e-6
            n_hard += bound < 1e-3
    assert n_hard > 100


# ---------------------------------------------------------------- gate weights and the RBF mode

def test_gate_weights_two_kernel_logistic(om):
    """Eq. 4 with weights: two constant experts give
    y = m2 + (m1 - m2) expit((q2 - q1)/2 + logpi1 - logpi2)."""
    m = om.Model(32, 16, 1, np.array([[0.35, 0.5], [0.6, 0.45]]),
                 np.array([[0.2, 0.05, 0.18], [0.15, -0.04, 0.22]]), np.array([[0.1], [0.9]]),
                 logpi=np.array([0.8, -0.35]))
    y, _ = om.render(m)
    l1, l2 = float(np.float32(0.8)), float(np.float32(-0.35))
    m1, m2 = float(np.float32(0.1)), float(np.float32(0.9))
    n = 0
    for j in range(m.H):
        for i in range(m.W):
            if om.included(m, 0, i, j) and om.included(m, 1, i, j):
                n += 1
                q1, q2 = q64(m, 0, i, j), q64(m, 1, i, j)
                ref = m2 + (m1 - m2) * scipy.special.expit(0.5 * (q2 - q1) + l1 - l2)
                assert y[0, j, i] == pytest.approx(ref, rel=1e-12)
    assert n > 50


def test_gate_weights_shift_invariance(om):
    """The softmax is invariant to a common factor on every pi: adding c to
    every logpi leaves y unchanged, and so the gate-weight gradients sum to
    zero at every pixel and over the image (d/dc of the loss is 0)."""
    rng = np.random.default_rng(80)
    m = rand_model(om, rng, W=24, H=20, K=12, linear=True)
    # multiples of 2^-10, so that adding 1.25 is exact in float32
    m.logpi = (rng.integers(-600, 600, m.K) / 1024.0).astype(np.float32)
    y0, _ = om.render(m)
    m2 = om.Model(m.W, m.H, m.C, m.mu, m.chol, m.ea, m.eW, tile=m.tile, logpi=m.logpi + 1.25)
    np.testing.assert_allclose(om.render(m2)[0], y0, rtol=1e-12, atol=1e-14)
    gy = rng.normal(0, 1, (m.C, m.H, m.W))
    g, sc = om.backward(m, gy=gy, with_scale=True)
    assert abs(g[4].sum()) <= 1e-12 * sc[4].sum()
    assert np.abs(g[4]).max() > 1e-3


def test_gate_weight_central_differences(om):
    rng = np.random.default_rng(81)
    for rbf in (False, True):
        m = rand_model(om, rng, W=18, H=16, K=6, sig=(2.5, 4.0))
        m.logpi = rng.normal(0, 0.5, m.K).astype(np.float32)
        m.rbf = rbf
        gy = rng.normal(0, 1, (m.C, m.H, m.W))
        g = om.backward(m, gy=gy)[4]
        for k in range(m.K):
            v0 = m.logpi[k]
            h = np.float32(1e-3)
            vals = []
            for sgn in (1, -1):
                m.logpi[k] = np.float32(v0 + sgn * h)
                vals.append(float((om.render(m)[0] * gy).sum()))
            m.logpi[k] = v0
            real_h = (float(np.float32(v0 + h)) - float(np.float32(v0 - h))) / 2
            fd = (vals[0] - vals[1]) / (2 * real_h)
            assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-7 * np.abs(g).max()), (rbf, k)


def test_rbf_single_kernel_and_superposition(om):
    """Eq. 1: with no normalisation a single kernel renders pi K(x) m(x)
    (not m(x)), and the render of a model is the sum of the renders of its
    kernels taken one at a time (superposition), unlike the softmax gates."""
    rng = np.random.default_rng(82)
    m = rand_model(om, rng, W=22, H=18, K=5, linear=True, sig=(2.0, 4.0))
    m.logpi = rng.normal(0, 0.5, m.K).astype(np.float32)
    m.rbf = True
    y, _ = om.render(m)
    parts = np.zeros_like(y)
    for k in range(m.K):
        one = om.Model(m.W, m.H, m.C, m.mu[k:k + 1], m.chol[k:k + 1], m.ea[k:k + 1],
                       m.eW[k:k + 1], tile=m.tile, logpi=m.logpi[k:k + 1], rbf=True)
        yk, _ = om.render(one)
        c, _ = kernel_px64(m, k)
        for j in range(m.H):
            for i in range(m.W):
                if om.included(m, k, i, j):
                    q = q64(m, k, i, j)
                    mexp = m.ea[k] + m.eW[k].astype(np.float64) @ (np.array([i + 0.5, j + 0.5]) - c)
                    ref = math.exp(float(m.logpi[k]) - 0.5 * q) * mexp
                    np.testing.assert_allclose(yk[:, j, i], ref, rtol=1e-12, atol=1e-15)
                else:
                    assert np.all(yk[:, j, i] == 0)
        parts += yk
    np.testing.assert_allclose(y, parts, rtol=1e-12, atol=1e-15)
    m.rbf = False
    assert np.abs(om.render(m)[0] - parts).max() > 1e-2


def test_fit_with_gate_weights_decreases_loss(om):
    t = synth.polygon_image(24, 20, 3, 3, 83)
    p = synth.init_params(t, 16, 3.0, True, 83)
    m = om.Model(24, 20, 3, p.mu, p.chol, p.ea, p.eW, tile=8, logpi=np.zeros(16, np.float32))
    loss = om.fit(m, t, 15, lr=(1e-2, 1e-3, 1e-2, 1e-2, 1e-2, 5e-2))
    assert loss[-1] < 0.9 * loss[0]
    assert np.abs(m.logpi).max() > 1e-3            # the weights moved


def test_render_term_scale_bounds_the_render(om):
    """The render's term scale (used for the parity tolerance) bounds |y| by
    the triangle inequality, equals y for non-negative constant experts, and
    exceeds |y| where a linear expert cancels its offset."""
    rng = np.random.default_rng(90)
    m = rand_model(om, rng, W=20, H=18, K=8, linear=True)
    y, _, s = om.render(m, with_scale=True)
    assert np.all(np.abs(y) <= s * (1 + 1e-12))
    c = rand_model(om, rng, W=20, H=18, K=8, linear=False)
    yc, _, sc = om.render(c, with_scale=True)
    np.testing.assert_allclose(sc, yc, rtol=1e-12, atol=0)
    one = om.Model(16, 16, 1, np.array([[0.5, 0.5]]), np.array([[0.3, 0.0, 0.3]]),
                   np.array([[0.0]]), np.array([[[0.1, 0.0]]]))
    y1, _, s1 = om.render(one, with_scale=True)
    # m(x) = 0.1 (x - 8): at x = 8.5 the value is 0.05 and the scale 0.05, at
    # x = 0.5 (m = -0.75) both 0.75: with a zero offset the scale is |m|
    np.testing.assert_allclose(s1[0, 8], np.abs(y1[0, 8]), rtol=1e-12)
    rng2 = np.random.default_rng(91)
    m2 = rand_model(om, rng2, W=20, H=18, K=1, linear=True)
    m2.ea[:] = 1.0
    m2.eW[:] = 0.0
    m2.eW[0, :, 0] = 0.2
    y2, _, s2 = om.render(m2, with_scale=True)
    cov = s2 > 0
    assert np.any(s2[cov] > np.abs(y2[cov]) * (1 + 1e-9))   # cancelling pixels


def test_binned_baseline_equals_dense(om):
    """The binned CPU baseline (per-tile lists) gives the dense oracle's MSE
    and gradients: the lists are conservative, only the FP64 summation order
    differs."""
    rng = np.random.default_rng(95)
    for linear, tile, rbf in ((True, 8, False), (False, 16, False), (True, 16, True)):
        m = rand_model(om, rng, W=37, H=29, K=14, linear=linear, tile=tile)
        m.rbf = rbf
        t = rng.uniform(0, 1, (3, 29, 37)).astype(np.float32)
        mse, g = om.fwd_bwd_binned(m, t)
        y, _ = om.render(m)
        assert mse == pytest.approx(float(np.mean((y - t) ** 2)), rel=1e-12)
        ref = om.backward(m, target=t)
        for a, b in zip(g, ref):
            if b is not None:
                np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-14 * np.abs(b).max())
