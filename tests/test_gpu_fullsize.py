"""Parity at the full size of the 2048x2048 workload (K = 262144 anisotropic
kernels, linear experts, 16x16 tiles), through the C ABI and the autograd
wrapper, on sampled outputs the oracle computes one by one.

The oracle is dense (every pixel against every kernel).  To keep it fast,
each check gives it the sub-model of the kernels listed in the tiles that
hold the sampled pixels: a kernel outside those lists has no included pixel
there (the lists are conservative, pinned exhaustively on small cases), so
the dense result on those pixels is unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as om  # noqa: E402
from paper_2510_05814_gb300 import api, synth  # noqa: E402

T = 16


@pytest.fixture(scope="module")
def wl():
    from paper_2510_05814_gb300 import build
    build.build()
    om.build()
    return synth.rgb_2048()


def sub_model(p, W, H, tiles, scale=1.0, extra=()):
    """Oracle model of the kernels listed in `tiles` (plus `extra` ids);
    returns (model, ids) with ids the global kernel ids in sub-model order."""
    full = om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=T, scale=scale)
    off, pk = om.bin_tiles(full, tiles)
    ids = np.unique(np.concatenate([pk, np.asarray(extra, np.int64)]).astype(np.int64))
    m = om.Model(W, H, 3, p.mu[ids], p.chol[ids], p.ea[ids], p.eW[ids], tile=T, scale=scale)
    return m, ids


def tiles_of_pixels(px, W):
    tx = (W + T - 1) // T
    return np.unique((px // W) // T * tx + (px % W) // T)


def test_fullsize_lists_and_render_sampled(wl):
    C, H, W = wl.target.shape
    p = api.SMoEParams.from_numpy(wl.params)
    y, inv, r = api.render(p, W, H, tile=T)
    off, pk = r.lists()
    rng = np.random.default_rng(100)
    tiles = np.concatenate([[0, (W // T) - 1, len(off) - 2], rng.choice(len(off) - 1, 61, replace=False)])
    full = om.Model(W, H, C, wl.params.mu, wl.params.chol, wl.params.ea, wl.params.eW, tile=T)
    ref_off, ref_pk = om.bin_tiles(full, tiles)
    for s, t in enumerate(tiles):
        np.testing.assert_array_equal(pk[off[t]:off[t + 1]], ref_pk[ref_off[s]:ref_off[s + 1]])
    px = np.concatenate([[0, W - 1, (H - 1) * W, H * W - 1], rng.choice(H * W, 508, replace=False)])
    m, _ = sub_model(wl.params, W, H, tiles_of_pixels(px, W))
    ref, ref_inv, absm = om.render(m, pixels=px, with_scale=True)
    got = y.reshape(C, -1)[:, torch.tensor(px, device="cuda")].cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.maximum(np.abs(ref), absm))
    gi = inv.reshape(-1)[torch.tensor(px, device="cuda")].cpu().numpy()
    assert np.all(np.abs(gi - ref_inv) <= 1e-5 * ref_inv)


def test_fullsize_super_resolution_sampled(wl):
    """Native super-resolution: the model rendered at 2x (4096x4096)."""
    C, H, W = wl.target.shape
    p = api.SMoEParams.from_numpy(wl.params)
    y, inv, r = api.render(p, 2 * W, 2 * H, tile=T, scale=2.0)
    rng = np.random.default_rng(101)
    px = rng.choice(4 * H * W, 256, replace=False)
    m, _ = sub_model(wl.params, 2 * W, 2 * H, tiles_of_pixels(px, 2 * W), scale=2.0)
    ref, _, absm = om.render(m, pixels=px, with_scale=True)
    got = y.reshape(C, -1)[:, torch.tensor(px, device="cuda")].cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.maximum(np.abs(ref), absm))


def test_autograd_64_parameters_vs_oracle_and_central_differences(wl):
    """torch.autograd through SMoERender at full size: 64 random parameters
    against the oracle's analytic gradient (rel err <= 1e-4, denominator
    floored at 1e-2 x the sum of term magnitudes), and 16 of them against
    FP64 central differences of the oracle's loss."""
    C, H, W = wl.target.shape
    rng = np.random.default_rng(102)
    P = wl.params
    leaves = [torch.tensor(a, device="cuda", requires_grad=True) for a in (P.mu, P.chol, P.ea, P.eW)]
    desc = api.RasterDesc(W, H, C, T, True)
    gy = rng.normal(0, 1, (C, H, W)).astype(np.float32)
    y = api.smoe_render_fn(*leaves, desc)
    loss = (y * torch.tensor(gy, device="cuda")).sum()
    grads = torch.autograd.grad(loss, leaves)
    shapes = [(2,), (3,), (C,), (C, 2)]
    picks = []
    while len(picks) < 64:
        k = int(rng.integers(0, P.K))
        gi = int(rng.integers(0, 4))
        e = tuple(int(rng.integers(0, s)) for s in shapes[gi])
        picks.append((k, gi, e))
    gy64 = gy.astype(np.float64)
    full = om.Model(W, H, C, P.mu, P.chol, P.ea, P.eW, tile=T)
    checked_fd = 0
    for n, (k, gi, e) in enumerate(picks):
        (x0, y0, x1, y1), cnt = om.rect(full, k)
        assert cnt > 0
        tx = (W + T - 1) // T
        tiles = np.array([ty * tx + t for ty in range(y0, y1 + 1) for t in range(x0, x1 + 1)])
        m, ids = sub_model(P, W, H, tiles, extra=[k])
        pos = int(np.searchsorted(ids, k))
        # the pixels of those tiles (every pixel where kernel k can be included)
        px = np.array([(ty * T + j) * W + t * T + i for ty in range(y0, y1 + 1)
                       for t in range(x0, x1 + 1) for j in range(T) for i in range(T)
                       if ty * T + j < H and t * T + i < W])
        (rg, rt) = om.backward(m, gy=gy64, kernels=[pos], with_scale=True)
        ref = rg[gi].reshape(-1)[np.ravel_multi_index(e, shapes[gi])]
        terms = rt[gi].reshape(-1)[np.ravel_multi_index(e, shapes[gi])]
        got = float(grads[gi][k][e].item())
        den = max(abs(ref), 1e-2 * terms)
        assert abs(got - ref) <= 1e-4 * den, (k, gi, e, got, ref, terms)
        if checked_fd < 16:
            arr = [m.mu, m.chol, m.ea, m.eW][gi]
            v0 = arr[(pos,) + e]
            h = np.float32(1e-3 * max(1.0, abs(float(v0))) if gi != 0 else 1e-4)
            vals = []
            base = None
            for sgn in (1, -1):
                arr[(pos,) + e] = np.float32(v0 + sgn * h)
                incl = np.array([om.included(m, pos, int(q % W), int(q // W)) for q in px])
                if base is None:
                    base = incl
                elif not np.array_equal(incl, base):
                    vals = None
                    break
                yy, _ = om.render(m, pixels=px)
                vals.append(float((yy * gy64.reshape(C, -1)[:, px]).sum()))
            dh = (float(np.float32(v0 + h)) - float(np.float32(v0 - h))) / 2
            arr[(pos,) + e] = v0
            if vals is not None:
                fd = (vals[0] - vals[1]) / (2 * dh)
                assert abs(got - fd) <= 1e-3 * max(abs(fd), 1e-2 * terms) + 1e-9, (k, gi, e, got, fd)
                checked_fd += 1
    assert checked_fd >= 12


def test_fullsize_fit_gradients_sampled(wl):
    """The gradients of the fused fit path (fused forward / MSE / backward
    tile launch and the Adam launch's finalize, read out by
    smoe_fit_gradients) at the full 2048^2 workload in the bench's launch
    configuration (T = 16, one CTA per tile, float atomics): every parameter
    of 48 random kernels against the oracle's analytic MSE gradient,
    |g - g_ref| <= 1e-4 max(|g_ref|, 1e-2 x the sum of term magnitudes)."""
    from paper_2510_05814_gb300.fit import FitBatch
    C, H, W = wl.target.shape
    P = wl.params
    fb = FitBatch([torch.tensor(wl.target, device="cuda")], [api.SMoEParams.from_numpy(P)], 2,
                  lr=synth.PAPER_LR, tile=T)
    g = fb.gradients()[0]
    assert fb.status_code() == 0
    got = [x.cpu().numpy() for x in g.tensors()]
    full = om.Model(W, H, C, P.mu, P.chol, P.ea, P.eW, tile=T)
    tx = (W + T - 1) // T
    rng = np.random.default_rng(103)
    checked = 0
    for k in rng.choice(P.K, 48, replace=False):
        (x0, y0, x1, y1), cnt = om.rect(full, int(k))
        if cnt == 0:
            continue
        tiles = np.array([ty * tx + t for ty in range(y0, y1 + 1) for t in range(x0, x1 + 1)])
        m, ids = sub_model(P, W, H, tiles, extra=[k])
        pos = int(np.searchsorted(ids, k))
        rg, rt = om.backward(m, target=wl.target, kernels=[pos], with_scale=True)
        for gi, name in enumerate(["mu", "chol", "ea", "eW"]):
            ref, terms = rg[gi][0].ravel(), rt[gi][0].ravel()
            a = got[gi][k].ravel()
            den = np.maximum(np.abs(ref), 1e-2 * terms)
            assert np.all(np.abs(a - ref) <= 1e-4 * den), (int(k), name, a, ref, terms)
        checked += 1
    assert checked >= 40


def test_ragged_batch_fullsize_losses():
    """Config 4 at full size: the 64 ragged images (128x96 .. 1920x1080,
    K = pixels/16, 35 M pixels) as one fit batch.  After one fused iteration
    the per-image MSE of the initial models, computed inside the batched tile
    kernel, matches the oracle's dense FP64 render for the six smallest images
    (whose tiles sit between the big images' in the ragged table) and is
    finite for all."""
    from paper_2510_05814_gb300.fit import FitBatch
    sizes = synth.ragged_sizes(64, 4)
    targets, params, nps = [], [], []
    for i, (W, H) in enumerate(sizes):
        t = synth.polygon_image(W, H, 3, 40, 400 + i, texture_amp=0.1)
        p = synth.init_params(t, (W * H) // 16, 5.0, True, 400 + i)
        targets.append(t)
        nps.append(p)
        params.append(api.SMoEParams.from_numpy(p))
    fb = FitBatch([torch.tensor(t, device="cuda") for t in targets], params, 1,
                  lr=synth.PAPER_LR, tile=T)
    fb.run(1)
    loss = fb.losses()[:, 0]
    assert np.all(np.isfinite(loss)) and np.all(loss > 0)
    small = sorted(range(64), key=lambda b: sizes[b][0] * sizes[b][1])[:6]
    for b in small:
        W, H = sizes[b]
        p = nps[b]
        m = om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=T)
        y, _ = om.render(m)
        ref = float(np.mean((y - targets[b].astype(np.float64)) ** 2))
        assert loss[b] == pytest.approx(ref, rel=1e-5), (b, loss[b], ref)
