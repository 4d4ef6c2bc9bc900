"""GPU parity of the culling shortcuts against the oracle, through the C ABI.

- Binning with warp-aggregated walks: kernels in grid order (a warp's 32
  consecutive kernels are neighbours, so most warps count and scatter per
  union tile) mixed with wide kernels that send their warp to the per-lane
  walk; the lists stay bit-exact (Sec. IV-C, Eq. 5).
- Row masks evaluated over the tile's columns: thin, tilted, mirrored
  (a < 0), nearly degenerate and very narrow kernels whose ellipses graze
  tile edges; the render (Eqs. 2-4) and the backward stay within the bars
  against the dense oracle, which evaluates every pixel against every kernel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as om  # noqa: E402
from paper_2510_05814_gb300 import api, synth  # noqa: E402
from paper_2510_05814_gb300.fit import FitBatch  # noqa: E402

RTOL_Y = 1e-5
RTOL_G = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_05814_gb300 import build
    build.build()
    om.build()


def model(p, W, H, C, tile):
    return om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=tile)


def lists_gpu(p, W, H, C, tile):
    params = api.SMoEParams.from_numpy(p)
    desc = api.RasterDesc(W, H, C, tile, p.eW is not None, 9.0, 1.0)
    r = api.Rasterizer(desc, params.K).bin(params)
    return params, r


def aggregated_warps(ref_off, ref_pk, K, W, H, tile):
    """From the oracle's lists: each kernel's tile rectangle, then the
    number of warps (32 consecutive kernels) whose union box is compact
    enough for the aggregated walk (at most 128 tiles and fewer than the
    rectangles' total), and the number of warps that are not."""
    tx = (W + tile - 1) // tile
    x0 = np.full(K, 1 << 30); x1 = np.full(K, -1); y0 = np.full(K, 1 << 30); y1 = np.full(K, -1)
    for t in range(len(ref_off) - 1):
        ks = ref_pk[ref_off[t]:ref_off[t + 1]]
        cx, cy = t % tx, t // tx
        x0[ks] = np.minimum(x0[ks], cx); x1[ks] = np.maximum(x1[ks], cx)
        y0[ks] = np.minimum(y0[ks], cy); y1[ks] = np.maximum(y1[ks], cy)
    agg = other = 0
    for w0 in range(0, K, 32):
        s = slice(w0, min(w0 + 32, K))
        has = x1[s] >= 0
        if not has.any():
            continue
        area = ((x1[s] - x0[s] + 1) * (y1[s] - y0[s] + 1))[has].sum()
        nu = (x1[s][has].max() - x0[s][has].min() + 1) * (y1[s][has].max() - y0[s][has].min() + 1)
        if nu <= 128 and nu < area:
            agg += 1
        else:
            other += 1
    return agg, other


@pytest.mark.parametrize("tile,W,H,K", [(16, 256, 192, 3072), (8, 200, 120, 1500),
                                        (32, 640, 480, 4800), (16, 333, 97, 2020)])
def test_grid_ordered_lists_bitexact(tile, W, H, K):
    """Kernels on a jittered grid (grid order, anisotropic), every 97th made
    12x wider: most warps take the aggregated walk, the warps holding a wide
    kernel (and those straddling grid rows) the per-lane one."""
    t = synth.polygon_image(W, H, 3, 8, K)
    p = synth.init_params(t, K, 3.0, True, K, aniso=(1.0, 3.0), slope_std=1e-2)
    chol = p.chol.copy()
    chol[::97] /= 12.0
    p = synth.Params(p.mu, chol, p.ea, p.eW)
    params, r = lists_gpu(p, W, H, 3, tile)
    off, pk = r.lists()
    m = model(p, W, H, 3, tile)
    ref_off, ref_pk = om.bin_tiles(m)
    np.testing.assert_array_equal(off.astype(np.int64), ref_off)
    np.testing.assert_array_equal(pk, ref_pk)
    agg, other = aggregated_warps(ref_off, ref_pk, K, W, H, tile)
    assert agg > 0 and other > 0, (agg, other)
    y, _ = r.render()
    ref, _, absm = om.render(m, with_scale=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= RTOL_Y * np.maximum(np.abs(ref), absm))


def adversarial(seed, W, H, tile, K=160):
    """Thin and tilted ellipses (aspect up to 60), a < 0 (mirrored factor),
    very narrow (a up to 40 / px) and nearly flat (a down to 1e-4) kernels,
    centres on pixel centres, pixel corners and tile corners."""
    rng = np.random.default_rng(seed)
    mu = np.empty((K, 2)); chol = np.empty((K, 3))
    for k in range(K):
        kind = k % 5
        if kind == 0:                   # centre on a pixel centre
            cx, cy = rng.integers(0, W) + 0.5, rng.integers(0, H) + 0.5
        elif kind == 1:                 # pixel corner
            cx, cy = float(rng.integers(0, W + 1)), float(rng.integers(0, H + 1))
        elif kind == 2:                 # tile corner
            cx = float(tile * rng.integers(0, W // tile + 1))
            cy = float(tile * rng.integers(0, H // tile + 1))
        else:
            cx, cy = rng.uniform(-0.1 * W, 1.1 * W), rng.uniform(-0.1 * H, 1.1 * H)
        mu[k] = (cx / W, cy / H)
        s_long = rng.uniform(2.0, 30.0)
        s_short = s_long / rng.uniform(1.0, 60.0)
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        L = np.linalg.cholesky(np.linalg.inv(R @ np.diag([s_long ** 2, s_short ** 2]) @ R.T))
        a, b, c = L[0, 0], L[1, 0], L[1, 1]
        if k % 7 == 3:
            a = -a                      # mirrored factor: same |z0| family
        if k % 11 == 4:
            a = rng.choice([1e-4, 40.0])
        chol[k] = (a, b, c)
    ea = rng.uniform(0, 1, (K, 3))
    eW = rng.normal(0, 0.05, (K, 3, 2))
    f = lambda x: x.astype(np.float32)
    return synth.Params(f(mu), f(chol), f(ea), f(eW))


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_row_masks_exact_on_adversarial_kernels(tile, seed):
    W, H = 5 * tile + 3, 4 * tile + 5
    p = adversarial(100 * tile + seed, W, H, tile)
    params, r = lists_gpu(p, W, H, 3, tile)
    m = model(p, W, H, 3, tile)
    off, pk = r.lists()
    ref_off, ref_pk = om.bin_tiles(m)
    np.testing.assert_array_equal(off.astype(np.int64), ref_off)
    np.testing.assert_array_equal(pk, ref_pk)
    y, invd = r.render()
    ref, ref_inv, absm = om.render(m, with_scale=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= RTOL_Y * np.maximum(np.abs(ref), absm)), float(err.max())
    # the empty-pixel rule and D itself: a dropped kernel changes 1/D
    gi = invd.cpu().numpy()
    assert np.array_equal(gi == 0, ref_inv == 0)
    assert np.all(np.abs(gi - ref_inv) <= RTOL_Y * ref_inv)
    gy = np.random.default_rng(seed).normal(0, 1, (3, H, W)).astype(np.float32)
    g = r.backward(params, y, invd, gy=torch.tensor(gy, device="cuda"))
    ref_g, terms = om.backward(m, gy=gy.astype(np.float64), with_scale=True)
    for name, a_, b_, t_ in zip(["mu", "chol", "ea", "eW"], g.numpy(), ref_g, terms):
        b_ = np.asarray(b_, np.float64)
        den = np.maximum(np.abs(b_), 1e-3 * np.abs(b_).max())
        den = np.maximum(den, 1e-2 * np.asarray(t_, np.float64))
        rel = np.abs(np.asarray(a_, np.float64) - b_) / np.where(den > 0, den, 1.0)
        assert rel.max() <= RTOL_G, f"{name}: {rel.max():.3g}"


def test_batch_warps_straddling_images_with_offimage_kernels():
    """A warp holding the last kernels of one image, moved off its raster
    (empty rectangles), and the first kernels of the next image (another
    width): the batched fit bins and steps every image exactly as a fit of
    that image alone (deterministic accumulation: bit for bit)."""
    from paper_2510_05814_gb300.fit import FitBatch
    shapes = [(70, 50, 40), (120, 40, 70), (50, 90, 45)]
    ts, ps = [], []
    for i, (W, H, K) in enumerate(shapes):
        t = synth.polygon_image(W, H, 3, 5, 80 + i)
        p = synth.init_params(t, K, 4.0, True, 80 + i)
        mu = p.mu.copy()
        mu[-9:] = (3.0, -2.0)                 # off the raster: empty rectangles
        ts.append(torch.tensor(t, device="cuda"))
        ps.append(synth.Params(mu, p.chol, p.ea, p.eW))
    lr = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2)
    fb = FitBatch(ts, [api.SMoEParams.from_numpy(p) for p in ps], 3, lr=lr, tile=8,
                  deterministic=True)
    fb.run(3)
    for b in range(len(shapes)):
        one = FitBatch([ts[b]], [api.SMoEParams.from_numpy(ps[b])], 3, lr=lr, tile=8,
                       deterministic=True)
        one.run(3)
        np.testing.assert_allclose(fb.losses()[b, :3], one.losses()[0, :3], rtol=1e-12)
        for x, y in zip(fb.params_of(b).tensors(), one.params_of(0).tensors()):
            assert torch.equal(x, y)


def huge_case(W, H, seed, C=3):
    """Normal kernels plus kernels whose box holds more than 1024 tiles at
    T = 16: degenerate ones (a zero Cholesky entry: every tile), stripes (a
    near-zero entry stretching the kernel across the raster) and a very wide
    round one."""
    rng = np.random.default_rng(seed)
    K = 160
    mu = rng.uniform(0.05, 0.95, (K, 2))
    s = rng.uniform(2.0, 6.0, K)
    chol = np.stack([1 / s, rng.normal(0, 0.05, K), 1 / s], 1)
    chol[0] = (0.0, 0.3, 0.3)                    # det = 0: every tile
    chol[1] = (0.3, 0.0, 0.0)                    # det = 0 (c = 0)
    chol[2] = (1e-4, 0.0, 0.4)                   # a horizontal stripe
    chol[3] = (0.5, 0.0, 2e-4)                   # a vertical stripe
    chol[4] = (1e-3, 0.02, 1e-3)                 # very wide
    ea = rng.uniform(0, 1, (K, C))
    eW = rng.normal(0, 0.02, (K, C, 2))
    return synth.Params(mu.astype(np.float32), chol.astype(np.float32), ea.astype(np.float32),
                        eW.astype(np.float32))


def test_huge_rectangles_are_binned_bit_exact():
    """Rectangles of more than 1024 tiles are counted and appended per tile
    instead of walked: the lists stay the oracle's, bit for bit, and the
    render and backward stay within the bars."""
    W, H = 1024, 768                                       # 64 x 48 = 3072 tiles
    p = huge_case(W, H, 71)
    m = om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=16)
    rects = [om.rect(m, k)[1] for k in range(5)]
    assert min(rects) > 1024
    params = api.SMoEParams.from_numpy(p)
    r = api.Rasterizer(api.RasterDesc(W, H, 3, 16, True), params.K).bin(params)
    off, pk = r.lists()
    ref_off, ref_pk = om.bin_tiles(m)
    np.testing.assert_array_equal(off.astype(np.int64), ref_off)
    np.testing.assert_array_equal(pk, ref_pk)
    y, inv = r.render()
    rng = np.random.default_rng(72)
    px = rng.choice(W * H, 400, replace=False)
    ref, _, absm = om.render(m, pixels=px, with_scale=True)
    got = y.reshape(3, -1)[:, torch.tensor(px, device="cuda")].cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.maximum(np.abs(ref), absm))


def test_huge_rectangles_in_a_batch_stay_in_their_image():
    """A deterministic batch of two images, each with huge rectangles: every
    image's fit equals its fit alone, bit for bit (a queued kernel is added
    to its own image's tiles only)."""
    ts, ps = [], []
    for i, (W, H) in enumerate([(640, 512), (512, 640)]):
        ts.append(torch.tensor(synth.polygon_image(W, H, 3, 5, 80 + i), device="cuda"))
        ps.append(api.SMoEParams.from_numpy(huge_case(W, H, 90 + i)))
    lr = (1e-4, 1e-4, 1e-3, 1e-2, 1e-2)
    both = FitBatch(ts, [p.clone() for p in ps], 3, lr=lr, deterministic=True).run(3)
    for b in range(2):
        one = FitBatch([ts[b]], [ps[b].clone()], 3, lr=lr, deterministic=True).run(3)
        for x, y in zip(both.params_of(b).tensors(), one.params_of(0).tensors()):
            assert torch.equal(x, y)
        np.testing.assert_allclose(both.losses()[b], one.losses()[0], rtol=1e-12)


@pytest.mark.parametrize("n_huge", [40, 150])
def test_appended_huge_ids_in_long_lists_are_bit_exact(n_huge):
    """Lists of 129 to 512 ids that also carry queued huge kernels: the
    scatter's blocks are merged, the appended ids sorted and the two runs
    merged by rank (up to 128 appended ids; 150 take the full sort).  The
    lists are the oracle's, bit for bit."""
    W = H = 768                                            # 48 x 48 tiles
    rng = np.random.default_rng(500 + n_huge)
    K = 30000
    mu = rng.uniform(0.0, 1.0, (K, 2))
    s = rng.uniform(6.0, 12.0, K)
    chol = np.stack([1 / s, rng.normal(0, 0.02, K), 1 / s], 1)
    # the first n_huge kernels cover every tile: a zero Cholesky entry, or a
    # stripe across the raster, at scattered positions in the kernel order
    idx = rng.choice(K, n_huge, replace=False)
    for i, k in enumerate(idx):
        chol[k] = (0.0, 0.3, 0.3) if i % 2 else (1e-5, 0.0, 1e-5)
    p = synth.Params(mu.astype(np.float32), chol.astype(np.float32),
                     rng.uniform(0, 1, (K, 3)).astype(np.float32),
                     rng.normal(0, 0.02, (K, 3, 2)).astype(np.float32))
    m = om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=16)
    ref_off, ref_pk = om.bin_tiles(m)
    lens = np.diff(ref_off)
    assert (lens > 128).mean() > 0.5 and lens.max() <= 512 + n_huge, (lens.min(), lens.max())
    assert all(om.rect(m, int(k))[1] > 1024 for k in idx)
    params = api.SMoEParams.from_numpy(p)
    r = api.Rasterizer(api.RasterDesc(W, H, 3, 16, True), params.K).bin(params)
    off, pk = r.lists()
    np.testing.assert_array_equal(off.astype(np.int64), ref_off)
    np.testing.assert_array_equal(pk, ref_pk)
