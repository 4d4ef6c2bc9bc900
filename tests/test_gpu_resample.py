"""GPU parity of native sharpening (kernel editing) and of resampling at
arbitrary points (Sec. II-B, Sec. VII-C) against the oracle, through the C ABI.

Bar: as the render -- |y - y_ref| <= 1e-5 max(|y_ref|, sum_k w_k |m_k|) per
point and channel, 1/D within 1e-5 relative; the edited Cholesky factors
bit-exact (one float product each).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as om  # noqa: E402
from paper_2510_05814_gb300 import _lib, api, synth  # noqa: E402

RTOL_Y = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_05814_gb300 import build
    build.build()
    om.build()


def rand_params(seed, C, K, linear, sig=(1.5, 6.0), span=(-0.05, 1.05)):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(*span, (K, 2))
    chol = np.zeros((K, 3))
    for k in range(K):
        s = rng.uniform(*sig, 2)
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        L = np.linalg.cholesky(np.linalg.inv(R @ np.diag(s ** 2) @ R.T))
        chol[k] = (L[0, 0], L[1, 0], L[1, 1])
    ea = rng.uniform(0, 1, (K, C))
    eW = rng.normal(0, 0.05, (K, C, 2)) if linear else None
    return synth.Params(mu.astype(np.float32), chol.astype(np.float32), ea.astype(np.float32),
                        None if eW is None else eW.astype(np.float32))


def sample_points(rng, W, H, T, n):
    """Uniform points, pixel centres, exact tile and raster edges, points
    just inside / outside the raster and non-finite coordinates."""
    u = rng.uniform([0, 0], [W, H], (n, 2))
    centres = np.stack([rng.integers(0, W, 64) + 0.5, rng.integers(0, H, 64) + 0.5], 1)
    edges = np.array([[t * T, y] for t in range(0, W // T + 1) for y in (0.0, H / 3)] +
                     [[x, t * T] for t in range(0, H // T + 1) for x in (0.25, W / 2)])
    special = np.array([[0.0, 0.0], [W - 1e-3, H - 1e-3], [-1e-3, 1.0], [W, 1.0], [1.0, H],
                        [np.nan, 1.0], [1.0, np.inf], [-np.inf, -5.0]])
    pts = np.concatenate([u, centres, edges, special]).astype(np.float32)
    return pts[rng.permutation(len(pts))]


def test_sharpen_is_one_float_product():
    p = rand_params(1, 3, 333, True)
    chol = torch.tensor(p.chol, device="cuda")
    params = api.SMoEParams(torch.tensor(p.mu, device="cuda"), chol,
                            torch.tensor(p.ea, device="cuda"), torch.tensor(p.eW, device="cuda"))
    for f in (1.5, 2.0, 3.3, 0.7):
        s, q = api.sharpen(params, f)
        np.testing.assert_array_equal(s.chol.cpu().numpy(), p.chol * np.float32(f))
        assert q == float(np.float32(9.0) * (np.float32(f) * np.float32(f)))
        assert s.mu is params.mu and s.ea is params.ea
    with pytest.raises(ValueError):
        api.sharpen(params, 5.0)


# (seed, W, H, C, K, linear, tile)
CASES = [
    (1, 64, 48, 3, 40, True, 16),
    (2, 53, 47, 1, 30, False, 8),
    (3, 70, 66, 3, 45, True, 32),
    (4, 37, 29, 3, 25, False, 16),
]


@pytest.mark.parametrize("case", CASES, ids=[f"case{c[0]}" for c in CASES])
def test_render_points_matches_oracle(case):
    seed, W, H, C, K, linear, T = case
    p = rand_params(seed, C, K, linear)
    rng = np.random.default_rng(seed + 50)
    pts = sample_points(rng, W, H, T, 3000)
    y, inv, _ = api.render_points(api.SMoEParams.from_numpy(p), W, H,
                                  torch.tensor(pts, device="cuda"), tile=T)
    m = om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=T)
    ref, ref_inv, absm = om.render_points(m, pts, with_scale=True)
    got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= RTOL_Y * np.maximum(np.abs(ref), absm))
    gi = inv.cpu().numpy()
    assert np.all(np.abs(gi - ref_inv) <= RTOL_Y * ref_inv)
    assert np.all(gi[ref_inv == 0] == 0)


def test_render_points_at_pixel_centres_match_render():
    p = api.SMoEParams.from_numpy(rand_params(5, 3, 50, True))
    W, H = 61, 43
    y, inv, _ = api.render(p, W, H, tile=16)
    xs = np.stack(np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5), -1).reshape(-1, 2)
    yp, ip, _ = api.render_points(p, W, H, torch.tensor(xs, dtype=torch.float32, device="cuda"),
                                  tile=16)
    # same truncated model and FP32 coordinates; only the summation order differs
    torch.testing.assert_close(yp.reshape(3, H, W), y, rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(ip.reshape(H, W), inv, rtol=1e-5, atol=0)


@pytest.mark.parametrize("f", [1.6, 2.5])
def test_sharpened_render_and_points_match_oracle(f):
    W, H, C = 72, 56, 3
    p = rand_params(6, C, 60, True, sig=(2.0, 7.0))
    sp, q = api.sharpen(api.SMoEParams.from_numpy(p), f)
    y, inv, r = api.render(api.SMoEParams.from_numpy(p), W, H, tile=16, sharpen_factor=f)
    m = om.sharpen(om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=16), f)
    assert m.qmax == q
    ref, ref_inv, absm = om.render(m, with_scale=True)
    got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= RTOL_Y * np.maximum(np.abs(ref), absm))
    rng = np.random.default_rng(7)
    pts = sample_points(rng, W, H, 16, 2000)
    yp, _, _ = api.render_points(api.SMoEParams.from_numpy(p), W, H,
                                 torch.tensor(pts, device="cuda"), tile=16, sharpen_factor=f)
    ref, _, absm = om.render_points(m, pts, with_scale=True)
    assert np.all(np.abs(yp.cpu().numpy() - ref) <= RTOL_Y * np.maximum(np.abs(ref), absm))


def test_render_points_edge_cases():
    p = api.SMoEParams.from_numpy(rand_params(8, 3, 20, True))
    r = api.Rasterizer(api.RasterDesc(40, 30, 3, 16, True), p.K).bin(p)
    y, inv = r.render_points(torch.zeros(0, 2, device="cuda"))
    assert y.shape == (3, 0) and inv.shape == (0,)
    out = torch.tensor([[-1.0, 2.0], [41.0, 3.0], [float("nan"), 1.0]], device="cuda")
    y, inv = r.render_points(out)
    assert torch.all(y == 0) and torch.all(inv == 0)
    # the point buffer must be 8-byte aligned (pairs are loaded as float2)
    buf = torch.zeros(9, device="cuda")
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    d = r.desc.c()
    assert lib.smoe_points_workspace_size(ctypes.byref(d), 4, ctypes.byref(n)) == 0
    pws = torch.empty(n.value + 256, dtype=torch.uint8, device="cuda")
    off = (-pws.data_ptr()) % 256
    st = lib.smoe_render_points(ctypes.byref(d), p.K, r.ws.data_ptr(), r.ws.numel(),
                                r.tile_off.data_ptr(), r.pair_k.data_ptr(), 4,
                                buf.data_ptr() + 4, pws.data_ptr() + off, n.value,
                                torch.empty(12, device="cuda").data_ptr(), None,
                                r.status.data_ptr(), None)
    assert st == _lib.SMOE_ERR_ARG


def test_cutoff_above_fp32_range_is_refused():
    d = api.RasterDesc(32, 32, 3, 16, True, 200.0, 1.0).c()
    n = ctypes.c_size_t(0)
    assert _lib.load().smoe_workspace_size(ctypes.byref(d), 10, 100, ctypes.byref(n)) == \
        _lib.SMOE_ERR_ARG


def test_ten_times_magnification_of_the_2048_model_sampled():
    """Sec. VII-C's 10x magnification on the 2048x2048 workload: points on a
    10x finer regular raster over a 96x96 crop, plus random points over the
    whole image, against the oracle's sub-model of the listed kernels."""
    wl = synth.rgb_2048()
    C, H, W = wl.target.shape
    P = wl.params
    x0, y0 = 1000.0, 700.0
    g = (np.arange(960) + 0.5) / 10.0
    grid = np.stack(np.meshgrid(x0 + g, y0 + g), -1).reshape(-1, 2)
    rng = np.random.default_rng(9)
    pts = np.concatenate([grid, rng.uniform([0, 0], [W, H], (20000, 2))]).astype(np.float32)
    params = api.SMoEParams.from_numpy(P)
    y, inv, r = api.render_points(params, W, H, torch.tensor(pts, device="cuda"), tile=16)
    got = y.cpu().numpy()
    sel = rng.choice(len(pts), 3000, replace=False)
    tx = (W + 15) // 16
    tiles = np.unique((pts[sel, 1].astype(np.int64) // 16) * tx + pts[sel, 0].astype(np.int64) // 16)
    off, pk = r.lists()
    ids = np.unique(np.concatenate([pk[off[t]:off[t + 1]] for t in tiles]))
    m = om.Model(W, H, C, P.mu[ids], P.chol[ids], P.ea[ids], P.eW[ids], tile=16)
    ref, _, absm = om.render_points(m, pts[sel], with_scale=True)
    assert np.all(np.abs(got[:, sel] - ref) <= RTOL_Y * np.maximum(np.abs(ref), absm))


@pytest.mark.parametrize("C,linear", [(3, True), (1, False)])
def test_warp_row_culling_is_bit_identical_to_the_point_walk(C, linear):
    """The same sparse points rendered alone (their warps span several tiles
    and walk the lists point by point) and among a dense jittered raster
    (their warps share a tile and cull the list against their rows first):
    the values are equal bit for bit, and match the oracle."""
    W, H, T = 96, 80, 16
    p = rand_params(77 + C, C, 400, linear, sig=(1.0, 9.0))
    params = api.SMoEParams.from_numpy(p)
    rng = np.random.default_rng(78)
    sparse = np.stack([rng.uniform(0, W, 300), rng.uniform(0, H, 300)], 1).astype(np.float32)
    g = (np.arange(W * 4) + 0.5) / 4.0
    gy = (np.arange(H * 4) + 0.5) / 4.0
    dense = np.stack(np.meshgrid(g, gy), -1).reshape(-1, 2)
    dense = (dense + rng.uniform(-0.1, 0.1, dense.shape)).astype(np.float32)
    alone, _, _ = api.render_points(params, W, H, torch.tensor(sparse, device="cuda"), tile=T)
    mixed, _, _ = api.render_points(params, W, H,
                                    torch.tensor(np.concatenate([dense, sparse]), device="cuda"),
                                    tile=T)
    assert torch.equal(mixed[:, dense.shape[0]:], alone)
    m = om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=T)
    ref, _, absm = om.render_points(m, sparse, with_scale=True)
    assert np.all(np.abs(alone.cpu().numpy() - ref) <= RTOL_Y * np.maximum(np.abs(ref), absm))
