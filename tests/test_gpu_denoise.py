"""GPU parity of multi-model fusion (Sec. V-C, Eq. 11) through the C ABI
(smoe_fit_render_mean) against the oracle, and of the MM-RSMoE denoising
pipeline (H fits of one noisy image as one batch, then the fused render).

Bar: the fused image within 1e-5 x the mean over the models of the render
bar's per-pixel scale max(|y_h|, sum_k w_k |m_k|) -- the render bar averaged,
since y_m is the mean of H renders each held to it; one model alone gives
smoe_render's image bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as om  # noqa: E402
from paper_2510_05814_gb300 import api, denoise, synth  # noqa: E402
from paper_2510_05814_gb300.fit import FitBatch  # noqa: E402

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


def fused_gpu(ps, W, H, C, tile, pair_cap=None):
    t = torch.zeros(C, H, W, device="cuda")
    fb = FitBatch([t] * len(ps), [api.SMoEParams.from_numpy(p) for p in ps], 1, tile=tile,
                  pair_cap=pair_cap)
    return fb.render_mean(), fb


# (seed, W, H, C, linear, tile, n_models)
CASES = [
    (1, 75, 53, 3, True, 16, 5),
    (2, 64, 40, 3, True, 8, 3),
    (3, 70, 66, 1, False, 32, 4),
    (4, 48, 48, 3, False, 16, 2),
    (5, 33, 17, 1, True, 8, 7),
]


@pytest.mark.parametrize("case", CASES, ids=[f"case{c[0]}" for c in CASES])
def test_render_mean_matches_oracle(case):
    seed, W, H, C, linear, tile, n = case
    ps = [rand_params(100 * seed + h, C, 20 + 7 * h, linear) for h in range(n)]
    y, _ = fused_gpu(ps, W, H, C, tile)
    ref, scale = om.render_mean([om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=tile)
                                 for p in ps], with_scale=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= RTOL_Y * scale), float((err / np.maximum(scale, 1e-30)).max())


def test_render_mean_with_degenerate_and_empty_models():
    """A model of degenerate kernels (NaN centre, infinite or zero
    precision, off-image) and a model with no kernel at all (renders 0)
    fused with an ordinary one."""
    W, H, C = 41, 39, 3
    mu = np.array([[0.5, 0.5], [np.nan, 0.5], [1.4, 0.5], [0.3, 0.7], [0.5, 0.5]], np.float32)
    chol = np.array([[0.0, 0.3, 0.3], [0.3, 0.0, 0.3], [0.2, 0.0, 0.2], [5.0, 0.0, 5.0],
                     [np.inf, 0.0, 0.3]], np.float32)
    rng = np.random.default_rng(7)
    deg = synth.Params(mu, chol, rng.uniform(0, 1, (5, C)).astype(np.float32),
                       rng.normal(0, 0.05, (5, C, 2)).astype(np.float32))
    empty = synth.Params(np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32),
                         np.zeros((0, C), np.float32), np.zeros((0, C, 2), np.float32))
    ps = [rand_params(71, C, 30, True), deg, empty]
    y, _ = fused_gpu(ps, W, H, C, 16)
    ref, scale = om.render_mean([om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=16)
                                 for p in ps], with_scale=True)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= RTOL_Y * scale)


def test_render_mean_of_one_model_is_its_render():
    p = rand_params(8, 3, 60, True)
    y1, _ = fused_gpu([p], 77, 45, 3, 16)
    y, _, _ = api.render(api.SMoEParams.from_numpy(p), 77, 45, tile=16)
    assert torch.equal(y1, y)


def test_render_mean_grows_the_pair_buffer():
    """A pair count above the buffer sets the capacity status; FitBatch
    grows the buffer and renders again, with the same result."""
    ps = [rand_params(900 + h, 3, 40, True) for h in range(3)]
    y_small, fb = fused_gpu(ps, 64, 48, 3, 8, pair_cap=16)
    assert fb.pair_cap > 16
    y_ref, _ = fused_gpu(ps, 64, 48, 3, 8)
    assert torch.equal(y_small, y_ref)


def test_mm_pipeline_matches_oracle():
    """Four models of one noisy image (lattices shifted by 4 px), 6 Adam
    iterations as one batch, then the fused render; the oracle runs the
    same pipeline in FP64.  The FP32 fits follow the FP64 ones (losses within
    1e-4 relative, as the single-image fit trajectory); the fused images
    then agree to 1e-4 on average and 2e-3 at worst (a few pixels near the
    cutoff of kernels whose parameters moved by FP32 rounding)."""
    W, H = 40, 32
    clean, noisy = synth.denoise_case(W, H, 0.01, seed=63)
    lr = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2)
    offs = denoise.shift_offsets(4, 8)
    ps = [synth.init_params(noisy, 20, 3.0, True, 63 + h, offset=o) for h, o in enumerate(offs)]
    models = [om.Model(W, H, 3, p.mu.copy(), p.chol.copy(), p.ea.copy(), p.eW.copy(), tile=8)
              for p in ps]
    ref, ref_losses = om.mm_denoise(models, noisy, 6, lr=lr)
    y, fb = denoise.mm_rsmoe(torch.tensor(noisy, device="cuda"),
                             [api.SMoEParams.from_numpy(p) for p in ps], 6, lr=lr, tile=8)
    np.testing.assert_allclose(fb.losses()[:, :6], np.array(ref_losses), rtol=1e-4)
    d = np.abs(y.cpu().numpy() - ref)
    assert d.mean() <= 1e-4 and d.max() <= 2e-3, (d.mean(), d.max())


def test_more_models_less_noise():
    """Eq. 14: fusing models that start from shifted lattices lowers the
    error to the clean image against one model, and (convexity) the fused
    squared error is below the mean of the four models' own errors."""
    W, H = 128, 96
    clean, noisy = synth.denoise_case(W, H, 0.01, seed=64)
    tn = torch.tensor(noisy, device="cuda")
    K = W * H // 32
    one = denoise.init_models(noisy, 1, K, 5.0, True, seed=64)
    y1, _ = denoise.mm_rsmoe(tn, one, 300, lr=(1e-2, 1e-4, 1e-2, 1e-2, 1e-2))
    four = denoise.init_models(noisy, 4, K, 5.0, True, seed=64)
    y4, fb = denoise.mm_rsmoe(tn, four, 300, lr=(1e-2, 1e-4, 1e-2, 1e-2, 1e-2))
    c = torch.tensor(clean, device="cuda")
    e1 = float(((y1 - c) ** 2).mean())
    e4 = float(((y4 - c) ** 2).mean())
    assert e4 < e1
    singles = [api.render(fb.params_of(h), W, H, tile=16)[0] for h in range(4)]
    assert e4 < np.mean([float(((s - c) ** 2).mean()) for s in singles])
    noisy_err = float(((tn - c) ** 2).mean())
    assert e4 < noisy_err


def test_mm_pipeline_deterministic_mode_is_reproducible():
    W, H = 64, 48
    _, noisy = synth.denoise_case(W, H, 0.005, seed=65)
    tn = torch.tensor(noisy, device="cuda")
    outs = []
    for _ in range(2):
        ms = denoise.init_models(noisy, 4, 96, 4.0, True, seed=65)
        y, _ = denoise.mm_rsmoe(tn, ms, 20, deterministic=True)
        outs.append(y)
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("scale,tile", [(1.0, 16), (1.5, 8), (2.0, 16), (3.25, 32)])
def test_standalone_render_mean_at_scale(scale, tile):
    """smoe_render_mean: separate models on a raster `scale` times finer
    (the resampled MM-RSMoE result), against the oracle's mean of the
    scale-s renders; at scale 1 it equals the fit batch's fused render."""
    W, H, C = 40, 30, 3
    ps = [rand_params(700 + h, C, 18 + 5 * h, True) for h in range(3)]
    Wo, Ho = int(round(W * scale)), int(round(H * scale))
    models = [api.SMoEParams.from_numpy(p) for p in ps]
    y = api.render_mean(models, Wo, Ho, tile=tile, scale=scale).cpu().numpy()
    ref, sc = om.render_mean([om.Model(Wo, Ho, C, p.mu, p.chol, p.ea, p.eW, tile=tile,
                                       scale=scale) for p in ps], with_scale=True)
    assert np.all(np.abs(y - ref) <= RTOL_Y * sc)
    if scale == 1.0:
        yb, _ = fused_gpu(ps, W, H, C, tile)
        assert np.array_equal(y, yb.cpu().numpy())


def test_standalone_render_mean_grows_its_pair_buffer():
    ps = [rand_params(720 + h, 3, 40, True) for h in range(2)]
    models = [api.SMoEParams.from_numpy(p) for p in ps]
    a = api.render_mean(models, 64, 48, tile=8, pair_cap=8)
    b = api.render_mean(models, 64, 48, tile=8)
    assert torch.equal(a, b)
