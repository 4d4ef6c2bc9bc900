"""GPU checks of the spatial reordering of a fit batch's kernels
(smoe_fit_reorder, smoe_scatter_params): it is a permutation that keeps
kernels in their image and moves each kernel's parameters and Adam moments
together, into tile-major order of the centres; params_of returns the
caller's order; a fit that reorders follows the same trajectory as one that
does not (only the FP32 summation order differs) and the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as om  # noqa: E402
from paper_2510_05814_gb300 import api, synth  # noqa: E402
from paper_2510_05814_gb300.fit import FitBatch  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_05814_gb300 import build
    build.build()
    om.build()


def scrambled(W, H, K, seed, pi=False):
    """A kernel set in random order (as after a long fit), some centres off
    the raster."""
    t = synth.polygon_image(W, H, 3, 6, seed)
    p = synth.init_params(t, K, 3.0, True, seed, aniso=(1.0, 2.0), slope_std=1e-2)
    perm = np.random.default_rng(seed).permutation(K)
    mu = p.mu[perm].copy()
    mu[::37] = mu[::37] * 1.3 - 0.15
    lp = np.random.default_rng(seed + 1).normal(0, 0.3, K).astype(np.float32) if pi else None
    return t, synth.Params(mu, p.chol[perm], p.ea[perm], p.eW[perm], lp)


def centre_tiles(p, W, H, T):
    mx = np.float32(p.mu[:, 0]) * np.float32(W)
    my = np.float32(p.mu[:, 1]) * np.float32(H)
    tx = np.clip(np.floor(mx / np.float32(T)), 0, (W + T - 1) // T - 1)
    ty = np.clip(np.floor(my / np.float32(T)), 0, (H + T - 1) // T - 1)
    return (ty * ((W + T - 1) // T) + tx).astype(np.int64)


@pytest.mark.parametrize("pi", [False, True])
def test_reorder_is_a_tile_major_permutation(pi):
    sizes = [(96, 64, 384), (70, 50, 200)]
    ts, ps = [], []
    for i, (W, H, K) in enumerate(sizes):
        t, p = scrambled(W, H, K, 10 + i, pi)
        ts.append(torch.tensor(t, device="cuda"))
        ps.append(p)
    params = [api.SMoEParams.from_numpy(p) for p in ps]
    lr = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2, 1e-2)
    fb = FitBatch(ts, params, 10, lr=lr, tile=16, reorder_every=1000)
    fb.run(3)                                   # non-zero moments
    before = [[x.clone() for x in fb.params_of(b).tensors()] for b in range(2)]
    mom = [[x.clone() for x in (fb.m[b].tensors() + fb.v[b].tensors())] for b in range(2)]
    fb.reorder()
    torch.cuda.synchronize()
    assert fb.status_code() == 0
    order = fb.order.cpu().numpy()
    for b, (W, H, K) in enumerate(sizes):
        # the caller's view is unchanged, bit for bit
        for x, y in zip(fb.params_of(b).tensors(), before[b]):
            assert torch.equal(x, y)
        # slots: a permutation within the image, tile-major, ascending index per tile
        o = order[fb.k_off[b]:fb.k_off[b] + K] - fb.k_off[b]
        assert np.array_equal(np.sort(o), np.arange(K))
        slot = fb.params[b].numpy()
        tiles = centre_tiles(synth.Params(slot[0], slot[1], slot[2], slot[3]), W, H, 16)
        assert np.all(np.diff(tiles) >= 0)
        same = np.diff(tiles) == 0
        assert np.all(np.diff(o)[same] > 0)
        # the moments moved with their kernels
        for x, y in zip(fb.m[b].tensors() + fb.v[b].tensors(), mom[b]):
            np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy()[o])


def test_fit_with_reordering_follows_the_plain_fit_and_the_oracle():
    W, H, K = 80, 64, 320
    t, p = scrambled(W, H, K, 21)
    lr = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2)
    tt = torch.tensor(t, device="cuda")
    plain = FitBatch([tt], [api.SMoEParams.from_numpy(p)], 12, lr=lr, tile=16)
    plain.run(12)
    ro = FitBatch([tt], [api.SMoEParams.from_numpy(p)], 12, lr=lr, tile=16, reorder_every=4)
    ro.run(12, graph_iters=2)
    np.testing.assert_allclose(ro.losses()[0], plain.losses()[0], rtol=1e-5)
    for x, y in zip(ro.params_of(0).numpy(), plain.params_of(0).numpy()):
        np.testing.assert_allclose(x, y, rtol=1e-4, atol=1e-6)
    m = om.Model(W, H, 3, p.mu.copy(), p.chol.copy(), p.ea.copy(), p.eW.copy(), tile=16)
    ref = om.fit(m, t, 12, lr=lr)
    np.testing.assert_allclose(ro.losses()[0], ref, rtol=1e-4)


def test_reorder_then_render_matches_oracle():
    """After reordering, the batch's own (slot-ordered) parameters render
    within the bar of the oracle's render of the same kernel set."""
    W, H, K = 75, 53, 150
    t, p = scrambled(W, H, K, 31)
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 1,
                  tile=8, reorder_every=1)
    fb.reorder()
    y, _, _ = api.render(fb.params[0], W, H, tile=8)
    ref, _, absm = om.render(om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=8),
                             with_scale=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * np.maximum(np.abs(ref), absm))


def test_run_with_overflow_keeps_the_resort_schedule():
    """FitBatch.run checks the status only at the end here, re-sorting every
    4 iterations in between; a pair buffer that overflows (at once, or when
    the lists outgrow the initial count) stops the batch at that
    iteration's binning, grows, and resumes with the re-sort at the same
    iterations: the deterministic fit equals the one with room to spare,
    bit for bit."""
    t = synth.polygon_image(64, 48, 3, 5, 910, texture_amp=0.1)
    p = synth.init_params(t, 192, 3.0, True, 910, aniso=(1.0, 2.0), slope_std=0.02)
    tt = torch.tensor(t, device="cuda")
    lr = (4e-4, 4e-4, 1e-2, 1e-2, 1e-2)
    desc = api.RasterDesc(64, 48, 3, 8, True)
    n0 = int(api.Rasterizer(desc, p.K).bin(api.SMoEParams.from_numpy(p)).n_pairs.item())

    def fit(cap):
        fb = FitBatch([tt], [api.SMoEParams.from_numpy(p)], 12, lr=lr, tile=8, reorder_every=4,
                      deterministic=True, pair_cap=cap)
        return fb.run(12, graph_iters=2)

    ref = fit(4 * n0)
    for cap in (64, n0):
        got = fit(cap)
        assert int(got.step.item()) == 12
        # the reported MSE adds per-tile FP64 partial sums in completion order
        np.testing.assert_allclose(got.losses(), ref.losses(), rtol=1e-12)
        for a, b in zip(got.params_of(0).tensors(), ref.params_of(0).tensors()):
            assert torch.equal(a, b)
    assert fit(64).pair_cap > 64
