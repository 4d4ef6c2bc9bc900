"""Element-wise parity of the gradients of the fused fit path.

The fit's iteration is the binning, the fused forward / MSE / backward tile
launch and the Adam launch, which turns every kernel's raw sums into
gradients (the chain rule of Eqs. 2-4) and steps Adam on them.  Adam's first
step is +-lr whatever the gradient's magnitude, so the fit's loss curve cannot
see a lost factor in those gradients.  smoe_fit_gradients reads out the
gradients that the Adam launch would apply (the same device code) and this
file holds them to the oracle's analytic gradient of the MSE, element by
element, at the gradient bar of the parity tests (Sec. III-D: gradient
descent through the rasteriser; Sec. VI-B: the MSE fit).
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

from test_gpu_parity import check_grad, rand_case  # noqa: E402

LR = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2, 1e-2)
NAMES = ["mu", "chol", "ea", "eW", "logpi"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_05814_gb300 import build
    build.build()
    om.build()


def with_pi(p, seed):
    rng = np.random.default_rng(seed)
    return synth.Params(p.mu, p.chol, p.ea, p.eW,
                        rng.normal(0.0, 0.5, p.K).astype(np.float32))


def oracle_grads(p, t, tile, rbf=False):
    C, H, W = t.shape
    m = om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=tile,
                 logpi=getattr(p, "logpi", None), rbf=rbf)
    return om.backward(m, target=t, with_scale=True)


def compare(got, ref, terms, what):
    for name, a, b, s in zip(NAMES, got.numpy(), ref, terms):
        if b is not None:
            check_grad(a.reshape(b.shape), b, f"{what} {name}", s)


# (seed, W, H, C, K, linear, tile, pi, rbf)
CASES = [
    (1, 53, 47, 3, 60, True, 8, False, False),
    (2, 64, 48, 1, 50, False, 8, False, False),
    (3, 77, 45, 3, 50, True, 16, False, False),
    (4, 70, 66, 1, 45, True, 16, False, False),
    (5, 96, 64, 3, 40, False, 32, False, False),
    (6, 70, 66, 1, 45, True, 32, False, False),
    (7, 60, 52, 3, 55, True, 16, True, False),     # learned gate weights
    (8, 60, 52, 3, 55, True, 16, False, True),     # RBF sum (Eq. 1)
    (9, 48, 40, 1, 35, False, 8, True, True),      # both, grey, T = 8
]


@pytest.mark.parametrize("case", CASES, ids=[f"g{c[0]}" for c in CASES])
def test_fit_gradients_match_oracle(case):
    seed, W, H, C, K, linear, tile, pi, rbf = case
    p = rand_case(seed, W, H, C, K, linear)
    if pi:
        p = with_pi(p, seed)
    t = synth.polygon_image(W, H, C, 5, 300 + seed, texture_amp=0.1)
    params = api.SMoEParams.from_numpy(p)
    before = [x.clone() for x in params.tensors()]
    fb = FitBatch([torch.tensor(t, device="cuda")], [params], 3, lr=LR, tile=tile, rbf=rbf)
    g = fb.gradients()[0]
    assert fb.status_code() == 0
    ref, terms = oracle_grads(p, t, tile, rbf)
    compare(g, ref, terms, f"case {seed}")
    # the read-out leaves the parameters and the schedule as they were
    for a, b in zip(params.tensors(), before):
        assert torch.equal(a, b)
    assert int(fb.step.item()) == 0
    # ... and Adam's first step then moves every parameter with a clear
    # gradient against that gradient's sign (torch Adam at step 1 moves by
    # -lr g / (|g| + eps))
    fb.run(1)
    for name, a, b, gg in zip(NAMES, params.tensors(), before, g.tensors()):
        d = (a - b).cpu().numpy().ravel()
        gv = gg.cpu().numpy().ravel()
        clear = np.abs(gv) > 1e-3 * max(np.abs(gv).max(), 1e-30)
        assert np.all(np.sign(d[clear]) == -np.sign(gv[clear])), name


def test_fit_gradients_twice_are_equal_and_sums_are_cleared():
    """Two read-outs in a row give the same gradients (FP32 atomics: to
    rounding), so the first left the workspace's sums at zero."""
    p = rand_case(11, 64, 64, 3, 80, True)
    t = synth.polygon_image(64, 64, 3, 5, 311)
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 2, lr=LR)
    g1 = fb.gradients()[0]
    g2 = fb.gradients()[0]
    # equal up to the order of the float atomics (sums left over from the
    # first read-out would double the second)
    for name, a, b in zip(NAMES, g1.numpy(), g2.numpy()):
        check_grad(b, a.astype(np.float64), name)


@pytest.mark.parametrize("mode", ["grid", "persistent", "deterministic"])
def test_fit_gradients_ragged_batch(mode):
    """A ragged batch of three images (tiles of different widths in one
    table): every image's gradients match the oracle's for that image alone,
    for the grid, persistent and deterministic launches."""
    sizes = [(40, 30), (64, 48), (23, 37)]
    ts, ps = [], []
    for i, (W, H) in enumerate(sizes):
        t = synth.polygon_image(W, H, 3, 4, 70 + i, texture_amp=0.1)
        ts.append(t)
        ps.append(synth.init_params(t, (W * H) // 16, 3.0, True, 70 + i, aniso=(1.0, 2.5),
                                    slope_std=0.02))
    fb = FitBatch([torch.tensor(t, device="cuda") for t in ts],
                  [api.SMoEParams.from_numpy(p) for p in ps], 4, lr=LR, tile=8,
                  persistent=mode == "persistent", deterministic=mode == "deterministic")
    gs = fb.gradients()
    assert fb.status_code() == 0
    for b, (t, p) in enumerate(zip(ts, ps)):
        ref, terms = oracle_grads(p, t, 8)
        compare(gs[b], ref, terms, f"image {b}")


def test_fit_gradients_deterministic_are_bit_reproducible():
    t = synth.polygon_image(80, 60, 3, 5, 320, texture_amp=0.1)
    p = synth.init_params(t, 300, 3.0, True, 320, aniso=(1.0, 2.0), slope_std=0.02)
    mk = lambda: FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 2,
                          lr=LR, deterministic=True)
    g1, g2 = mk().gradients()[0], mk().gradients()[0]
    for a, b in zip(g1.tensors(), g2.tensors()):
        assert torch.equal(a, b)


def test_fit_gradients_finished_image_is_zero():
    """An image whose run has ended takes no step: its gradient read-out is 0
    while a running image in the same batch gets its own."""
    ts = [synth.polygon_image(48, 40, 3, 4, 330 + i) for i in range(2)]
    ps = [synth.init_params(t, 120, 3.0, True, 330 + i) for i, t in enumerate(ts)]
    fb = FitBatch([torch.tensor(t, device="cuda") for t in ts],
                  [api.SMoEParams.from_numpy(p) for p in ps], [1, 3], lr=LR)
    fb.run(1)                                      # image 0 is done after one iteration
    g = fb.gradients()
    assert all(torch.count_nonzero(x).item() == 0 for x in g[0].tensors())
    assert any(torch.count_nonzero(x).item() > 0 for x in g[1].tensors())


def test_fit_gradients_argument_errors():
    from paper_2510_05814_gb300 import _lib
    import ctypes
    t = synth.polygon_image(32, 32, 3, 3, 340)
    p = synth.init_params(t, 64, 3.0, True, 340)
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 2, lr=LR)
    lib = _lib.load()
    bad = api.SMoEParams.zeros(63, 3, True)           # wrong K
    st = lib.smoe_fit_gradients(ctypes.byref(fb._batch), fb._imgs, fb.pair_cap,
                                api._ptr(fb.ws), fb.ws.numel(), ctypes.byref(bad.c()),
                                api._ptr(fb.status), api._stream(None))
    assert st == _lib.SMOE_ERR_ARG
    bad = api.SMoEParams.zeros(64, 3, False)          # slopes missing for linear experts
    st = lib.smoe_fit_gradients(ctypes.byref(fb._batch), fb._imgs, fb.pair_cap,
                                api._ptr(fb.ws), fb.ws.numel(), ctypes.byref(bad.c()),
                                api._ptr(fb.status), api._stream(None))
    assert st == _lib.SMOE_ERR_ARG


@pytest.mark.parametrize("C,linear,tile", [(3, True, 8), (1, False, 16)])
def test_fit_gradients_degenerate_kernels(C, linear, tile):
    """Degenerate kernels (a NaN centre, an infinite or a zero Cholesky
    entry, centres off the raster, a kernel far narrower than a pixel): the
    fused path's read-out matches the oracle's gradient, and a kernel listed
    in no tile gets exactly 0."""
    from test_gpu_parity import degenerate_case
    W, H = 41, 39
    p = degenerate_case(W, H, C, linear)
    t = synth.polygon_image(W, H, C, 4, 350 + C, texture_amp=0.1)
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 2, lr=LR,
                  tile=tile)
    g = fb.gradients()[0]
    assert fb.status_code() == 0
    ref, terms = oracle_grads(p, t, tile)
    compare(g, ref, terms, f"degenerate C={C}")
    nan_k = 9                                  # mu = (nan, 0.5): listed in no tile
    assert all(float(x[nan_k].abs().sum()) == 0.0 for x in g.tensors())


@pytest.mark.parametrize("mode", ["grid", "persistent", "deterministic"])
def test_fit_gradients_long_lists(mode):
    """Tile lists of 505 to 810 kernels: the fused kernel stages a list in
    chunks and walks a chunk in sub-chunks of 256, so its forward and its
    backward cross both boundaries.  Thin kernels keep the count included at
    a pixel near 350 while their square boxes list them almost everywhere;
    the gradients match the oracle's at the gradient bar."""
    W, H = 64, 48
    p = rand_case(43, W, H, 3, 900, True, sig=(1.0, 12.0), span=(0.05, 0.95))
    t = synth.polygon_image(W, H, 3, 5, 343, texture_amp=0.1)
    off, _ = om.bin_tiles(om.Model(W, H, 3, p.mu, p.chol, p.ea, p.eW, tile=16))
    lens = np.diff(off)
    assert lens.min() > 256 and lens.max() > 512, (lens.min(), lens.max())
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 2, lr=LR,
                  tile=16, persistent=mode == "persistent", deterministic=mode == "deterministic")
    g = fb.gradients()[0]
    assert fb.status_code() == 0
    ref, terms = oracle_grads(p, t, 16)
    compare(g, ref, terms, f"long lists ({mode})")
