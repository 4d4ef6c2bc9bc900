"""GPU parity of the gate weights pi_k (Eq. 4, learned as log pi_k) and of the
RBF / Gaussian-splatting mode (Eq. 1: y = sum_k pi_k K_k m_k, D = 1), through
the C ABI, against the oracle: render, backward (all groups and dL/dlogpi),
the fused fit, Adam on the weight group, the autograd wrapper, the fused
multi-model render and point resampling.  Bars as in test_gpu_parity.
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


def rand_case(seed, W, H, C, K, linear, pi=True, sig=(1.5, 6.0), span=(-0.05, 1.05)):
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
    lp = rng.normal(0, 0.8, K) if pi else None
    f = lambda a: None if a is None else a.astype(np.float32)
    return synth.Params(f(mu), f(chol), f(ea), f(eW), f(lp))


def om_model(p, W, H, C, tile, rbf, scale=1.0):
    return om.Model(W, H, C, p.mu, p.chol, p.ea, p.eW, tile=tile, scale=scale, logpi=p.logpi,
                    rbf=rbf)


def check_y(y, ref, absm):
    err = np.abs(y - ref)
    assert np.all(err <= RTOL_Y * np.maximum(np.abs(ref), absm)), float(err.max())


def check_grad(g, ref, terms, what):
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    den = np.maximum(den, 1e-2 * np.asarray(terms, np.float64))
    rel = np.abs(np.asarray(g, np.float64) - ref) / np.where(den > 0, den, 1.0)
    assert rel.max() <= RTOL_G, f"{what}: {rel.max():.3g}"


# (seed, W, H, C, K, linear, tile, scale, pi, rbf)
CASES = [
    (1, 64, 48, 3, 40, True, 16, 1.0, True, False),
    (2, 53, 47, 1, 30, False, 8, 1.0, True, False),
    (3, 70, 66, 3, 45, True, 32, 1.0, True, False),
    (4, 60, 50, 3, 35, True, 16, 1.5, True, False),
    (5, 64, 48, 3, 40, True, 16, 1.0, False, True),
    (6, 53, 47, 1, 30, False, 8, 1.0, True, True),
    (7, 70, 66, 3, 45, True, 32, 1.0, True, True),
    (8, 60, 50, 1, 35, True, 16, 2.0, True, True),
]
IDS = [f"c{c[0]}{'_pi' if c[8] else ''}{'_rbf' if c[9] else ''}" for c in CASES]


def gpu(case):
    seed, W, H, C, K, linear, tile, scale, pi, rbf = case
    p = rand_case(seed, int(round(W / scale)), int(round(H / scale)), C, K, linear, pi)
    params = api.SMoEParams.from_numpy(p)
    desc = api.RasterDesc(W, H, C, tile, linear, 9.0, scale, rbf)
    r = api.Rasterizer(desc, K).bin(params)
    return p, params, r


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_render_parity(case):
    seed, W, H, C, K, linear, tile, scale, pi, rbf = case
    p, _, r = gpu(case)
    y, inv = r.render()
    ref, ref_inv, absm = om.render(om_model(p, W, H, C, tile, rbf, scale), with_scale=True)
    check_y(y.cpu().numpy(), ref, absm)
    gi = inv.cpu().numpy()
    assert np.all(np.abs(gi - ref_inv) <= RTOL_Y * ref_inv)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_backward_parity(case):
    seed, W, H, C, K, linear, tile, scale, pi, rbf = case
    p, params, r = gpu(case)
    y, inv = r.render()
    gy = np.random.default_rng(seed + 300).normal(0, 1, (C, H, W))
    grad = params.zeros_like()
    if grad.logpi is None:           # dL/dlogpi at pi = 1 is still defined
        grad.logpi = torch.zeros(K, device="cuda")
    g = r.backward(params, y, inv, gy=torch.tensor(gy, dtype=torch.float32, device="cuda"),
                   grad=grad)
    m = om_model(p, W, H, C, tile, rbf, scale)
    if m.logpi is None:
        m.logpi = np.zeros(K, np.float32)
    ref, terms = om.backward(m, gy=gy.astype(np.float32).astype(np.float64), with_scale=True)
    got = dict(zip(["mu", "chol", "ea", "eW", "logpi"], g.slots()))
    for name, b, t in zip(["mu", "chol", "ea", "eW", "logpi"], ref, terms):
        if b is not None:
            check_grad(got[name].cpu().numpy(), b, t, name)


def test_unit_weights_equal_no_weights_bit_for_bit():
    """logpi = 0 stores 0 in the record: the gate argument fma(q, c, 0) is
    the plain product, so the render is the pi = 1 render exactly."""
    p = rand_case(9, 77, 45, 3, 60, True, pi=False)
    a, _, _ = api.render(api.SMoEParams.from_numpy(p), 77, 45, tile=16)
    p0 = synth.Params(p.mu, p.chol, p.ea, p.eW, np.zeros(60, np.float32))
    b, _, _ = api.render(api.SMoEParams.from_numpy(p0), 77, 45, tile=16)
    assert torch.equal(a, b)


@pytest.mark.parametrize("rbf", [False, True])
def test_fused_mse_backward_parity(rbf):
    p = rand_case(10, 72, 60, 3, 50, True)
    params = api.SMoEParams.from_numpy(p)
    r = api.Rasterizer(api.RasterDesc(72, 60, 3, 16, True, 9.0, 1.0, rbf), 50).bin(params)
    y, inv = r.render()
    t = synth.polygon_image(72, 60, 3, 5, 10)
    g = r.backward(params, y, inv, target=torch.tensor(t, device="cuda"))
    ref, terms = om.backward(om_model(p, 72, 60, 3, 16, rbf), target=t, with_scale=True)
    for name, a, b, s_ in zip(["mu", "chol", "ea", "eW", "logpi"], g.slots(), ref, terms):
        check_grad(a.cpu().numpy(), b, s_, name)


def test_adam_step_updates_the_weight_group():
    K = 300
    rng = np.random.default_rng(11)
    mk = lambda: api.SMoEParams.from_numpy(synth.Params(
        *(rng.normal(0, 1, s).astype(np.float32) for s in [(K, 2), (K, 3), (K, 3), (K, 3, 2), (K,)])))
    p, g = mk(), mk()
    m = mk()
    v = api.SMoEParams(*(t.abs() for t in mk().tensors()))
    lp0 = p.logpi.cpu().numpy().astype(np.float64)
    gl = g.logpi.cpu().numpy().astype(np.float64)
    ml = m.logpi.cpu().numpy().astype(np.float64)
    vl = v.logpi.cpu().numpy().astype(np.float64)
    api.smoe_adam_step(p, g, m, v, (1e-2, 1e-3, 1e-3, 1e-3, 5e-2), step=3)
    om.adam(lp0, gl, ml, vl, 5e-2, step=3)
    np.testing.assert_allclose(p.logpi.cpu().numpy(), lp0, rtol=2e-6, atol=1e-7)
    assert torch.count_nonzero(g.logpi).item() == 0


@pytest.mark.parametrize("rbf", [False, True])
def test_fit_trajectory_with_weights_matches_oracle(rbf):
    """smoe_fit with learned gate weights (and in the RBF mode) follows the
    oracle's FP64 fit: per-iteration MSE within 1e-4 relative."""
    t = synth.polygon_image(40, 32, 3, 4, 12)
    p = synth.init_params(t, 20, 3.0, True, 12)
    p = synth.Params(p.mu, p.chol, p.ea * (0.3 if rbf else 1.0), p.eW, np.zeros(20, np.float32))
    lr = (1e-2, 1e-3, 1e-2, 1e-2, 1e-2, 3e-2)
    m = om.Model(40, 32, 3, p.mu.copy(), p.chol.copy(), p.ea.copy(), p.eW.copy(), tile=8,
                 logpi=p.logpi.copy(), rbf=rbf)
    ref = om.fit(m, t, 8, lr=lr)
    fb = FitBatch([torch.tensor(t, device="cuda")], [api.SMoEParams.from_numpy(p)], 8, lr=lr,
                  tile=8, rbf=rbf)
    fb.run(8)
    np.testing.assert_allclose(fb.losses()[0], ref, rtol=1e-4)
    np.testing.assert_allclose(fb.params_of(0).logpi.cpu().numpy(), m.logpi, rtol=0, atol=2e-4)


def test_autograd_with_weights_vs_oracle():
    W, H, C, K = 48, 40, 3, 30
    p = rand_case(13, W, H, C, K, True)
    leaves = [torch.tensor(a, device="cuda", requires_grad=True)
              for a in (p.mu, p.chol, p.ea, p.eW, p.logpi)]
    desc = api.RasterDesc(W, H, C, 16, True)
    gy = np.random.default_rng(14).normal(0, 1, (C, H, W)).astype(np.float32)
    y = api.smoe_render_fn(*leaves[:4], desc, leaves[4])
    loss = (y * torch.tensor(gy, device="cuda")).sum()
    grads = torch.autograd.grad(loss, leaves)
    ref, terms = om.backward(om_model(p, W, H, C, 16, False), gy=gy.astype(np.float64),
                             with_scale=True)
    for name, a, b, s_ in zip(["mu", "chol", "ea", "eW", "logpi"], grads, ref, terms):
        check_grad(a.cpu().numpy(), b, s_, name)


def test_rbf_fused_mean_and_points():
    """The fused multi-model render and point resampling in the RBF mode."""
    W, H, C = 60, 44, 3
    ps = [rand_case(20 + h, W, H, C, 25, True) for h in range(3)]
    t = torch.zeros(C, H, W, device="cuda")
    fb = FitBatch([t] * 3, [api.SMoEParams.from_numpy(p) for p in ps], 1, tile=16, rbf=True)
    y = fb.render_mean().cpu().numpy()
    ref, scale = om.render_mean([om_model(p, W, H, C, 16, True) for p in ps], with_scale=True)
    assert np.all(np.abs(y - ref) <= RTOL_Y * scale)
    pts = np.random.default_rng(23).uniform([0, 0], [W, H], (2000, 2)).astype(np.float32)
    yp, _, _ = api.render_points(api.SMoEParams.from_numpy(ps[0]), W, H,
                                 torch.tensor(pts, device="cuda"), tile=16, rbf=True)
    ref, _, absm = om.render_points(om_model(ps[0], W, H, C, 16, True), pts, with_scale=True)
    check_y(yp.cpu().numpy(), ref, absm)
