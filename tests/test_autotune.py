"""The autotuner of the batched fit: its grouping of images by kernel count
(host logic, CPU) and, on the GPU, that it returns the fastest entry of its
own table and that every tile size it chooses between fits the same model
(the truncated SMoE does not depend on the tile grid, Sec. IV-C; only the
lists and the FP32 summation order do)."""
import numpy as np
import pytest

from paper_2510_05814_gb300.autotune import groups_by_kernels


def test_groups_without_a_limit_is_one_group():
    assert groups_by_kernels([5, 7, 9], None) == [[0, 1, 2]]
    assert groups_by_kernels([5, 7, 9], 0) == [[0, 1, 2]]


def test_groups_of_no_images():
    assert groups_by_kernels([], None) == []
    assert groups_by_kernels([], 100) == []


def test_oversized_image_gets_its_own_group():
    assert groups_by_kernels([500], 100) == [[0]]
    assert groups_by_kernels([10, 500, 10], 100) == [[0], [1], [2]]
    assert groups_by_kernels([500, 10, 20], 100) == [[0], [1, 2]]


def test_exact_fit_boundaries():
    # a group that reaches the limit exactly stays one group
    assert groups_by_kernels([40, 60, 100], 100) == [[0, 1], [2]]
    # one kernel over the limit starts a new group
    assert groups_by_kernels([40, 61, 39], 100) == [[0], [1, 2]]
    assert groups_by_kernels([1] * 5, 1) == [[0], [1], [2], [3], [4]]


def test_groups_are_consecutive_and_cover_every_image():
    rng = np.random.default_rng(7)
    for _ in range(50):
        Ks = rng.integers(1, 200, rng.integers(1, 30)).tolist()
        lim = int(rng.integers(1, 400))
        gs = groups_by_kernels(Ks, lim)
        assert [i for g in gs for i in g] == list(range(len(Ks)))
        for g in gs:
            assert len(g) == 1 or sum(Ks[i] for i in g) <= lim


@pytest.mark.gpu
def test_tune_picks_its_fastest_candidate_and_tiles_fit_the_same_model():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05814_gb300 import api, autotune, build, synth
    from paper_2510_05814_gb300.fit import FitBatch
    build.build()
    sizes = [(96, 64), (130, 70), (64, 100)]
    ts, ps = [], []
    for i, (W, H) in enumerate(sizes):
        t = synth.polygon_image(W, H, 3, 6, 800 + i, texture_amp=0.1)
        ts.append(torch.tensor(t, device="cuda"))
        ps.append(api.SMoEParams.from_numpy(synth.init_params(t, (W * H) // 16, 4.0, True, 800 + i)))
    lr = synth.PAPER_LR
    tr = autotune.tune(ts, ps, lr, tiles=(8, 16, 32), persistent=(False, True),
                       max_kernels=(None, 900), warmup=1, iters=3)
    assert len(tr.table) == 12
    best = min(tr.table, key=lambda r: r[3])
    assert (tr.tile, tr.persistent, tr.max_kernels, tr.ms_per_iter) == tuple(best)
    assert all(r[3] > 0 for r in tr.table)
    # the candidates fit the same model: equal losses over a few iterations
    losses = []
    for T in (8, 16, 32):
        fb = FitBatch(ts, [p.clone() for p in ps], 6, lr=lr, tile=T).run(6)
        losses.append(fb.losses())
    for other in losses[1:]:
        np.testing.assert_allclose(other, losses[0], rtol=1e-5)
