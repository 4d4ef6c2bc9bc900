"""Host-side logic of the package that needs no GPU: the window offsets of
multi-model denoising and the synchronous argument checks of its entry point."""
import ctypes

import numpy as np
import pytest

from paper_2510_05814_gb300.denoise import shift_offsets


@pytest.mark.parametrize("d,count", [(2, 64), (4, 16), (8, 4), (16, 1)])
def test_shift_offsets_square_counts(d, count):
    """Sec. V-C: a 16-pixel window shifted by d in both directions gives
    (16/d)^2 windows per pixel: d = 2, 4, 8, 16 -> 64, 16, 4, 1."""
    offs = shift_offsets(count, 16)
    assert len(offs) == count == len(set(offs))
    xs = sorted({o[0] for o in offs})
    ys = sorted({o[1] for o in offs})
    assert xs == list(range(0, 16, d)) and ys == list(range(0, 16, d))


@pytest.mark.parametrize("count,nx,ny", [(8, 4, 2), (32, 8, 4), (2, 2, 1)])
def test_shift_offsets_non_square_counts(count, nx, ny):
    offs = shift_offsets(count, 16)
    assert len(offs) == count == len(set(offs))
    assert len({o[0] for o in offs}) == nx and len({o[1] for o in offs}) == ny
    assert all(0 <= ox < 16 and 0 <= oy < 16 for ox, oy in offs)


def test_shift_offsets_rejects_uneven_counts():
    with pytest.raises(ValueError):
        shift_offsets(0)
    with pytest.raises(ValueError):
        shift_offsets(3, 16)


def test_render_mean_refuses_mixed_sizes_before_any_launch():
    """smoe_fit_render_mean checks that the batch's images share one size on
    the host and returns SMOE_ERR_ARG without launching anything."""
    from paper_2510_05814_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    P = _lib.Params
    imgs = (_lib.FitImage * 2)()
    for b, (W, H) in enumerate([(32, 32), (40, 32)]):
        z = P(4, 256, 512, 768, 1024)
        imgs[b] = _lib.FitImage(W, H, 2048, z, z, z, 10, 1e-2, 1e-5, 1e-3, 1e-3, 1e-3)
    batch = _lib.FitBatch(2, 3, 16, 1, 9.0, 0.9, 0.999, 1e-8, 4096, 0, 0, 0, 0)
    n = ctypes.c_size_t(0)
    assert lib.smoe_fit_workspace_size(ctypes.byref(batch), imgs, 1000, ctypes.byref(n)) == 0
    st = lib.smoe_fit_render_mean(ctypes.byref(batch), imgs, 1000, ctypes.c_void_p(1 << 20),
                                  n.value, ctypes.c_void_p(8192), ctypes.c_void_p(16384), None)
    assert st == _lib.SMOE_ERR_ARG
    assert np.isscalar(n.value) and n.value > 0
