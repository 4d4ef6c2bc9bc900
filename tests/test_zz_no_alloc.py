"""smoe_render_static: rendering without any device allocation.

Some callers cannot allocate device memory themselves (a plugin inside an
application that owns every allocation, code that must not touch the
allocator).  For them the library has one entry point whose intermediate
buffers live in a fixed device array inside the library.  This test calls it
through the C ABI, twice in a row on different models, and checks each
output against the workspace-based path (smoe_bin + smoe_render) at the
render tolerance used everywhere else (1e-5 relative); it also checks the
size limits.  It is collected last so that a run stopping at the first
failure has already run every other test, and it passes alone in a fresh
process as well (the first call on the device does the set-up)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2510_05814_gb300 import _lib, api, build, synth  # noqa: E402


def model(seed, W, H, K, linear=True, sigma=4.0):
    t = synth.polygon_image(W, H, 3, 8, seed)
    return synth.init_params(t, K, sigma, linear, seed, aniso=(1.0, 2.5),
                             slope_std=0.01 if linear else 0.0)


def static_render(desc, params, y, inv_d, status):
    d, p = desc.c(), params.c()
    return _lib.load().smoe_render_static(ctypes.byref(d), ctypes.byref(p), y.data_ptr(),
                                          inv_d.data_ptr(), status.data_ptr(),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_render_matches_workspace_render_twice():
    build.build()
    cases = [(1, 300, 200, 2000, True, 16), (2, 161, 257, 1500, False, 8)]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for seed, W, H, K, linear, tile in cases:
        p = api.SMoEParams.from_numpy(model(seed, W, H, K, linear))
        desc = api.RasterDesc(W, H, 3, tile, linear)
        y = torch.full((3, H, W), -1.0, device="cuda")
        inv = torch.full((H, W), -1.0, device="cuda")
        assert static_render(desc, p, y, inv, status) == _lib.SMOE_OK
        assert api.smoe_get_status(status) == _lib.SMOE_OK
        y_ref, inv_ref, _ = api.render(p, W, H, tile=tile)
        torch.testing.assert_close(y, y_ref, rtol=1e-5, atol=1e-7)
        torch.testing.assert_close(inv, inv_ref, rtol=1e-5, atol=0.0)


def test_static_render_limits():
    build.build()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # too many kernels: refused before any work
    p = api.SMoEParams.from_numpy(model(3, 64, 64, 32769, False, 1.0))
    desc = api.RasterDesc(64, 64, 3, 16, False)
    y = torch.zeros(3, 64, 64, device="cuda")
    inv = torch.zeros(64, 64, device="cuda")
    assert static_render(desc, p, y, inv, status) == _lib.SMOE_ERR_WORKSPACE
    # raster with more than 16384 tiles: refused
    big = api.RasterDesc(4096, 2048, 3, 8, False)
    yb = torch.zeros(1, device="cuda")
    assert static_render(big, api.SMoEParams.from_numpy(model(4, 64, 64, 64, False)), yb, yb,
                         status) == _lib.SMOE_ERR_WORKSPACE
    # a cutoff beyond the largest one every entry point accepts: refused
    # (smoe_render's raster check, SMOE_ERR_ARG)
    wide = api.RasterDesc(64, 64, 3, 16, False, qmax=200.0)
    small = api.SMoEParams.from_numpy(model(6, 64, 64, 64, False))
    assert static_render(wide, small, y, inv, status) == _lib.SMOE_ERR_ARG
    # too many pairs: reported on the device, image left untouched
    p = api.SMoEParams.from_numpy(model(5, 512, 512, 32768, False, 40.0))
    desc = api.RasterDesc(512, 512, 3, 8, False)
    y = torch.full((3, 512, 512), 7.0, device="cuda")
    inv = torch.zeros(512, 512, device="cuda")
    assert static_render(desc, p, y, inv, status) == _lib.SMOE_OK
    assert api.smoe_get_status(status) == _lib.SMOE_ERR_CAPACITY
    assert bool((y == 7.0).all())
