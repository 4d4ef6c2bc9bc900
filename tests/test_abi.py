"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/smoe.h declares (no GPU needed: nothing is launched)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "smoe.h")).read()
    return sorted(set(re.findall(r"^SMOE_API\s+\w+\s+(smoe_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["smoe_bin", "smoe_render", "smoe_render_backward", "smoe_adam_step", "smoe_fit",
              "smoe_fit_init", "smoe_workspace_size", "smoe_get_status"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2510_05814_gb300 import build, _lib
    build.build()
    lib = ctypes.CDLL(build.LIB)
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(declared()) == sorted(_lib.EXPORTS)
    assert lib.smoe_version() >> 16 == 1


def test_argument_errors_are_synchronous():
    """Host-side argument checks answer without touching a GPU."""
    from paper_2510_05814_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    bad = _lib.Desc(64, 64, 2, 16, 1, 9.0, 1.0)          # C = 2 unsupported
    assert lib.smoe_workspace_size(ctypes.byref(bad), 10, 100, ctypes.byref(n)) == _lib.SMOE_ERR_ARG
    bad = _lib.Desc(64, 64, 3, 12, 1, 9.0, 1.0)          # tile 12 unsupported
    assert lib.smoe_workspace_size(ctypes.byref(bad), 10, 100, ctypes.byref(n)) == _lib.SMOE_ERR_ARG
    ok = _lib.Desc(64, 48, 3, 16, 1, 9.0, 1.0)
    assert lib.smoe_workspace_size(ctypes.byref(ok), 10, 100, ctypes.byref(n)) == _lib.SMOE_OK
    assert n.value > 0 and n.value % 256 == 0
    # unaligned workspace is refused before any launch
    p = _lib.Params(10, 256, 512, 768, 1024)
    st = lib.smoe_bin(ctypes.byref(ok), ctypes.byref(p), ctypes.c_void_p(257), n.value,
                      ctypes.c_void_p(4096), ctypes.c_void_p(8192), 100, ctypes.c_void_p(16),
                      ctypes.c_void_p(32), None)
    assert st == _lib.SMOE_ERR_WORKSPACE
    # constant experts must not pass slopes
    p2 = _lib.Params(10, 256, 512, 768, 1024)
    const = _lib.Desc(64, 48, 3, 16, 0, 9.0, 1.0)
    st = lib.smoe_bin(ctypes.byref(const), ctypes.byref(p2), ctypes.c_void_p(256), n.value,
                      ctypes.c_void_p(4096), ctypes.c_void_p(8192), 100, ctypes.c_void_p(16),
                      ctypes.c_void_p(32), None)
    assert st == _lib.SMOE_ERR_ARG


def test_static_render_and_sharpen_refuse_cutoffs_beyond_the_fp32_range():
    """q_max above 174 (an included pair's gate would flush to 0) is refused
    by the no-allocation render as by smoe_render, and smoe_sharpen refuses a
    factor whose q_max' = q_max f^2 exceeds it; both answer on the host."""
    from paper_2510_05814_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    wide = _lib.Desc(64, 64, 3, 16, 0, 200.0, 1.0, 0)
    p = _lib.Params(10, 256, 512, 768, None, None)
    st = lib.smoe_render_static(ctypes.byref(wide), ctypes.byref(p), ctypes.c_void_p(4096),
                                ctypes.c_void_p(8192), ctypes.c_void_p(16), None)
    assert st == _lib.SMOE_ERR_ARG
    q = ctypes.c_float(-1.0)
    st = lib.smoe_sharpen(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 5.0, 9.0,
                          ctypes.byref(q), None)
    assert st == _lib.SMOE_ERR_ARG and q.value == -1.0
    st = lib.smoe_sharpen(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 2.0, 9.0,
                          None, None)
    assert st == _lib.SMOE_ERR_ARG
    # K = 0 launches nothing: the cutoff comes back from the host
    st = lib.smoe_sharpen(None, None, 0, 3.3, 9.0, ctypes.byref(q), None)
    assert st == _lib.SMOE_OK
    import numpy as np
    assert q.value == float(np.float32(9.0) * (np.float32(3.3) * np.float32(3.3)))
