"""ctypes declarations of libsmoe.so (mirrors include/smoe.h)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmoe.so")

SMOE_OK, SMOE_ERR_ARG, SMOE_ERR_CAPACITY, SMOE_ERR_CUDA, SMOE_ERR_TIMEOUT, SMOE_ERR_WORKSPACE = range(6)
STATUS_NAMES = {0: "SMOE_OK", 1: "SMOE_ERR_ARG", 2: "SMOE_ERR_CAPACITY", 3: "SMOE_ERR_CUDA",
                4: "SMOE_ERR_TIMEOUT", 5: "SMOE_ERR_WORKSPACE"}

EXPORTS = ["smoe_version", "smoe_workspace_size", "smoe_bin", "smoe_render",
           "smoe_render_backward", "smoe_adam_step", "smoe_sq_error",
           "smoe_fit_workspace_size", "smoe_fit_init", "smoe_fit", "smoe_fit_phase",
           "smoe_fit_gradients",
           "smoe_fit_render_mean", "smoe_render_mean_workspace_size", "smoe_render_mean",
           "smoe_sharpen", "smoe_points_workspace_size",
           "smoe_render_points", "smoe_count_inrange", "smoe_render_static",
           "smoe_get_status", "smoe_fit_reorder", "smoe_scatter_params"]


class SmoeError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS_NAMES.get(self.code, self.code)}")


class Desc(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("C", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("expert", ctypes.c_int32),
                ("qmax", ctypes.c_float), ("scale", ctypes.c_float), ("gate", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("mu", ctypes.c_void_p), ("chol", ctypes.c_void_p),
                ("ea", ctypes.c_void_p), ("eW", ctypes.c_void_p), ("logpi", ctypes.c_void_p)]


class FitImage(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("target", ctypes.c_void_p),
                ("p", Params), ("m", Params), ("v", Params),
                ("iters", ctypes.c_int32), ("lr_mu0", ctypes.c_float),
                ("lr_mu1", ctypes.c_float), ("lr_chol", ctypes.c_float),
                ("lr_ea", ctypes.c_float), ("lr_eW", ctypes.c_float), ("lr_pi", ctypes.c_float)]


class FitBatch(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("C", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("expert", ctypes.c_int32), ("qmax", ctypes.c_float), ("b1", ctypes.c_double),
                ("b2", ctypes.c_double), ("eps", ctypes.c_double), ("step", ctypes.c_void_p),
                ("loss", ctypes.c_void_p), ("hist", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("gate", ctypes.c_int32)]


_lib = None


def load():
    """Load libsmoe.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, F32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    D, PP = ctypes.POINTER(Desc), ctypes.POINTER(Params)
    FB, FI = ctypes.POINTER(FitBatch), ctypes.POINTER(FitImage)
    SZ = ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "smoe_version": (I32, []),
        "smoe_workspace_size": (I32, [D, I64, I64, SZ]),
        "smoe_bin": (I32, [D, PP, P, ctypes.c_size_t, P, P, I64, P, P, P]),
        "smoe_render": (I32, [D, I64, P, ctypes.c_size_t, P, P, P, P, P, P]),
        "smoe_render_backward": (I32, [D, PP, P, ctypes.c_size_t, P, P, P, P, P, P, PP, P, P]),
        "smoe_adam_step": (I32, [PP, PP, PP, PP, I32, ctypes.POINTER(F32), ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, I32, P]),
        "smoe_sq_error": (I32, [P, P, I64, I32, P, P]),
        "smoe_fit_workspace_size": (I32, [FB, FI, I64, SZ]),
        "smoe_fit_init": (I32, [FB, FI, I64, P, ctypes.c_size_t, I32, P, P]),
        "smoe_fit": (I32, [FB, FI, I64, P, ctypes.c_size_t, I32, P, P]),
        "smoe_fit_phase": (I32, [FB, FI, I64, P, ctypes.c_size_t, I32, P, P]),
        "smoe_fit_gradients": (I32, [FB, FI, I64, P, ctypes.c_size_t, PP, P, P]),
        "smoe_fit_render_mean": (I32, [FB, FI, I64, P, ctypes.c_size_t, P, P, P]),
        "smoe_render_mean_workspace_size": (I32, [D, PP, I32, I64, SZ]),
        "smoe_render_mean": (I32, [D, PP, I32, P, ctypes.c_size_t, I64, P, P, P]),
        "smoe_sharpen": (I32, [P, P, I64, ctypes.c_float, ctypes.c_float,
                                ctypes.POINTER(ctypes.c_float), P]),
        "smoe_points_workspace_size": (I32, [D, I64, ctypes.POINTER(ctypes.c_size_t)]),
        "smoe_render_points": (I32, [D, I64, P, ctypes.c_size_t, P, P, I64, P, P,
                                     ctypes.c_size_t, P, P, P, P]),
        "smoe_count_inrange": (I32, [D, I64, P, ctypes.c_size_t, P, P, P, P, P]),
        "smoe_render_static": (I32, [D, PP, P, P, P, P]),
        "smoe_get_status": (I32, [P, P]),
        "smoe_fit_reorder": (I32, [FB, FI, I64, P, ctypes.c_size_t, P, P, P]),
        "smoe_scatter_params": (I32, [PP, P, I64, I32, PP, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(code, what):
    if code != SMOE_OK:
        raise SmoeError(code, what)
