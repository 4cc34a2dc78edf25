"""ctypes binding of libbdis.so -- argument marshalling only.

Every entry point has the same name as the C function in ``include/bdis.h``.
Every step of the computation runs in the library's CUDA kernels; this file
passes pointers and sizes.  If the library is not built, loading fails with
an error (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libbdis.so")

BDIS_OK, BDIS_EINVAL, BDIS_ENOMEM, BDIS_ECUDA, BDIS_EUNSUPPORTED = range(5)
STORE_F32, STORE_F16, STORE_U8 = 0, 1, 2
SIGMA_R_POOLED, SIGMA_R_LITERAL, SIGMA_R_FIXED = 0, 1, 2
WEIGHT_BDIS, WEIGHT_DIS = 0, 1

F_FLAT, F_UNCONVERGED, F_MOVED, F_OUTSIDE, F_SADDLE, F_NONFINITE = (1 << i for i in range(6))
PDF_NOT_PEAK, PDF_FAILED, PDF_RESIDUAL = (1 << i for i in range(3))


class bdis_params(C.Structure):
    _fields_ = [
        ("patch", C.c_int), ("stride", C.c_int), ("levels", C.c_int), ("iters", C.c_int),
        ("sigma_s", C.c_float), ("window_step", C.c_float), ("conv_eps", C.c_float),
        ("valid_gamma", C.c_float), ("pix_thresh", C.c_float), ("search_radius", C.c_float),
        ("sigma_r_mode", C.c_int), ("sigma_r_floor", C.c_float), ("sigma_r_fixed", C.c_float),
        ("variance", C.c_int), ("pdf_iters", C.c_int), ("pdf_resid", C.c_float),
        ("storage", C.c_int), ("hess_eps", C.c_float), ("use_sgmm", C.c_int),
        ("use_c2f", C.c_int), ("weight_mode", C.c_int), ("finest_level", C.c_int),
        ("fast_exp", C.c_int),
    ]


class bdis_pair(C.Structure):
    _fields_ = [
        ("left", C.c_void_p), ("right", C.c_void_p), ("w", C.c_int), ("h", C.c_int),
        ("pitch", C.c_int), ("disp", C.c_void_p), ("var", C.c_void_p), ("valid", C.c_void_p),
    ]


class bdis_stats(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("pairs", C.c_int), ("patches", C.c_int * 8),
        ("valid_patches", C.c_int * 8), ("sigma_r", C.c_float * 8),
        ("valid_pixels", C.c_longlong), ("persistent", C.c_int), ("barrier_timeouts", C.c_int),
    ]


class bdis_patch_record(C.Structure):
    _fields_ = [
        ("d", C.c_float), ("dinit", C.c_float), ("dlast", C.c_float), ("H", C.c_float),
        ("E", C.c_float * 5), ("cT", C.c_float), ("flags", C.c_uint32), ("nout", C.c_uint16),
        ("pdf_flags", C.c_uint16), ("pi", C.c_float), ("rho", C.c_float), ("sig2", C.c_float),
        ("mu", C.c_float),
    ]


class bdis_level_view(C.Structure):
    _fields_ = [
        ("w", C.c_int), ("h", C.c_int), ("npx", C.c_int), ("npy", C.c_int),
        ("image_pitch", C.c_int), ("grad_pitch", C.c_int), ("storage", C.c_int), ("left", C.c_void_p),
        ("right", C.c_void_p), ("grad", C.c_void_p), ("records", C.c_void_p),
        ("D", C.c_void_p), ("Q", C.c_void_p), ("sigma_r", C.c_void_p),
    ]


class bdis_pair_f32(C.Structure):
    _fields_ = [
        ("left", C.c_void_p), ("right", C.c_void_p), ("w", C.c_int), ("h", C.c_int),
        ("pitch", C.c_int), ("disp", C.c_void_p), ("var", C.c_void_p), ("valid", C.c_void_p),
    ]


class bdis_grad(C.Structure):
    _fields_ = [("loss", C.c_void_p), ("g_disp", C.c_void_p), ("g_left", C.c_void_p),
                ("g_right", C.c_void_p), ("g_patch_disp", C.c_void_p)]


class bdis_profile(C.Structure):
    _fields_ = [("launches", C.c_int * 5), ("ms", C.c_double * 5),
                ("launches_level", (C.c_int * 8) * 5), ("ms_level", (C.c_double * 8) * 5)]


OPT_GRAPH, OPT_PROFILE, OPT_AUTOTUNE, OPT_FORM, OPT_PDL, OPT_PYRAMID_STEPS, OPT_ADJOINT_LEVELS = (
    1, 2, 3, 4, 5, 6, 7)
OPT_HOST_MAPPED = 8
OPT_BARRIER_LIMIT, OPT_BARRIER_TEST, OPT_COARSE_LEVELS, OPT_BULK_COPY = 9, 10, 11, 12
OPT_SEARCH_PASSES, OPT_FUSE_TILE = 13, 14
KERNEL_NAMES = ["pyramid", "search", "fuse", "persistent", "upsample"]


# (name, restype, argtypes) of every exported function of include/bdis.h
_vp = C.c_void_p
_h = C.c_void_p
EXPORTS = [
    ("bdis_default_params", None, [C.POINTER(bdis_params)]),
    ("bdis_create", C.c_int, [C.POINTER(bdis_params), C.POINTER(C.c_void_p)]),
    ("bdis_destroy", None, [_h]),
    ("bdis_strerror", C.c_char_p, [C.c_int]),
    ("bdis_last_error", C.c_char_p, [_h]),
    ("bdis_get_params", C.c_int, [_h, C.POINTER(bdis_params)]),
    ("bdis_match", C.c_int, [_h, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
    ("bdis_match_host", C.c_int, [_h, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
    ("bdis_match_batched", C.c_int, [_h, C.c_int, C.POINTER(bdis_pair), _vp]),
    ("bdis_get_stats", C.c_int, [_h, C.POINTER(bdis_stats), _vp]),
    ("bdis_wait", C.c_int, [_h, _vp]),
    ("bdis_level_view_get", C.c_int, [_h, C.c_int, C.c_int, C.POINTER(bdis_level_view)]),
    ("bdis_copy", C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    ("bdis_set_option", C.c_int, [_h, C.c_int, C.c_int]),
    ("bdis_get_profile", C.c_int, [_h, C.POINTER(bdis_profile), C.c_int]),
    ("bdis_match_f32", C.c_int, [_h, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
    ("bdis_match_batched_f32", C.c_int, [_h, C.c_int, C.POINTER(bdis_pair_f32), _vp]),
    ("bdis_saved_create", C.c_int, [_h, C.POINTER(C.c_void_p)]),
    ("bdis_saved_destroy", None, [_vp]),
    ("bdis_match_batched_f32_saved", C.c_int, [_h, C.c_int, C.POINTER(bdis_pair_f32), _vp, _vp]),
    ("bdis_loss", C.c_int, [_h, _vp, C.c_float, C.POINTER(bdis_grad), _vp]),
    ("bdis_backward", C.c_int, [_h, _vp, C.POINTER(bdis_grad), _vp]),
    ("bdis_match_noalloc", C.c_int, [C.POINTER(bdis_params), _vp, _vp, C.c_int, C.c_int, C.c_int,
                                     _vp, _vp, _vp, _vp]),
    ("bdis_depth", C.c_int, [_vp, _vp, C.c_longlong, C.c_float, _vp, _vp, _vp]),
    ("bdis_probe_l2_read", C.c_int, [_vp, C.c_size_t, C.c_int, _vp]),
]

_lib = None


def lib():
    """Load libbdis.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libbdis.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2205_03133_gb300.build` (CUDA toolkit required)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in EXPORTS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class BdisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status: int, handle=None):
    if status != BDIS_OK:
        msg = lib().bdis_last_error(handle).decode() if handle else lib().bdis_strerror(status).decode()
        raise BdisError(status, msg)
