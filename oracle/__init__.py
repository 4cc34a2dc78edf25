"""FP64 CPU oracle for BDIS (arXiv 2205.03133) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``bdis_oracle.c`` (plain
C, FP64, one loop per step of the paper); this module only compiles it with
gcc and marshals arrays through ctypes.

Parity status: the functions are pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute force).
Agreement with the authors' own C++ implementation is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_bdis.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 8
STORE = {"f64": 0, "f32": 1, "f16": 2, "u8": 3}
SIGMA_R = {"pooled": 0, "literal": 1, "fixed": 2}
WEIGHT = {"bdis": 0, "dis": 1}

F_FLAT, F_UNCONVERGED, F_MOVED, F_OUTSIDE, F_SADDLE, F_NONFINITE = (1 << i for i in range(6))
PDF_NOT_PEAK, PDF_FAILED, PDF_RESIDUAL = (1 << i for i in range(3))


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (host code, -O2)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("patch", C.c_int), ("stride", C.c_int), ("levels", C.c_int), ("iters", C.c_int),
        ("sigma_s", C.c_double), ("window_step", C.c_double), ("conv_eps", C.c_double),
        ("valid_gamma", C.c_double), ("pix_thresh", C.c_double), ("search_radius", C.c_double),
        ("sigma_r_mode", C.c_int), ("sigma_r_floor", C.c_double), ("sigma_r_fixed", C.c_double),
        ("variance", C.c_int), ("pdf_iters", C.c_int), ("pdf_resid", C.c_double),
        ("storage", C.c_int), ("hess_eps", C.c_double),
        ("use_sgmm", C.c_int), ("use_c2f", C.c_int),
        ("weight_mode", C.c_int), ("finest_level", C.c_int), ("fast_exp", C.c_int),
    ]


PATCH_DTYPE = np.dtype([
    ("d", "f8"), ("dinit", "f8"), ("E", "f8", (5,)), ("H", "f8"), ("cT", "f8"),
    ("dlast", "f8"), ("nout", "i4"), ("flags", "u4"), ("pi", "f8"), ("rho", "f8"),
    ("sig2", "f8"), ("prop", "f8"), ("pdf_flags", "u4"), ("mu", "f8"),
], align=True)


class Trace(C.Structure):
    _fields_ = [
        ("L", C.c_void_p * MAX_LEVELS), ("R", C.c_void_p * MAX_LEVELS),
        ("G", C.c_void_p * MAX_LEVELS), ("D", C.c_void_p * MAX_LEVELS),
        ("Q", C.c_void_p * MAX_LEVELS), ("patches", C.c_void_p * MAX_LEVELS),
        ("sigma_r", C.c_double * MAX_LEVELS),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.ob_round_f16.restype = C.c_double
        L.ob_round_f16.argtypes = [C.c_double]
        L.ob_round_u8.restype = C.c_double
        L.ob_round_u8.argtypes = [C.c_double]
        L.ob_level_dim.argtypes = [C.c_int, C.c_int]
        L.ob_origins.argtypes = [C.c_int, C.c_int, C.c_int, vp]
        L.ob_gamma_weight.restype = C.c_double
        L.ob_gamma_weight.argtypes = [C.c_int, C.c_int]
        L.ob_gamma_weight_f.restype = C.c_double
        L.ob_gamma_weight_f.argtypes = [C.c_int, C.c_int, C.c_int]
        L.ob_exp_schraudolph.restype = C.c_double
        L.ob_exp_schraudolph.argtypes = [C.c_double]
        L.ob_upsample_output.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                         vp, vp, vp]
        L.ob_pyr_down.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int]
        L.ob_sobel_x.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int]
        L.ob_window_offsets.argtypes = [C.c_double, vp]
        L.ob_search_patch.argtypes = [C.POINTER(Params), vp, vp, vp, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_double, vp]
        L.ob_search_level.argtypes = [C.POINTER(Params), vp, vp, vp, C.c_int, C.c_int,
                                      vp, C.c_int, C.c_int, vp]
        L.ob_sigma_r.restype = C.c_double
        L.ob_sigma_r.argtypes = [C.POINTER(Params), vp, C.c_int]
        L.ob_pdf_fit.restype = C.c_double
        L.ob_pdf_fit.argtypes = [vp, vp, C.c_int, C.c_double, C.c_double, vp, dp, dp, dp]
        L.ob_posterior.argtypes = [C.POINTER(Params), C.c_int, vp, C.c_int, C.c_double,
                                   vp, C.c_int, C.c_int, vp, vp, C.c_int]
        L.ob_sgmm_table.argtypes = [C.c_int, C.c_double, vp]
        L.ob_densify.argtypes = [C.POINTER(Params), vp, vp, C.c_int, vp, C.c_int, C.c_int,
                                 C.c_int, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp, vp]
        L.ob_num_patches.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_int, vp, vp]
        L.ob_check.argtypes = [C.POINTER(Params), C.c_int, C.c_int]
        L.ob_match.argtypes = [C.POINTER(Params), vp, vp, C.c_int, C.c_int, vp, vp, vp,
                               C.POINTER(Trace)]
        L.ob_depth.argtypes = [vp, vp, C.c_long, C.c_double, vp, vp]
        assert L.ob_sizeof_patch() == PATCH_DTYPE.itemsize, "patch record layout mismatch"
        assert L.ob_sizeof_params() == C.sizeof(Params), "params layout mismatch"
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(patch=8, stride=4, levels=3, iters=8, sigma_s=4.0, window_step=0.5,
                conv_eps=0.05, valid_gamma=0.75, pix_thresh=0.15, search_radius=0.0,
                sigma_r_mode="pooled", sigma_r_floor=0.5, sigma_r_fixed=8.0, variance=0,
                pdf_iters=10, pdf_resid=0.1, storage="f32", hess_eps=1e-4, use_sgmm=1,
                use_c2f=1, weight_mode="bdis", finest_level=0, fast_exp=0) -> Params:
    return Params(patch, stride, levels, iters, sigma_s, window_step, conv_eps, valid_gamma,
                  pix_thresh, search_radius, SIGMA_R[sigma_r_mode], sigma_r_floor,
                  sigma_r_fixed, variance, pdf_iters, pdf_resid, STORE[storage], hess_eps,
                  use_sgmm, use_c2f, WEIGHT[weight_mode] if isinstance(weight_mode, str)
                  else int(weight_mode), finest_level, fast_exp)


def level_dim(n: int, l: int) -> int:
    return lib().ob_level_dim(n, l)


def origins(n: int, P: int, S: int) -> np.ndarray:
    k = lib().ob_origins(n, P, S, None)
    out = np.zeros(max(k, 1), dtype=np.int32)
    lib().ob_origins(n, P, S, _ptr(out))
    return out[:k]


def gamma_weight(n: int, levels: int, finest: int = 0) -> float:
    return lib().ob_gamma_weight_f(n, finest, levels)


def exp_schraudolph(y: float) -> float:
    return lib().ob_exp_schraudolph(float(y))


def upsample_output(Df, Vf, okf, f: int, w: int, h: int):
    """Full-resolution disp, var, valid from the level-f maps (f > 0)."""
    Df = np.ascontiguousarray(Df, dtype=np.float64)
    Vf = None if Vf is None else np.ascontiguousarray(Vf, dtype=np.float64)
    okf = np.ascontiguousarray(okf, dtype=np.uint8)
    hf, wf = Df.shape
    disp = np.zeros((h, w)); var = np.zeros((h, w)); valid = np.zeros((h, w), dtype=np.uint8)
    lib().ob_upsample_output(_ptr(Df), _ptr(Vf), _ptr(okf), wf, hf, f, w, h, _ptr(disp),
                             _ptr(var), _ptr(valid))
    return disp, var, valid.astype(bool)


def round_f16(v: float) -> float:
    return lib().ob_round_f16(float(v))


def round_u8(v: float) -> float:
    return lib().ob_round_u8(float(v))


def pyr_down(img: np.ndarray, storage: str = "f64") -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.float64)
    h, w = img.shape
    out = np.zeros(((h + 1) // 2, (w + 1) // 2))
    lib().ob_pyr_down(_ptr(img), w, h, _ptr(out), STORE[storage])
    return out


def sobel_x(img: np.ndarray, storage: str = "f64") -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.float64)
    h, w = img.shape
    out = np.zeros_like(img)
    lib().ob_sobel_x(_ptr(img), w, h, _ptr(out), STORE[storage])
    return out


def window_offsets(h: float = 0.5) -> np.ndarray:
    out = np.zeros(5)
    lib().ob_window_offsets(h, _ptr(out))
    return out


def search_patch(p: Params, L, R, G, ox: int, oy: int, dinit: float) -> np.ndarray:
    L, R, G = (np.ascontiguousarray(a, dtype=np.float64) for a in (L, R, G))
    h, w = L.shape
    rec = np.zeros(1, dtype=PATCH_DTYPE)
    lib().ob_search_patch(C.byref(p), _ptr(L), _ptr(R), _ptr(G), w, h, ox, oy, dinit, _ptr(rec))
    return rec[0]


def search_level(p: Params, L, R, G, Dc=None) -> np.ndarray:
    L, R, G = (np.ascontiguousarray(a, dtype=np.float64) for a in (L, R, G))
    h, w = L.shape
    npx = len(origins(w, p.patch, p.stride))
    npy = len(origins(h, p.patch, p.stride))
    rec = np.zeros(npx * npy, dtype=PATCH_DTYPE)
    if Dc is not None:
        Dc = np.ascontiguousarray(Dc, dtype=np.float64)
        hc, wc = Dc.shape
    else:
        hc = wc = 0
    lib().ob_search_level(C.byref(p), _ptr(L), _ptr(R), _ptr(G), w, h, _ptr(Dc), wc, hc, _ptr(rec))
    return rec.reshape(npy, npx)


def sigma_r(p: Params, rec: np.ndarray) -> float:
    rec = np.ascontiguousarray(rec.ravel())
    return lib().ob_sigma_r(C.byref(p), _ptr(rec), rec.size)


def pdf_fit(lnp, delta, iters=10, resid_max=0.1, tau=8.0):
    lnp = np.ascontiguousarray(lnp, dtype=np.float64)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    fl = np.zeros(1, dtype=np.uint32)
    s, c, rms = C.c_double(), C.c_double(), C.c_double()
    sig2 = lib().ob_pdf_fit(_ptr(lnp), _ptr(delta), iters, resid_max, tau, _ptr(fl),
                            C.byref(s), C.byref(c), C.byref(rms))
    return dict(sig2=sig2, flags=int(fl[0]), sigma=s.value, c=c.value, rms=rms.value)


def posterior(p: Params, level: int, rec: np.ndarray, sr: float, Qc=None, w=None, h=None):
    """Fill pi, rho, sig2 and pdf_flags of one level's record grid (a copy is
    returned).  Qc is the coarser fused probability map; with it, the level
    size (w, h) is needed to place the patch centres."""
    npy, npx = rec.shape
    out = np.ascontiguousarray(rec.copy().ravel())
    if Qc is not None:
        Qc = np.ascontiguousarray(Qc, dtype=np.float64)
        hc, wc = Qc.shape
        ox = origins(w, p.patch, p.stride)
        oy = origins(h, p.patch, p.stride)
    else:
        hc = wc = 0
        ox = origins(npx * p.stride + p.patch, p.patch, p.stride)
        oy = origins(npy * p.stride + p.patch, p.patch, p.stride)
    lib().ob_posterior(C.byref(p), level, _ptr(out), out.size, sr, _ptr(Qc), wc, hc,
                       _ptr(ox), _ptr(oy), npx)
    return out.reshape(npy, npx)


def sgmm_table(P: int, sigma_s: float) -> np.ndarray:
    M = np.zeros((P, P))
    lib().ob_sgmm_table(P, sigma_s, _ptr(M))
    return M


def densify(p: Params, rec: np.ndarray, w: int, h: int, Dc=None, L=None, R=None):
    """Fuse a level's patch records (grid npy x npx) into D, Q, V, count.
    L, R (the level's images) are needed with the DIS weight mode."""
    rec = np.ascontiguousarray(rec)
    if L is not None:
        L = np.ascontiguousarray(L, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
    ox = origins(w, p.patch, p.stride)
    oy = origins(h, p.patch, p.stride)
    assert rec.shape == (len(oy), len(ox))
    D = np.zeros((h, w)); Q = np.zeros((h, w)); V = np.zeros((h, w))
    cnt = np.zeros((h, w), dtype=np.int32)
    if Dc is not None:
        Dc = np.ascontiguousarray(Dc, dtype=np.float64)
        hc, wc = Dc.shape
    else:
        hc = wc = 0
    lib().ob_densify(C.byref(p), _ptr(rec), _ptr(ox), len(ox), _ptr(oy), len(oy), w, h,
                     _ptr(L), _ptr(R), _ptr(Dc), wc, hc, _ptr(D), _ptr(Q), _ptr(V), _ptr(cnt))
    return D, Q, V, cnt


def num_patches(p: Params, w: int, h: int, level: int):
    a, b = C.c_int(), C.c_int()
    n = lib().ob_num_patches(C.byref(p), w, h, level, C.byref(a), C.byref(b))
    return n, a.value, b.value


def match(p: Params, left: np.ndarray, right: np.ndarray, trace: bool = False):
    """Run the whole coarse-to-fine pipeline.  Returns dict with disp, var,
    valid and, if trace, per-level pyramids, records, D, Q and sigma_r."""
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    if lib().ob_check(C.byref(p), w, h):
        raise ValueError("invalid parameters for this image size")
    disp = np.zeros((h, w)); var = np.zeros((h, w)); valid = np.zeros((h, w), dtype=np.uint8)
    tr = None
    keep = {}
    if trace:
        tr = Trace()
        for l in range(p.levels):
            wl, hl = level_dim(w, l), level_dim(h, l)
            n, npx, npy = num_patches(p, w, h, l)
            for key in ("L", "R", "G", "D", "Q"):
                a = np.zeros((hl, wl))
                keep[(key, l)] = a
                getattr(tr, key)[l] = a.ctypes.data
            rec = np.zeros((npy, npx), dtype=PATCH_DTYPE)
            keep[("patches", l)] = rec
            tr.patches[l] = rec.ctypes.data
    rc = lib().ob_match(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, _ptr(disp), _ptr(var),
                        _ptr(valid), C.byref(tr) if tr is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    out = dict(disp=disp, var=var, valid=valid.astype(bool))
    if trace:
        out["levels"] = []
        for l in range(p.levels):
            out["levels"].append({k: keep[(k, l)] for k in ("L", "R", "G", "D", "Q", "patches")}
                                 | {"sigma_r": tr.sigma_r[l]})
    return out


def depth(disp, var, fb: float):
    """Depth z = fb / d (Eq. 13) and its variance (fb)^2 / d^4 * var (Eq. 17);
    NaN where d is not a positive finite number.  var may be None."""
    d = np.ascontiguousarray(disp, dtype=np.float64)
    v = None if var is None else np.ascontiguousarray(var, dtype=np.float64)
    z = np.zeros_like(d)
    zv = None if v is None else np.zeros_like(d)
    lib().ob_depth(_ptr(d), _ptr(v), d.size, float(fb), _ptr(z), _ptr(zv))
    return z, zv


# ---------------------------------------------------------------- differentiable form

def frozen_state(p: Params, out: dict) -> dict:
    """Level-0 discrete state of a traced forward (oracle.match(..., trace=True)):
    kept patches, initial disparities, inherited coarse probabilities, valid
    pixels, and whether sigma_r sat at its floor."""
    lv0 = out["levels"][0]
    rec = lv0["patches"]
    return dict(kept=np.ascontiguousarray((rec["flags"] == 0).astype(np.uint8).ravel()),
                dinit=np.ascontiguousarray(rec["dinit"].ravel()),
                prop=np.ascontiguousarray(rec["prop"].ravel()),
                valid=np.ascontiguousarray(out["valid"].astype(np.uint8)),
                sr_const=int(lv0["sigma_r"] <= p.sigma_r_floor))


def _diff_sigs(L):
    vp = C.c_void_p
    common = [C.POINTER(Params), vp, vp, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, C.c_double]
    L.ob_diff_forward.restype = C.c_double
    L.ob_diff_forward.argtypes = common + [vp, vp, vp]
    L.ob_diff_grad.restype = C.c_double
    L.ob_diff_grad.argtypes = common + [vp, vp, vp, vp]
    L.ob_diff_adjoint.restype = None
    L.ob_diff_adjoint.argtypes = common[:-1] + [vp, vp, vp, vp]


def diff_forward(p: Params, left, right, st: dict, lam: float = 0.1, d_override=None):
    """Frozen-state level-0 function: returns (loss, D, d_k)."""
    L = lib()
    _diff_sigs(L)
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    D = np.zeros((h, w))
    dk = np.zeros(st["kept"].size)
    do = None if d_override is None else np.ascontiguousarray(d_override, dtype=np.float64)
    loss = L.ob_diff_forward(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, _ptr(st["kept"]), _ptr(st["dinit"]),
                             _ptr(st["prop"]), _ptr(st["valid"]), st["sr_const"], lam, _ptr(do),
                             _ptr(D), _ptr(dk))
    return loss, D, dk


def diff_grad(p: Params, left, right, st: dict, lam: float = 0.1):
    """Analytic gradient: returns (loss, dL/dI_l, dL/dI_r, dL/dd_k, dL/dD)."""
    L = lib()
    _diff_sigs(L)
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    gL = np.zeros((h, w)); gR = np.zeros((h, w)); gD = np.zeros((h, w))
    gdk = np.zeros(st["kept"].size)
    loss = L.ob_diff_grad(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, _ptr(st["kept"]), _ptr(st["dinit"]),
                          _ptr(st["prop"]), _ptr(st["valid"]), st["sr_const"], lam, _ptr(gL), _ptr(gR),
                          _ptr(gdk), _ptr(gD))
    return loss, gL, gR, gdk, gD


def diff_adjoint(p: Params, left, right, st: dict, g_disp):
    """The adjoint chain alone (fusion, posterior, window energies, patch
    solve, Sobel) for a given dL/dD: returns (dL/dI_l, dL/dI_r, dL/dd_k)."""
    L = lib()
    _diff_sigs(L)
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    gD = np.ascontiguousarray(np.nan_to_num(g_disp, nan=0.0), dtype=np.float64)
    gL = np.zeros((h, w)); gR = np.zeros((h, w))
    gdk = np.zeros(st["kept"].size)
    L.ob_diff_adjoint(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, _ptr(st["kept"]), _ptr(st["dinit"]),
                      _ptr(st["prop"]), _ptr(st["valid"]), st["sr_const"], _ptr(gD), _ptr(gL),
                      _ptr(gR), _ptr(gdk))
    return gL, gR, gdk


# ---------------------------------------------------------------- differentiable form, all levels

class MState(C.Structure):
    _fields_ = [("kept", C.c_void_p * MAX_LEVELS), ("dinit", C.c_void_p * MAX_LEVELS),
                ("sr_const", C.c_int * MAX_LEVELS), ("valid", C.c_void_p)]


def frozen_state_ml(p: Params, out: dict) -> dict:
    """Per-level discrete state of a traced forward: kept patches, their
    Gauss-Newton starting values, sigma_r at its floor; level-0 valid pixels."""
    st = {"kept": [], "dinit": [], "sr_const": [],
          "valid": np.ascontiguousarray(out["valid"].astype(np.uint8))}
    for lv in out["levels"][:p.levels]:
        rec = lv["patches"]
        st["kept"].append(np.ascontiguousarray((rec["flags"] == 0).astype(np.uint8).ravel()))
        st["dinit"].append(np.ascontiguousarray(rec["dinit"].ravel()))
        st["sr_const"].append(int(lv["sigma_r"] <= p.sigma_r_floor))
    return st


def _mstate(st: dict) -> MState:
    m = MState()
    for n, (k, d) in enumerate(zip(st["kept"], st["dinit"])):
        m.kept[n] = k.ctypes.data
        m.dinit[n] = d.ctypes.data
        m.sr_const[n] = st["sr_const"][n]
    m.valid = st["valid"].ctypes.data
    return m


def mdiff_forward(p: Params, left, right, st: dict, lam: float = 0.1, d_override=None):
    """Frozen-state forward through every level: returns (loss, D, d_k of level 0)."""
    L = lib()
    vp = C.c_void_p
    L.ob_mdiff_forward.restype = C.c_double
    L.ob_mdiff_forward.argtypes = [C.POINTER(Params), vp, vp, C.c_int, C.c_int, C.POINTER(MState),
                                   C.c_double, vp, vp, vp]
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    D = np.zeros((h, w))
    dk = np.zeros(st["kept"][0].size)
    do = None if d_override is None else np.ascontiguousarray(d_override, dtype=np.float64)
    ms = _mstate(st)
    loss = L.ob_mdiff_forward(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, C.byref(ms), lam, _ptr(do),
                              _ptr(D), _ptr(dk))
    return loss, D, dk


def mdiff_grad(p: Params, left, right, st: dict, lam: float = 0.1):
    """Analytic gradient through every level: (loss, dL/dI_l, dL/dI_r, dL/dd_k level 0)."""
    L = lib()
    vp = C.c_void_p
    L.ob_mdiff_grad.restype = C.c_double
    L.ob_mdiff_grad.argtypes = [C.POINTER(Params), vp, vp, C.c_int, C.c_int, C.POINTER(MState),
                                C.c_double, vp, vp, vp]
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    gL = np.zeros((h, w)); gR = np.zeros((h, w))
    gdk = np.zeros(st["kept"][0].size)
    ms = _mstate(st)
    loss = L.ob_mdiff_grad(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, C.byref(ms), lam, _ptr(gL),
                           _ptr(gR), _ptr(gdk))
    return loss, gL, gR, gdk


def mdiff_adjoint(p: Params, left, right, st: dict, g_disp):
    """The adjoint through every level alone for a given level-0 dL/dD:
    (dL/dI_l, dL/dI_r, dL/dd_k of level 0)."""
    L = lib()
    vp = C.c_void_p
    L.ob_mdiff_adjoint.restype = None
    L.ob_mdiff_adjoint.argtypes = [C.POINTER(Params), vp, vp, C.c_int, C.c_int, C.POINTER(MState),
                                   vp, vp, vp, vp]
    Lf = np.ascontiguousarray(left, dtype=np.float64)
    Rf = np.ascontiguousarray(right, dtype=np.float64)
    h, w = Lf.shape
    gD = np.ascontiguousarray(np.nan_to_num(g_disp, nan=0.0), dtype=np.float64)
    gL = np.zeros((h, w)); gR = np.zeros((h, w))
    gdk = np.zeros(st["kept"][0].size)
    ms = _mstate(st)
    L.ob_mdiff_adjoint(C.byref(p), _ptr(Lf), _ptr(Rf), w, h, C.byref(ms), _ptr(gD), _ptr(gL),
                       _ptr(gR), _ptr(gdk))
    return gL, gR, gdk
