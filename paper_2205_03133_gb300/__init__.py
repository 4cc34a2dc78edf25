"""GB300 (sm_103a) BDIS -- Bayesian Dense Inverse Search for rectified stereo
(arXiv 2205.03133) behind the C ABI of ``include/bdis.h``.

PyTorch supplies device memory and streams; every step of the pipeline runs
in the library's CUDA kernels.  Example::

    import torch, paper_2205_03133_gb300 as bd
    m = bd.BDIS(patch=12, stride=6, levels=4, variance=1)
    disp, var, valid = m.match(left_u8_cuda, right_u8_cuda)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _binding as B
from ._binding import BdisError

__all__ = ["BDIS", "BdisError", "default_params", "B", "_grad_table", "depth", "SavedState"]

_STORAGE = {"f32": B.STORE_F32, "f16": B.STORE_F16, "u8": B.STORE_U8}
_SIGMA_R = {"pooled": B.SIGMA_R_POOLED, "literal": B.SIGMA_R_LITERAL, "fixed": B.SIGMA_R_FIXED}
_WEIGHT = {"bdis": B.WEIGHT_BDIS, "dis": B.WEIGHT_DIS}


def default_params() -> B.bdis_params:
    p = B.bdis_params()
    B.lib().bdis_default_params(C.byref(p))
    return p


def _params(**kw) -> B.bdis_params:
    p = default_params()
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = _STORAGE[v]
        if k == "sigma_r_mode" and isinstance(v, str):
            v = _SIGMA_R[v]
        if k == "weight_mode" and isinstance(v, str):
            v = _WEIGHT[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown BDIS parameter {k!r}")
        setattr(p, k, v)
    return p


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class BDIS:
    """One library handle (owns a device scratch arena)."""

    def __init__(self, **params):
        self.params = _params(**params)
        h = C.c_void_p()
        B.check(B.lib().bdis_create(C.byref(self.params), C.byref(h)))
        self._h = h

    def set_option(self, option: int, value: int):
        B.check(B.lib().bdis_set_option(self._h, option, value), self._h)

    def close(self):
        if getattr(self, "_h", None):
            for sv in getattr(self, "_saved_pool", []):
                sv.destroy()
            self._saved_pool = []
            B.lib().bdis_destroy(self._h)
            self._h = None

    def wait(self, stream=None):
        """Wait for the handle's calls on `stream`; raises BdisError when a
        persistent-form call's grid-barrier wait ran out."""
        B.check(B.lib().bdis_wait(self._h, _stream_handle(stream)), self._h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ device API
    def match(self, left, right, out=None, stream=None):
        """left, right: (h, w) uint8 CUDA tensors (row stride >= w).
        Returns (disp float32, var float32 or None, valid uint8) CUDA tensors."""
        import torch
        assert left.dtype == torch.uint8 and right.dtype == torch.uint8
        assert left.is_cuda and right.is_cuda and left.shape == right.shape
        assert left.stride(1) == 1 and right.stride(1) == 1 and left.stride(0) == right.stride(0)
        h, w = left.shape
        if out is None:
            disp = torch.empty((h, w), dtype=torch.float32, device=left.device)
            var = (torch.empty((h, w), dtype=torch.float32, device=left.device)
                   if self.params.variance else None)
            valid = torch.empty((h, w), dtype=torch.uint8, device=left.device)
        else:
            disp, var, valid = out
        st = B.lib().bdis_match(self._h, left.data_ptr(), right.data_ptr(), w, h, left.stride(0),
                                disp.data_ptr(), var.data_ptr() if var is not None else None,
                                valid.data_ptr(), _stream_handle(stream))
        B.check(st, self._h)
        return disp, var, valid

    def match_batched(self, lefts, rights, outs=None, stream=None):
        """Lists of (h_i, w_i) uint8 CUDA tensors; returns a list of
        (disp, var, valid) per pair."""
        import torch
        n = len(lefts)
        arr = (B.bdis_pair * n)()
        results = []
        for i, (l, r) in enumerate(zip(lefts, rights)):
            h, w = l.shape
            if outs is None:
                d = torch.empty((h, w), dtype=torch.float32, device=l.device)
                v = (torch.empty((h, w), dtype=torch.float32, device=l.device)
                     if self.params.variance else None)
                m = torch.empty((h, w), dtype=torch.uint8, device=l.device)
            else:
                d, v, m = outs[i]
            arr[i] = B.bdis_pair(l.data_ptr(), r.data_ptr(), w, h, l.stride(0), d.data_ptr(),
                                 v.data_ptr() if v is not None else None, m.data_ptr())
            results.append((d, v, m))
        B.check(B.lib().bdis_match_batched(self._h, n, arr, _stream_handle(stream)), self._h)
        return results

    # ------------------------------------------------------------ host API
    def match_host(self, left: np.ndarray, right: np.ndarray, out=None, stream=None):
        """numpy uint8 (h, w) inputs (ideally pinned); returns numpy outputs."""
        left = np.ascontiguousarray(left, dtype=np.uint8)
        right = np.ascontiguousarray(right, dtype=np.uint8)
        h, w = left.shape
        if out is None:
            disp = np.empty((h, w), np.float32)
            var = np.empty((h, w), np.float32) if self.params.variance else None
            valid = np.empty((h, w), np.uint8)
        else:
            disp, var, valid = out
        st = B.lib().bdis_match_host(
            self._h, left.ctypes.data, right.ctypes.data, w, h, w, disp.ctypes.data,
            var.ctypes.data if var is not None else None, valid.ctypes.data,
            _stream_handle(stream) if stream is not None else None)
        B.check(st, self._h)
        return disp, var, valid

    def match_host_ptr(self, left_ptr, right_ptr, w, h, disp_ptr, var_ptr, valid_ptr, stream):
        """Raw host-pointer form (pinned torch tensors' data_ptr())."""
        st = B.lib().bdis_match_host(self._h, left_ptr, right_ptr, w, h, w, disp_ptr, var_ptr,
                                     valid_ptr, stream)
        B.check(st, self._h)

    # ------------------------------------------------------------ inspection
    def stats(self, stream=None) -> dict:
        s = B.bdis_stats()
        B.check(B.lib().bdis_get_stats(self._h, C.byref(s), _stream_handle(stream)), self._h)
        return dict(levels=s.levels, pairs=s.pairs, patches=list(s.patches)[:s.levels],
                    valid_patches=list(s.valid_patches)[:s.levels],
                    sigma_r=list(s.sigma_r)[:s.levels], valid_pixels=s.valid_pixels,
                    persistent=s.persistent, barrier_timeouts=s.barrier_timeouts)

    def level_view(self, pair: int, level: int) -> dict:
        """Copies of the last call's intermediate buffers of (pair, level)."""
        v = B.bdis_level_view()
        B.check(B.lib().bdis_level_view_get(self._h, pair, level, C.byref(v)), self._h)
        out = dict(w=v.w, h=v.h, npx=v.npx, npy=v.npy)

        def cp(ptr, dtype, shape):
            a = np.empty(shape, dtype=dtype)
            B.check(B.lib().bdis_copy(a.ctypes.data, ptr, a.nbytes, None))
            return a

        rec = np.dtype([("d", "f4"), ("dinit", "f4"), ("dlast", "f4"), ("H", "f4"),
                        ("E", "f4", (5,)), ("cT", "f4"), ("flags", "u4"), ("nout", "u2"),
                        ("pdf_flags", "u2"), ("pi", "f4"), ("rho", "f4"), ("sig2", "f4"),
                        ("mu", "f4")])
        assert rec.itemsize == C.sizeof(B.bdis_patch_record)
        if not v.records:  # below the finest processed level: no search there
            out["patches"] = None
        else:
            out["patches"] = cp(v.records, rec, (v.npy, v.npx))
        sr = cp(v.sigma_r, np.float32, (1,))
        out["sigma_r"] = float(sr[0])
        if level > 0:
            out["D"] = cp(v.D, np.float32, (v.h, v.w))
            out["Q"] = cp(v.Q, np.float32, (v.h, v.w))
            dt = {B.STORE_F16: np.float16, B.STORE_U8: np.uint8}.get(v.storage, np.float32)
            pitch = v.image_pitch
            for key, ptr in (("L", v.left), ("R", v.right)):
                out[key] = cp(ptr, dt, (v.h, pitch))[:, :v.w].astype(np.float64)
        gdt = np.float32 if self.params.storage == B.STORE_F32 else np.float16
        out["G"] = (cp(v.grad, gdt, (v.h, v.grad_pitch))[:, :v.w].astype(np.float64)
                    if v.grad else None)
        return out


# ---------------------------------------------------------------- differentiable form

class SavedState:
    """Caller-owned state of one differentiable forward (bdis_saved): the
    forward's pyramids, gradients, records and weight sums live in this
    object's device memory, plus the tensors of that forward (images and
    outputs) that the loss and the adjoint read, kept alive here."""

    def __init__(self, model: "BDIS"):
        s = C.c_void_p()
        B.check(B.lib().bdis_saved_create(model._h, C.byref(s)), model._h)
        self._s = s
        self.keep = None
        self.shapes = None

    @property
    def handle(self):
        return self._s

    def destroy(self):
        if getattr(self, "_s", None):
            B.lib().bdis_saved_destroy(self._s)
            self._s = None
        self.keep = None


def _f32_pair(l, r, d, v, m):
    h, w = l.shape
    return B.bdis_pair_f32(l.data_ptr(), r.data_ptr(), w, h, l.stride(0), d.data_ptr(),
                           v.data_ptr() if v is not None else None, m.data_ptr())


def _match_f32(self, lefts, rights, outs=None, stream=None, saved=None):
    """Forward on float32 CUDA images (lists of (h, w) tensors); returns a list
    of (disp, var, valid) (preallocated `outs` are filled if given).
    Required before loss_and_grad / backward.  With `saved` (a SavedState of
    this model) the forward's state is kept there instead of in the handle."""
    import torch
    n = len(lefts)
    arr = (B.bdis_pair_f32 * n)()
    res = []
    for i, (l, r) in enumerate(zip(lefts, rights)):
        assert l.dtype == torch.float32 and r.dtype == torch.float32 and l.is_cuda
        assert l.stride(1) == 1 and l.stride(0) == r.stride(0)
        h, w = l.shape
        if outs is not None:
            d, v, m = outs[i]
        else:
            d = torch.empty((h, w), dtype=torch.float32, device=l.device)
            v = (torch.empty((h, w), dtype=torch.float32, device=l.device)
                 if self.params.variance else None)
            m = torch.empty((h, w), dtype=torch.uint8, device=l.device)
        arr[i] = _f32_pair(l, r, d, v, m)
        res.append((d, v, m))
    # the loss and the adjoint read the forward's images and outputs: keep
    # them alive as long as the state that points at them
    keep = (list(lefts), list(rights), res)
    shapes = [tuple(l.shape) for l in lefts]
    if saved is None:
        B.check(B.lib().bdis_match_batched_f32(self._h, n, arr, _stream_handle(stream)), self._h)
        self._f32_shapes = shapes
        self._f32_keep = keep
    else:
        B.check(B.lib().bdis_match_batched_f32_saved(self._h, n, arr, saved.handle,
                                                     _stream_handle(stream)), self._h)
        saved.shapes = shapes
        saved.keep = keep
    return res


def _grad_table(self, bufs):
    """ctypes table of per-pair gradient buffers (dicts of CUDA tensors)."""
    n = len(bufs)
    arr = (B.bdis_grad * n)()
    for i, b in enumerate(bufs):
        arr[i] = B.bdis_grad(*(t.data_ptr() if t is not None else None for t in
                               (b.get("loss"), b["g_disp"], b["g_left"], b["g_right"],
                                b.get("g_patch_disp"))))
    return arr


def _patch_grid(self, w, h):
    """Level-0 patch grid (npx, npy) of a w x h pair (origins every S px plus
    a ragged last one, so that every pixel is covered)."""
    P, S = self.params.patch, self.params.stride

    def n(x):
        return (x - P) // S + 1 + (1 if (x - P) % S else 0)

    return n(w), n(h)


def _saved_ptr(saved):
    return saved.handle if saved is not None else None


def _loss_and_grad(self, lam=0.1, stream=None, saved=None):
    """L1 reprojection + lam * smoothness of a float forward (the one kept in
    `saved`, else the last one on the handle) and its gradients.  Returns per
    pair dict(loss, g_disp, g_left, g_right, g_patch_disp) (CUDA tensors)."""
    import torch
    bufs = []
    shapes = saved.shapes if saved is not None else self._f32_shapes
    for (h, w) in shapes:
        npx, npy = _patch_grid(self, w, h)
        dev = torch.device("cuda", torch.cuda.current_device())
        bufs.append(dict(loss=torch.empty(1, device=dev), g_disp=torch.empty((h, w), device=dev),
                         g_left=torch.empty((h, w), device=dev),
                         g_right=torch.empty((h, w), device=dev),
                         g_patch_disp=torch.empty((npy, npx), device=dev)))
    arr = _grad_table(self, bufs)
    st = _stream_handle(stream)
    B.check(B.lib().bdis_loss(self._h, _saved_ptr(saved), C.c_float(lam), arr, st), self._h)
    B.check(B.lib().bdis_backward(self._h, _saved_ptr(saved), arr, st), self._h)
    return bufs


def _backward(self, g_disps, stream=None, saved=None):
    """Adjoint of a float forward (the one kept in `saved`, else the last one
    on the handle) for caller-supplied dL/dD (list of (h, w) tensors);
    returns (g_left, g_right, g_patch_disp) per pair."""
    import torch
    bufs = []
    for gd in g_disps:
        h, w = gd.shape
        npx, npy = _patch_grid(self, w, h)
        bufs.append(dict(g_disp=torch.nan_to_num(gd.float(), nan=0.0).contiguous(),
                         g_left=torch.zeros((h, w), device=gd.device),
                         g_right=torch.zeros((h, w), device=gd.device),
                         g_patch_disp=torch.empty((npy, npx), device=gd.device)))
    arr = _grad_table(self, bufs)
    B.check(B.lib().bdis_backward(self._h, _saved_ptr(saved), arr, _stream_handle(stream)),
            self._h)
    return [(b["g_left"], b["g_right"], b["g_patch_disp"]) for b in bufs]


def _take_saved(self) -> SavedState:
    """A SavedState of this model: a released one if any (its device memory
    and the handle's captured launch sequence are reused), else a new one."""
    pool = self.__dict__.setdefault("_saved_pool", [])
    return pool.pop() if pool else SavedState(self)


def _release_saved(self, sv: SavedState):
    if getattr(self, "_h", None) is None:
        sv.destroy()
        return
    sv.keep = None
    self.__dict__.setdefault("_saved_pool", []).append(sv)


BDIS.match_f32 = _match_f32
BDIS.loss_and_grad = _loss_and_grad
BDIS.backward = _backward
BDIS.saved_state = lambda self: SavedState(self)
BDIS._take_saved = _take_saved
BDIS._release_saved = _release_saved


def disparity(model: "BDIS", left, right):
    """Differentiable dense disparity of one float32 pair (torch autograd).
    Returns (disp, valid); disp is NaN at invalid pixels and the gradient
    flows to `left` and `right` through the library's adjoint.  Each call's
    forward state lives in its own SavedState held by the autograd graph, so
    any number of forwards on one model can be differentiated, in any order;
    the state returns to the model's pool when the graph is freed."""
    return _Disparity.apply(model, left, right)


class _SavedLease:
    """Ties a SavedState to an autograd graph: released to the model's pool
    when the graph (and with it this object) is freed."""

    def __init__(self, model, sv):
        self.model, self.sv = model, sv

    def __del__(self):
        try:
            self.model._release_saved(self.sv)
        except Exception:
            pass


def _autograd_cls():
    import torch

    class Disparity(torch.autograd.Function):
        @staticmethod
        def forward(ctx, model, left, right):
            sv = model._take_saved()
            (d, _, m), = model.match_f32([left.detach().contiguous()],
                                         [right.detach().contiguous()], saved=sv)
            ctx.model = model
            ctx.lease = _SavedLease(model, sv)
            ctx.mark_non_differentiable(m)
            return d, m

        @staticmethod
        def backward(ctx, g_disp, g_valid):
            (gl, gr, _), = ctx.model.backward([g_disp], saved=ctx.lease.sv)
            return None, gl, gr

    return Disparity


class _Lazy:
    cls = None

    def apply(self, *a):
        if _Lazy.cls is None:
            _Lazy.cls = _autograd_cls()
        return _Lazy.cls.apply(*a)


_Disparity = _Lazy()
__all__ += ["disparity"]


# ---------------------------------------------------------------- depth

def depth(disp, var=None, fb: float = 1.0, stream=None):
    """Depth fb / disp (Eq. 13) and, given the disparity variance, the depth
    variance fb^2 / disp^4 var (Eq. 17) of device tensors, computed by the
    library's elementwise kernel.  fb = focal length (px) x baseline."""
    import torch
    disp = disp.contiguous()
    assert disp.is_cuda and disp.dtype == torch.float32
    z = torch.empty_like(disp)
    zv = None
    if var is not None:
        var = var.contiguous()
        assert var.shape == disp.shape and var.dtype == torch.float32
        zv = torch.empty_like(disp)
    B.check(B.lib().bdis_depth(C.c_void_p(disp.data_ptr()),
                               C.c_void_p(var.data_ptr()) if var is not None else None,
                               disp.numel(), C.c_float(fb), C.c_void_p(z.data_ptr()),
                               C.c_void_p(zv.data_ptr()) if zv is not None else None,
                               _stream_handle(stream)))
    return z, zv
