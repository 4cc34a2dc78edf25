"""bdis_match_noalloc -- the entry point for callers that cannot allocate
device memory (a memory pool that owns the device, a fixed memory budget, a
latency-critical loop that cannot take cudaMalloc's device-wide sync) --
gives the same results as bdis_match.

It is called through the C ABI twice in a row, on pairs of different sizes
and settings, so the second call also shows that the shared static scratch
array carries nothing over from the first.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

import synth
from parity import D_FRAC, D_TOL, V_RTOL

pytestmark = pytest.mark.gpu


def _outputs(h, w):
    import torch
    return (torch.full((h, w), -7.0, dtype=torch.float32, device="cuda"),
            torch.full((h, w), -7.0, dtype=torch.float32, device="cuda"),
            torch.full((h, w), 9, dtype=torch.uint8, device="cuda"))


def _noalloc(bd, params, left, right, out=None):
    import torch
    h, w = left.shape
    d, v, ok = out if out is not None else _outputs(h, w)
    st = bd.B.lib().bdis_match_noalloc(C.byref(params), left.data_ptr(), right.data_ptr(), w, h,
                                       left.stride(0), d.data_ptr(),
                                       v.data_ptr() if params.variance else None, ok.data_ptr(),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, d, v, ok


def _compare(ref, got, variance):
    import torch
    d0, v0, ok0 = ref
    d1, v1, ok1 = got
    assert torch.equal(ok0, ok1)
    m = ok0.bool()
    dd = (d0[m].double() - d1[m].double()).abs()
    assert (dd <= D_TOL).double().mean().item() >= D_FRAC
    assert torch.isnan(d1[~m]).all()
    if variance:
        rel = (v0[m].double() - v1[m].double()).abs() / v0[m].double().abs().clamp_min(1e-12)
        assert (rel <= V_RTOL).all()


def test_noalloc_matches_bdis_match_on_two_calls():
    import torch

    import paper_2205_03133_gb300 as bd
    from paper_2205_03133_gb300 import build
    build.build()
    cases = [
        (synth.config_pair("plain_640x480_var"),
         dict(patch=12, stride=6, levels=4, iters=8, variance=1)),
        (synth.config_pair("plain_320x240"),
         dict(patch=8, stride=4, levels=3, iters=8, variance=0, storage="f16")),
        # the largest pair the static scratch is stated to hold
        (synth.g1_pair(1280, 720, 21),
         dict(patch=8, stride=4, levels=3, iters=8, variance=0, storage="f32")),
    ]
    for pair, kw in cases:
        L = torch.from_numpy(pair.left).cuda()
        R = torch.from_numpy(pair.right).cuda()
        m = bd.BDIS(**kw)
        ref = m.match(L, R)
        torch.cuda.synchronize()
        h, w = pair.left.shape
        outs = [_outputs(h, w), _outputs(h, w)]
        for k in range(2):   # two calls in a row on the shared static scratch
            torch.cuda.synchronize()
            free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
            st, d, v, ok = _noalloc(bd, m.params, L, R, outs[k])
            free1, reserved1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
            assert st == bd.B.BDIS_OK
            _compare(ref, (d, v if kw["variance"] else None, ok), kw["variance"])
            if k == 1:
                # the call allocates no device memory (the first call of a
                # configuration may still load kernel code)
                assert free1 == free0 and reserved1 == reserved0, (free0 - free1)
        m.close()


def test_noalloc_rejects_pairs_beyond_its_scratch():
    import torch

    import paper_2205_03133_gb300 as bd
    p = bd.default_params()
    p.patch, p.stride, p.levels = 8, 4, 3
    L = torch.zeros((1080, 1920), dtype=torch.uint8, device="cuda")
    st, d, v, ok = _noalloc(bd, p, L, L)
    assert st == bd.B.BDIS_EUNSUPPORTED
    assert (ok == 9).all()  # nothing written
