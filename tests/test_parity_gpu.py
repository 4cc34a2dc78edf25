"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (tolerances in tests/parity.py)."""
import numpy as np
import pytest

import oracle
import synth
from parity import (D_FRAC, D_TOL, V_RTOL, V_RTOL_DIS, assert_gate, compare_outputs,
                    compare_records, oracle_params)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bd():
    import paper_2205_03133_gb300 as bd
    from paper_2205_03133_gb300 import build
    build.build()
    return bd


def _run(bd, kw, left, right, views=True):
    import torch
    m = bd.BDIS(**kw)
    L = torch.from_numpy(np.ascontiguousarray(left)).cuda()
    R = torch.from_numpy(np.ascontiguousarray(right)).cuda()
    disp, var, valid = m.match(L, R)
    torch.cuda.synchronize()
    out = dict(disp=disp.cpu().numpy(), var=None if var is None else var.cpu().numpy(),
               valid=valid.cpu().numpy(), params=m.params)
    if views:
        out["levels"] = [m.level_view(0, l) for l in range(m.params.levels)]
    m.close()
    return out


def _check_pair(bd, kw, pair, report=None):
    g = _run(bd, kw, pair.left, pair.right)
    op = oracle_params(g["params"])
    o = oracle.match(op, pair.left, pair.right, trace=True)
    F = op.finest_level
    for l in range(F, op.levels):
        c = compare_records(g["levels"][l]["patches"], o["levels"][l]["patches"])
        assert c["decision_flips"] <= max(2, int(0.001 * c["patches"])), (l, c)
        assert c["d_frac_within"] >= D_FRAC, (l, c)
    m = compare_outputs(g["params"], o, g["disp"], g["var"], g["valid"], g["levels"][F]["patches"])
    if report is not None:
        report.update(m)
    assert_gate(m, V_RTOL_DIS if op.weight_mode == 1 else V_RTOL)
    return g, o, m


CASES = {
    "plain_320x240": dict(patch=8, stride=4, levels=3, iters=8),
    "plain_640x480_var": dict(patch=12, stride=6, levels=4, iters=8, variance=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_workload_parity(bd, name):
    pair = synth.config_pair(name)
    m = {}
    _check_pair(bd, CASES[name], pair, m)
    print(name, m)


def test_pyramid_and_gradient_f32(bd):
    pair = synth.config_pair("plain_320x240")
    g = _run(bd, CASES["plain_320x240"], pair.left, pair.right)
    o = oracle.match(oracle_params(g["params"]), pair.left, pair.right, trace=True)
    for l in range(3):
        gv, ov = g["levels"][l], o["levels"][l]
        np.testing.assert_allclose(gv["G"], ov["G"], atol=2e-4)
        if l > 0:
            np.testing.assert_allclose(gv["L"], ov["L"], atol=2e-4)
            np.testing.assert_allclose(gv["R"], ov["R"], atol=2e-4)


def test_pyramid_and_gradient_f16(bd):
    pair = synth.g1_pair(250, 130, 3)
    kw = dict(patch=12, stride=4, levels=3, iters=8, storage="f16")
    g = _run(bd, kw, pair.left, pair.right)
    o = oracle.match(oracle_params(g["params"]), pair.left, pair.right, trace=True)
    for l in range(3):
        gv, ov = g["levels"][l], o["levels"][l]
        keys = ("G", "L", "R") if l > 0 else ("G",)
        for k in keys:
            diff = np.abs(gv[k] - ov[k])
            # fp16 values: equal except rare double-rounding cases (one ulp)
            assert (diff > 0).mean() <= 0.01, (l, k, (diff > 0).mean())
            assert diff.max() <= 0.13, (l, k, diff.max())


@pytest.mark.parametrize("w,h,kw", [
    (97, 61, dict(patch=8, stride=4, levels=2, iters=8)),          # ragged grid
    (203, 117, dict(patch=10, stride=4, levels=3, iters=6)),       # P not a power of two
    (250, 130, dict(patch=12, stride=4, levels=3, iters=8, storage="f16", variance=1)),
    (128, 96, dict(patch=8, stride=8, levels=2, iters=4)),         # no overlap
    (32, 32, dict(patch=8, stride=4, levels=3, iters=8)),          # minimum size
    (160, 120, dict(patch=16, stride=5, levels=2, iters=10, variance=1)),
    (160, 120, dict(patch=6, stride=3, levels=2, iters=8, sigma_r_mode="literal")),
    (160, 120, dict(patch=8, stride=4, levels=2, iters=8, sigma_r_mode="fixed")),
    (160, 120, dict(patch=8, stride=4, levels=3, iters=8, use_sgmm=0, use_c2f=0)),
    (160, 120, dict(patch=8, stride=4, levels=1, iters=8, variance=1)),
    (160, 120, dict(patch=8, stride=4, levels=2, iters=0)),
    (64, 48, dict(patch=4, stride=1, levels=2, iters=8)),          # smallest patch, densest grid
    (96, 80, dict(patch=16, stride=1, levels=1, iters=6, variance=1)),  # 256 patches per pixel
    # stride 1 with 16 lanes per patch: the groups of a warp are 16 patches
    # apart, and level 1 (82 x 49) ends each patch row with a chunk of 9
    (163, 97, dict(patch=10, stride=1, levels=2, iters=6, variance=1)),
])
def test_ragged_and_parameter_cases(bd, w, h, kw):
    pair = synth.g1_pair(w, h, w * 7 + h)
    _check_pair(bd, kw, pair)


def test_pyramid_and_gradient_u8(bd):
    # 8-bit pyramid levels (nearest integer, ties to even) and FP16 gradients
    pair = synth.g1_pair(250, 130, 4)
    kw = dict(patch=12, stride=4, levels=3, iters=8, storage="u8")
    g = _run(bd, kw, pair.left, pair.right)
    o = oracle.match(oracle_params(g["params"]), pair.left, pair.right, trace=True)
    for l in range(3):
        gv, ov = g["levels"][l], o["levels"][l]
        keys = ("G", "L", "R") if l > 0 else ("G",)
        for k in keys:
            diff = np.abs(gv[k] - ov[k])
            # equal except where the FP32 blur and the FP64 one round to
            # different integers (a value within rounding of a half step)
            assert (diff > 0).mean() <= 0.01, (l, k, (diff > 0).mean())
            assert diff.max() <= (1.0 if k != "G" else 0.5), (l, k, diff.max())
        if l > 0:
            assert np.array_equal(gv["L"], np.round(gv["L"]))  # integers 0..255
            assert gv["L"].min() >= 0 and gv["L"].max() <= 255


@pytest.mark.parametrize("name,kw", [
    ("plain_640x480_var", dict(patch=12, stride=6, levels=4, iters=8, variance=1, storage="u8")),
    ("plain_320x240", dict(patch=8, stride=4, levels=3, iters=8, storage="u8")),
])
def test_u8_storage_workload_parity(bd, name, kw):
    m = {}
    _check_pair(bd, kw, synth.config_pair(name), m)
    print(name, "u8 storage", m)


def test_u8_storage_batched_equals_plain(bd):
    import torch
    sizes = [(160, 120), (97, 61), (256, 144)]
    pairs = [synth.g1_pair(w, h, 200 + i) for i, (w, h) in enumerate(sizes)]
    kw = dict(patch=8, stride=4, levels=2, iters=8, variance=1, storage="u8")
    m = bd.BDIS(**kw)
    Ls = [torch.from_numpy(p.left).cuda() for p in pairs]
    Rs = [torch.from_numpy(p.right).cuda() for p in pairs]
    res = m.match_batched(Ls, Rs)
    torch.cuda.synchronize()
    for i in range(len(pairs)):
        one = bd.BDIS(**kw)
        d, v, ok = one.match(Ls[i], Rs[i])
        torch.cuda.synchronize()
        assert torch.equal(ok, res[i][2])
        assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(res[i][0], nan=-1.0))
        one.close()
    m.close()


def test_surgical_like_small(bd):
    pair = synth.g2_pair(320, 240, 5)
    _check_pair(bd, dict(patch=12, stride=6, levels=3, iters=8, variance=1), pair)


def test_textureless_image_is_all_invalid(bd):
    flat = np.full((64, 96), 90, np.uint8)
    g = _run(bd, dict(patch=8, stride=4, levels=2), flat, flat)
    assert not g["valid"].any()
    assert np.isnan(g["disp"]).all()
    assert np.all(g["levels"][0]["patches"]["flags"] & 1)


def test_integer_shift_exact(bd):
    pair = synth.shift_pair(160, 120, 1, 4)
    g = _run(bd, dict(patch=8, stride=4, levels=3, iters=8), pair.left, pair.right, views=False)
    inner = (slice(None), slice(4 + 8, 160 - 8))
    v = g["valid"][inner].astype(bool)
    assert v.mean() > 0.99
    assert np.max(np.abs(g["disp"][inner][v] - 4.0)) < 1e-5


def test_full_hd_f16_workload(bd):
    pair = synth.config_pair("plain_1920x1080_f16")
    kw = dict(patch=12, stride=4, levels=6, iters=8, variance=1, storage="f16")
    m = {}
    g, o, _ = _check_pair(bd, kw, pair, m)
    print("1920x1080 f16", m)
    # error of the fp16-stored GPU path against an unquantised FP64 oracle,
    # reported per output (not gated)
    o64 = oracle.match(oracle_params(g["params"], storage_override="f64"), pair.left, pair.right)
    both = o64["valid"] & g["valid"].astype(bool)
    dd = np.abs(g["disp"][both] - o64["disp"][both])
    print("vs unquantised fp64: disp median %.2e p99.9 %.2e; valid mismatch %d" %
          (np.median(dd), np.percentile(dd, 99.9), int((o64["valid"] != g["valid"].astype(bool)).sum())))


def test_batched_equals_plain(bd):
    import torch
    sizes = [(160, 120), (97, 61), (256, 144), (160, 120)]
    pairs = [synth.g1_pair(w, h, 100 + i) for i, (w, h) in enumerate(sizes)]
    kw = dict(patch=8, stride=4, levels=2, iters=8, variance=1)
    m = bd.BDIS(**kw)
    Ls = [torch.from_numpy(p.left).cuda() for p in pairs]
    Rs = [torch.from_numpy(p.right).cuda() for p in pairs]
    res = m.match_batched(Ls, Rs)
    torch.cuda.synchronize()
    for i, p in enumerate(pairs):
        d, v, ok = m.match(Ls[i], Rs[i])
        torch.cuda.synchronize()
        assert torch.equal(ok, res[i][2])
        assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(res[i][0], nan=-1.0))
        assert torch.equal(torch.nan_to_num(v, nan=-1.0), torch.nan_to_num(res[i][1], nan=-1.0))


def test_host_api_equals_device_api(bd):
    import torch
    pair = synth.config_pair("plain_320x240")
    m = bd.BDIS(patch=8, stride=4, levels=3, variance=1)
    d, v, ok = m.match(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda())
    torch.cuda.synchronize()
    hd, hv, hok = m.match_host(pair.left, pair.right)
    assert np.array_equal(hok, ok.cpu().numpy())
    assert np.array_equal(np.nan_to_num(hd, nan=-1), np.nan_to_num(d.cpu().numpy(), nan=-1))
    assert np.array_equal(np.nan_to_num(hv, nan=-1), np.nan_to_num(v.cpu().numpy(), nan=-1))


@pytest.mark.parametrize("mapped", [1, 0])
def test_pinned_host_buffers_equal_device_api(bd, mapped):
    """Page-locked host buffers: read and written in place by the kernels
    (mapped) or through staging copies; bitwise equal to the device API."""
    import ctypes as C
    import torch
    pair = synth.config_pair("plain_640x480_var")
    h, w = pair.left.shape
    m = bd.BDIS(patch=12, stride=6, levels=4, iters=8, variance=1)
    m.set_option(bd.B.OPT_HOST_MAPPED, mapped)
    d, v, ok = m.match(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda())
    torch.cuda.synchronize()
    hL = torch.from_numpy(pair.left).pin_memory()
    hR = torch.from_numpy(pair.right).pin_memory()
    hD = torch.full((h, w), 7.0).pin_memory()
    hV = torch.full((h, w), 7.0).pin_memory()
    hM = torch.full((h, w), 7, dtype=torch.uint8).pin_memory()
    stream = torch.cuda.Stream()
    for _ in range(2):   # first call tunes, second replays
        m.match_host_ptr(hL.data_ptr(), hR.data_ptr(), w, h, hD.data_ptr(), hV.data_ptr(),
                         hM.data_ptr(), C.c_void_p(stream.cuda_stream))
    assert torch.equal(hM, ok.cpu())
    assert torch.equal(torch.nan_to_num(hD, nan=-1.0), torch.nan_to_num(d.cpu(), nan=-1.0))
    assert torch.equal(torch.nan_to_num(hV, nan=-1.0), torch.nan_to_num(v.cpu(), nan=-1.0))
    m.close()


def test_stats_and_pitched_input(bd):
    import torch
    pair = synth.config_pair("plain_320x240")
    m = bd.BDIS(patch=8, stride=4, levels=3)
    # a pitched view: rows of 384 bytes, image 320 wide
    bigL = torch.zeros((240, 384), dtype=torch.uint8, device="cuda")
    bigR = torch.zeros((240, 384), dtype=torch.uint8, device="cuda")
    bigL[:, :320] = torch.from_numpy(pair.left).cuda()
    bigR[:, :320] = torch.from_numpy(pair.right).cuda()
    d1, _, ok1 = m.match(bigL[:, :320], bigR[:, :320])
    s = m.stats()
    d2, _, ok2 = m.match(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda())
    torch.cuda.synchronize()
    assert torch.equal(ok1, ok2)
    assert torch.equal(torch.nan_to_num(d1, nan=-1.0), torch.nan_to_num(d2, nan=-1.0))
    assert s["patches"] == [4661, 1131, 266]
    assert s["valid_pixels"] == int(ok1.sum().item())
    assert all(sr >= 0.5 for sr in s["sigma_r"])


@pytest.mark.parametrize("kw,size", [
    (dict(patch=12, stride=6, levels=4, iters=8, variance=1), (640, 480)),
    (dict(patch=8, stride=4, levels=3, iters=8, storage="f16"), (320, 240)),
    (dict(patch=16, stride=8, levels=2, iters=6, variance=1), (200, 150)),
    (dict(patch=10, stride=4, levels=6, iters=12, finest_level=1, variance=1), (640, 480)),
    (dict(patch=8, stride=4, levels=3, iters=8, weight_mode="dis", fast_exp=1), (320, 240)),
])
def test_persistent_form_equals_launch_sequence(bd, kw, size):
    import torch
    w, h = size
    pair = synth.g2_pair(w, h, 9) if kw.get("variance") else synth.g1_pair(w, h, 9)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    outs = []
    for form in (1, 2):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, form)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            d, v, ok = m.match(L, R, stream=stream)
            d2, v2, ok2 = m.match(L, R, stream=stream)   # a second call (graph / barrier reuse)
        torch.cuda.synchronize()
        st = m.stats()
        assert st["persistent"] == (1 if form == 2 else 0)
        assert st["barrier_timeouts"] == 0
        assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(d2, nan=-1.0))
        outs.append((d, v, ok))
        m.close()
    (d1, v1, o1), (d2, v2, o2) = outs
    assert torch.equal(o1, o2)
    assert torch.equal(torch.nan_to_num(d1, nan=-1.0), torch.nan_to_num(d2, nan=-1.0))
    if kw.get("variance"):
        assert torch.equal(torch.nan_to_num(v1, nan=-1.0), torch.nan_to_num(v2, nan=-1.0))


def test_persistent_form_after_batched_calls_on_one_handle(bd):
    """The persistent form's barrier words sit at a fixed place in the arena
    and are cleared before every cooperative launch, so plain and batched
    calls of any pair count can alternate on one handle."""
    import torch
    kw = dict(patch=8, stride=4, levels=3, iters=8)
    pairs = [synth.g1_pair(160 + 32 * i, 120, 40 + i) for i in range(4)]
    Ls = [torch.from_numpy(p.left).cuda() for p in pairs]
    Rs = [torch.from_numpy(p.right).cuda() for p in pairs]
    ref = bd.BDIS(**kw)
    ref.set_option(bd.B.OPT_FORM, 1)
    want = [ref.match(Ls[i], Rs[i]) for i in range(2)]
    torch.cuda.synchronize()
    m = bd.BDIS(**kw)
    m.set_option(bd.B.OPT_FORM, 2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        got0 = m.match(Ls[0], Rs[0], stream=stream)          # one pair
        m.match_batched(Ls, Rs, stream=stream)                # four pairs
        got1 = m.match(Ls[1], Rs[1], stream=stream)          # one pair again
    torch.cuda.synchronize()
    st = m.stats(stream)
    assert st["persistent"] == 1 and st["barrier_timeouts"] == 0
    m.set_option(bd.B.OPT_FORM, 1)
    with torch.cuda.stream(stream):
        m.match_batched(Ls, Rs, stream=stream)                # launch form, n = 4
        m.set_option(bd.B.OPT_FORM, 2)
        got0b = m.match(Ls[0], Rs[0], stream=stream)
    torch.cuda.synchronize()
    assert m.stats(stream)["barrier_timeouts"] == 0
    for (d, v, ok), (dw, vw, okw) in zip((got0, got1, got0b), (want[0], want[1], want[0])):
        assert torch.equal(ok, okw)
        assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(dw, nan=-1.0))
    m.close()
    ref.close()


@pytest.mark.parametrize("kw,size", [
    (dict(patch=12, stride=6, levels=4, iters=8, variance=1), (640, 480)),
    (dict(patch=8, stride=4, levels=3, iters=8, storage="f16"), (320, 240)),
    (dict(patch=10, stride=4, levels=6, iters=12, finest_level=1, variance=1), (640, 480)),
])
def test_coarse_levels_in_one_launch_equal_launch_sequence(bd, kw, size):
    """The k coarsest levels in one cooperative launch (grid barriers between
    their stages) give bitwise the outputs, records and images of one launch
    per stage, for every k, on graph replay too."""
    import torch
    w, h = size
    pair = synth.g2_pair(w, h, 13) if kw.get("variance") else synth.g1_pair(w, h, 13)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    nl = kw["levels"] - kw.get("finest_level", 0)
    ref = None
    for k in range(nl):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_COARSE_LEVELS, k)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            for _ in range(3):   # capture, then replays
                d, v, ok = m.match(L, R, stream=stream)
        torch.cuda.synchronize()
        st = m.stats(stream)
        assert st["persistent"] == (2 if k > 0 else 0) and st["barrier_timeouts"] == 0
        got = [torch.nan_to_num(d, nan=-1.0), ok] + ([torch.nan_to_num(v, nan=-1.0)] if v is not None else [])
        recs = [m.level_view(0, l)["patches"] for l in range(kw.get("finest_level", 0), kw["levels"])]
        if ref is None:
            ref, ref_recs = got, recs
        else:
            for a, b in zip(ref, got):
                assert torch.equal(a, b), k
            for a, b in zip(ref_recs, recs):
                assert a.tobytes() == b.tobytes(), k
        m.close()


def test_coarse_levels_in_one_launch_float_forward(bd):
    """The float-image (differentiable) forward in the same form, and its
    gradient, equal those of the launch sequence."""
    import torch
    pr = synth.g1_pair(320, 240, 17, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    L = torch.from_numpy(pr.left.astype(np.float32)).cuda()
    R = torch.from_numpy(pr.right.astype(np.float32)).cuda()
    outs = []
    for k in (0, 2):
        m = bd.BDIS(patch=8, stride=4, levels=3, iters=8)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_COARSE_LEVELS, k)
        (d, _, ok), = m.match_f32([L], [R])
        g, = m.loss_and_grad(0.1)
        torch.cuda.synchronize()
        outs.append((torch.nan_to_num(d, nan=-1.0), ok, g["loss"], g["g_disp"]))
        m.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_persistent_barrier_timeout_is_reported(bd):
    """Every grid-barrier wait of the persistent form is bounded.  A wait that
    runs out (forced here: with the test switch no arrival completes a
    barrier) lets the kernel finish, and the call is reported as failed by
    bdis_wait, by bdis_get_stats and by the next call on the handle; the
    context and the handle stay usable."""
    import ctypes as C
    import torch
    lib = bd.B.lib()
    kw = dict(patch=8, stride=4, levels=2, iters=8)
    pair = synth.g1_pair(160, 120, 5)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    ref = bd.BDIS(**kw)
    ref.set_option(bd.B.OPT_FORM, 1)
    dw, _, okw = ref.match(L, R)
    m = bd.BDIS(**kw)
    m.set_option(bd.B.OPT_FORM, 2)
    m.set_option(bd.B.OPT_BARRIER_LIMIT, 1024)
    stream = torch.cuda.Stream()
    sh = C.c_void_p(stream.cuda_stream)

    def call():
        d = torch.empty((120, 160), device="cuda")
        ok = torch.empty((120, 160), dtype=torch.uint8, device="cuda")
        rc = lib.bdis_match(m._h, L.data_ptr(), R.data_ptr(), 160, 120, 160, d.data_ptr(), None,
                            ok.data_ptr(), sh)
        return rc, d, ok

    m.set_option(bd.B.OPT_BARRIER_TEST, 1)
    rc, _, _ = call()
    assert rc == bd.B.BDIS_OK                       # asynchronous: not known yet
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_ECUDA
    assert b"grid-barrier" in lib.bdis_last_error(m._h)
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_OK  # reported once
    s = bd.B.bdis_stats()
    assert lib.bdis_get_stats(m._h, C.byref(s), sh) == bd.B.BDIS_OK
    assert s.persistent == 1 and s.barrier_timeouts == 1
    # the next call reports a timed-out call that nobody waited for
    rc, _, _ = call()
    assert rc == bd.B.BDIS_OK
    stream.synchronize()
    m.set_option(bd.B.OPT_BARRIER_TEST, 0)
    rc, _, _ = call()
    assert rc == bd.B.BDIS_ECUDA
    # and then the handle works normally again
    rc, d, ok = call()
    assert rc == bd.B.BDIS_OK
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_OK
    assert lib.bdis_get_stats(m._h, C.byref(s), sh) == bd.B.BDIS_OK
    assert s.barrier_timeouts == 0
    torch.cuda.synchronize()
    assert torch.equal(ok, okw)
    assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(dw, nan=-1.0))
    m.close()
    ref.close()


# ---------------------------------------------------------------- optional modes

MODE_CASES = {
    # Eq. 2 fusion weights instead of the sGMM x probability
    "dis_weights_320x240": ("plain_320x240", dict(patch=8, stride=4, levels=3, iters=8,
                                                  weight_mode="dis")),
    "dis_weights_640x480_var": ("plain_640x480_var", dict(patch=12, stride=6, levels=4, iters=8,
                                                          variance=1, weight_mode="dis")),
    # Schraudolph's exponential in the posterior
    "fast_exp_640x480_var": ("plain_640x480_var", dict(patch=12, stride=6, levels=4, iters=8,
                                                       variance=1, fast_exp=1)),
    # the paper's parameter set (Sec. IV-A): scales 2^5 .. 2^1, patch 10,
    # overlap 0.55 (stride 4), 12 iterations, then upsampling to full size
    "paper_preset_640x480_var": ("plain_640x480_var", dict(patch=10, stride=4, levels=6, iters=12,
                                                           finest_level=1, variance=1)),
}


@pytest.mark.parametrize("name", list(MODE_CASES))
def test_mode_parity(bd, name):
    cfg, kw = MODE_CASES[name]
    m = {}
    _check_pair(bd, kw, synth.config_pair(cfg), m)
    print(name, m)


@pytest.mark.parametrize("w,h,kw", [
    (203, 117, dict(patch=8, stride=4, levels=3, iters=8, finest_level=2)),
    (160, 120, dict(patch=6, stride=3, levels=3, iters=8, finest_level=1, weight_mode="dis",
                    storage="f16", variance=1)),
])
def test_mode_ragged_cases(bd, w, h, kw):
    _check_pair(bd, kw, synth.g1_pair(w, h, w + h))


def test_paper_preset_integer_shift(bd):
    pair = synth.shift_pair(320, 240, 3, 4)
    g = _run(bd, dict(patch=10, stride=4, levels=5, iters=12, finest_level=1), pair.left,
             pair.right, views=False)
    inner = (slice(8, 232), slice(4 + 24, 320 - 24))
    v = g["valid"][inner].astype(bool)
    assert v.mean() > 0.99
    assert np.max(np.abs(g["disp"][inner][v] - 4.0)) < 1e-5


def test_depth_kernel(bd):
    # bdis_depth (Eq. 13, Eq. 17) against the oracle's depth, element by element
    import torch
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 60.0, 100003).astype(np.float32)
    d[::7] = np.nan
    d[::11] = 0.0
    d[::13] = -1.0
    d[::17] = np.inf
    v = rng.uniform(0.0, 2.0, d.size).astype(np.float32)
    fb = 512.0 * 0.005
    z, zv = bd.depth(torch.from_numpy(d).cuda(), torch.from_numpy(v).cuda(), fb=fb)
    z, zv = z.cpu().numpy(), zv.cpu().numpy()
    zo, zvo = oracle.depth(d, v, fb)
    ok = np.isfinite(zo)
    assert np.array_equal(ok, np.isfinite(z)) and np.array_equal(ok, np.isfinite(zv))
    np.testing.assert_allclose(z[ok], zo[ok], rtol=1e-6)
    np.testing.assert_allclose(zv[ok], zvo[ok], rtol=1e-5)
    z2, none = bd.depth(torch.from_numpy(d).cuda(), None, fb=fb)
    assert none is None and np.array_equal(np.nan_to_num(z2.cpu().numpy(), nan=-1),
                                           np.nan_to_num(z, nan=-1))


def test_depth_of_a_match_against_the_oracle(bd):
    # the depth and depth variance of a real disparity / variance output
    import torch
    pair = synth.config_pair("plain_640x480_var", seed=3)
    m = bd.BDIS(patch=12, stride=6, levels=4, iters=8, variance=1)
    disp, var, ok = m.match(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda())
    z, zv = bd.depth(disp.reshape(-1), var.reshape(-1), fb=800.0 * 0.0055)
    torch.cuda.synchronize()
    dn, vn = disp.cpu().numpy().ravel(), var.cpu().numpy().ravel()
    zo, zvo = oracle.depth(dn, vn, 800.0 * 0.0055)
    z, zv = z.cpu().numpy(), zv.cpu().numpy()
    fin = np.isfinite(zo)
    assert fin.sum() > 0.25 * fin.size
    assert np.array_equal(fin, np.isfinite(z))
    np.testing.assert_allclose(z[fin], zo[fin], rtol=1e-6)
    np.testing.assert_allclose(zv[fin], zvo[fin], rtol=1e-5, atol=1e-30)
    m.close()


def test_modes_outside_the_adjoint_are_rejected(bd):
    import torch
    pr = synth.g1_pair(96, 64, 7, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    L = torch.from_numpy(pr.left.astype(np.float32)).cuda()
    R = torch.from_numpy(pr.right.astype(np.float32)).cuda()
    for kw in (dict(weight_mode="dis"), dict(finest_level=1), dict(fast_exp=1)):
        m = bd.BDIS(patch=8, stride=4, levels=2, iters=8, **kw)
        m.match_f32([L], [R])
        with pytest.raises(bd.BdisError) as e:
            m.loss_and_grad(0.1)
        assert e.value.status == bd.B.BDIS_EUNSUPPORTED
        m.close()


def test_u8_storage_outside_the_cooperative_forms(bd):
    # 8-bit pyramids have no persistent or coarse-level cooperative form: those
    # options fall back to the launch sequence; the allocation-free entry
    # point rejects them
    import ctypes as C
    import torch
    pair = synth.g1_pair(160, 120, 8)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    ref = bd.BDIS(patch=8, stride=4, levels=3, storage="u8")
    d0, _, ok0 = ref.match(L, R)
    for opt, val in ((bd.B.OPT_FORM, 2), (bd.B.OPT_COARSE_LEVELS, 2)):
        m = bd.BDIS(patch=8, stride=4, levels=3, storage="u8")
        if opt == bd.B.OPT_COARSE_LEVELS:
            m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(opt, val)
        d, _, ok = m.match(L, R)
        torch.cuda.synchronize()
        assert m.stats()["persistent"] == 0
        assert torch.equal(ok, ok0)
        assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(d0, nan=-1.0))
        m.close()
    p = bd._params(patch=8, stride=4, levels=3, storage="u8")
    out = torch.empty((120, 160), device="cuda")
    okb = torch.empty((120, 160), dtype=torch.uint8, device="cuda")
    rc = bd.B.lib().bdis_match_noalloc(C.byref(p), L.data_ptr(), R.data_ptr(), 160, 120, 160,
                                        out.data_ptr(), None, okb.data_ptr(), None)
    assert rc == bd.B.BDIS_EUNSUPPORTED
    ref.close()


def test_noalloc_rejects_finest_level(bd):
    import ctypes as C
    import torch
    p = bd._params(patch=8, stride=4, levels=3, finest_level=1)
    L = torch.zeros((120, 160), dtype=torch.uint8, device="cuda")
    d = torch.empty((120, 160), device="cuda")
    ok = torch.empty((120, 160), dtype=torch.uint8, device="cuda")
    rc = bd.B.lib().bdis_match_noalloc(C.byref(p), L.data_ptr(), L.data_ptr(), 160, 120, 160,
                                        d.data_ptr(), None, ok.data_ptr(), None)
    assert rc == bd.B.BDIS_EUNSUPPORTED


@pytest.mark.parametrize("kw", [
    dict(patch=12, stride=6, levels=4, iters=8, variance=1),
    dict(patch=10, stride=4, levels=6, iters=12, finest_level=1, variance=1),
])
def test_launch_options_do_not_change_results(bd, kw):
    """Programmatic dependent launch, graph replay and one or two pyramid
    steps per launch change only how the work is issued: outputs are bitwise
    equal with every combination."""
    import torch
    pair = synth.g2_pair(640, 480, 11)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    ref = None
    for graph, pdl, steps in ((0, 0, 1), (0, 1, 2), (1, 0, 2), (1, 1, 1), (1, 1, 2)):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_GRAPH, graph)
        m.set_option(bd.B.OPT_PDL, pdl)
        m.set_option(bd.B.OPT_PYRAMID_STEPS, steps)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            for _ in range(3):   # capture, then replays
                d, v, ok = m.match(L, R, stream=stream)
        torch.cuda.synchronize()
        got = (torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(v, nan=-1.0), ok)
        # every level's images and gradient as well (the two-step pyramid
        # computes the next level and its gradient from a recomputed halo)
        views = [m.level_view(0, l) for l in range(kw["levels"])]
        imgs = [np.nan_to_num(vw[key], nan=-1.0) for vw in views for key in ("L", "R", "G")
                if vw.get(key) is not None]
        if ref is None:
            ref = got
            ref_imgs = imgs
        else:
            for a, b in zip(ref, got):
                assert torch.equal(a, b), (graph, pdl, steps)
            assert len(imgs) == len(ref_imgs)
            for a, b in zip(ref_imgs, imgs):
                assert np.array_equal(a, b), (graph, pdl, steps)
        m.close()


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_bulk_copy_staging_equals_own_loads(bd, storage):
    """The one-step pyramid's bulk asynchronous staging of interior tiles
    gives bitwise the images, gradients and outputs of staging by the block's
    own loads, on pairs whose tiles are partly ineligible (odd sizes, a row
    pitch that is not a multiple of 16 bytes)."""
    import torch
    sizes = [(640, 480, 640), (333, 217, 333), (1280, 720, 1296), (250, 130, 257)]
    pairs = [synth.g1_pair(w, h, 50 + i) for i, (w, h, _) in enumerate(sizes)]
    Ls, Rs = [], []
    for (w, h, pitch), p in zip(sizes, pairs):
        for img, lst in ((p.left, Ls), (p.right, Rs)):
            buf = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
            buf[:, :w] = torch.from_numpy(img).cuda()
            lst.append(buf[:, :w])
    kw = dict(patch=8, stride=4, levels=3, iters=8, storage=storage)
    res = []
    for bulk in (0, 1):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_PYRAMID_STEPS, 1)
        m.set_option(bd.B.OPT_BULK_COPY, bulk)
        out = m.match_batched(Ls, Rs)
        torch.cuda.synchronize()
        views = [m.level_view(i, l) for i in range(len(sizes)) for l in range(3)]
        res.append((out, views))
        m.close()
    (o0, v0), (o1, v1) = res
    for (d0, _, k0), (d1, _, k1) in zip(o0, o1):
        assert torch.equal(k0, k1)
        assert torch.equal(torch.nan_to_num(d0, nan=-1.0), torch.nan_to_num(d1, nan=-1.0))
    for a, b in zip(v0, v1):
        for key in ("L", "R", "G"):
            if a.get(key) is not None:
                assert np.array_equal(a[key], b[key]), key



@pytest.mark.parametrize("patch,storage", [(8, "f16"), (8, "u8"), (12, "f32"), (12, "f16")])
def test_bulk_search_band_equals_own_loads(bd, patch, storage):
    """The search's bulk asynchronous staging of the right-image band
    (BDIS_OPT_BULK_COPY bit 2) gives bitwise the records and outputs of
    staging by the block's own loads, on pairs where some bands are
    ineligible (near the image edges, odd widths, row pitches that are not a
    multiple of 16 bytes), alone and together with the pyramid's (value 3)."""
    import torch
    sizes = [(640, 480, 640), (333, 217, 333), (1280, 720, 1296), (250, 130, 257)]
    pairs = [synth.g1_pair(w, h, 70 + i) for i, (w, h, _) in enumerate(sizes)]
    Ls, Rs = [], []
    for (w, h, pitch), p in zip(sizes, pairs):
        for img, lst in ((p.left, Ls), (p.right, Rs)):
            buf = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
            buf[:, :w] = torch.from_numpy(img).cuda()
            lst.append(buf[:, :w])
    kw = dict(patch=patch, stride=patch // 2, levels=3, iters=8, storage=storage, variance=1)
    res = []
    for bulk in (0, 2, 3):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_BULK_COPY, bulk)
        out = m.match_batched(Ls, Rs)
        torch.cuda.synchronize()
        views = [m.level_view(i, l) for i in range(len(sizes)) for l in range(3)]
        one = m.match(Ls[0], Rs[0])
        torch.cuda.synchronize()
        assert m.stats()["barrier_timeouts"] == 0
        res.append((out + [one], views))
        m.close()
    (o0, v0) = res[0]
    for o1, v1 in res[1:]:
        for (d0, q0, k0), (d1, q1, k1) in zip(o0, o1):
            assert torch.equal(k0, k1)
            assert torch.equal(torch.nan_to_num(d0, nan=-1.0), torch.nan_to_num(d1, nan=-1.0))
            assert torch.equal(torch.nan_to_num(q0, nan=-1.0), torch.nan_to_num(q1, nan=-1.0))
        for a, b in zip(v0, v1):
            assert np.array_equal(a["patches"].view(np.uint8), b["patches"].view(np.uint8))



@pytest.mark.parametrize("kw,size", [
    (dict(patch=12, stride=6, levels=3, iters=8, variance=1, storage="f32"), (333, 217)),
    (dict(patch=8, stride=4, levels=3, iters=8, variance=0, storage="f16"), (641, 359)),
    (dict(patch=10, stride=1, levels=2, iters=6, variance=1, storage="f32"), (163, 97)),
])
def test_search_chunking_does_not_change_results(bd, kw, size):
    """Every search chunking (BDIS_OPT_SEARCH_PASSES 1..4 passes of the
    block's lane groups, so 16 to 128 patches per block) and every fusion
    tile (BDIS_OPT_FUSE_TILE 32x16, 64x32, 64x64) gives bitwise the same
    records and outputs: the patches are independent, the sigma_r sums are
    exact integers and each pixel's fusion sums run in the same order.  The stride-1 case puts the groups of a warp 16
    patches apart, which a 3-pass chunk must still cover exactly once."""
    import torch
    w, h = size
    p = synth.g1_pair(w, h, 91)
    L = torch.from_numpy(p.left).cuda()
    R = torch.from_numpy(p.right).cuda()
    res = []
    for passes, tile in ((1, 1), (2, 2), (3, 3), (4, 1), (2, 3)):
        m = bd.BDIS(**kw)
        m.set_option(bd.B.OPT_FORM, 1)
        m.set_option(bd.B.OPT_SEARCH_PASSES, passes)
        m.set_option(bd.B.OPT_FUSE_TILE, tile)
        d, v, k = m.match(L, R)
        torch.cuda.synchronize()
        views = [m.level_view(0, l) for l in range(kw["levels"])]
        res.append(((d, v, k), views))
        m.close()
    (d0, v0, k0), w0 = res[0]
    for (d1, v1, k1), w1 in res[1:]:
        assert torch.equal(k0, k1)
        assert torch.equal(torch.nan_to_num(d0, nan=-1.0), torch.nan_to_num(d1, nan=-1.0))
        if v0 is not None:
            assert torch.equal(torch.nan_to_num(v0, nan=-1.0), torch.nan_to_num(v1, nan=-1.0))
        for a, b in zip(w0, w1):
            assert np.array_equal(a["patches"].view(np.uint8), b["patches"].view(np.uint8))
            assert a["sigma_r"] == b["sigma_r"]



def test_bulk_copy_wait_timeout_is_reported(bd):
    """Every wait for bulk asynchronous copies (the one-step pyramid's tiles
    and the search's bands) is bounded.  A wait that runs out (forced here:
    with the test switch each wait expects 16 bytes that no copy delivers)
    stops the block after its copies have landed, and the call is reported
    as failed by bdis_wait; the handle then works normally again, with the
    outputs of a handle that never used the copies."""
    import ctypes as C
    import torch
    lib = bd.B.lib()
    kw = dict(patch=8, stride=4, levels=3, iters=8, storage="f16")
    pair = synth.g1_pair(640, 480, 6)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    ref = bd.BDIS(**kw)
    ref.set_option(bd.B.OPT_FORM, 1)
    dw, _, okw = ref.match(L, R)
    torch.cuda.synchronize()
    m = bd.BDIS(**kw)
    for opt, val in ((bd.B.OPT_FORM, 1), (bd.B.OPT_AUTOTUNE, 0), (bd.B.OPT_PYRAMID_STEPS, 1),
                     (bd.B.OPT_BULK_COPY, 3), (bd.B.OPT_BARRIER_LIMIT, 4096)):
        m.set_option(opt, val)
    stream = torch.cuda.Stream()
    sh = C.c_void_p(stream.cuda_stream)
    d = torch.empty((480, 640), device="cuda")
    ok = torch.empty((480, 640), dtype=torch.uint8, device="cuda")

    def call():
        return lib.bdis_match(m._h, L.data_ptr(), R.data_ptr(), 640, 480, 640, d.data_ptr(), None,
                              ok.data_ptr(), sh)

    m.set_option(bd.B.OPT_BARRIER_TEST, 1)
    assert call() == bd.B.BDIS_OK                    # asynchronous: not known yet
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_ECUDA
    assert b"bulk copy" in lib.bdis_last_error(m._h)
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_OK   # reported once
    m.set_option(bd.B.OPT_BARRIER_TEST, 0)
    assert call() == bd.B.BDIS_OK
    assert lib.bdis_wait(m._h, sh) == bd.B.BDIS_OK
    assert torch.equal(ok, okw)
    assert torch.equal(torch.nan_to_num(d, nan=-1.0), torch.nan_to_num(dw, nan=-1.0))
    m.close()
    ref.close()


def _coverage(disp, var, valid, gt, z=1.96):
    v = valid.astype(bool) & np.isfinite(var) & (var > 0)
    e = np.abs(disp[v].astype(np.float64) - gt[v])
    return float((e <= z * np.sqrt(var[v])).mean()), int(v.sum())


@pytest.mark.parametrize("gen,kw", [
    ("g1", dict(patch=8, stride=4, levels=3, iters=8, variance=1)),
    ("g2", dict(patch=12, stride=6, levels=3, iters=8, variance=1)),
    ("g1", dict(patch=10, stride=4, levels=4, iters=12, variance=1, finest_level=1)),
])
def test_variance_coverage_matches_oracle(bd, gen, kw):
    """The synthetic coverage experiment (|e| <= 1.96 sigma against the known
    ground truth) gives the same fraction from the GPU outputs as from the oracle's."""
    pr = synth.g1_pair(320, 240, 0) if gen == "g1" else synth.g2_pair(320, 240, 5)
    g = _run(bd, kw, pr.left, pr.right, views=False)
    o = oracle.match(oracle_params(g["params"]), pr.left, pr.right)
    gt = pr.gt_left()
    cg, ng = _coverage(g["disp"], g["var"], g["valid"], gt)
    co, no = _coverage(o["disp"], o["var"], o["valid"], gt)
    assert abs(ng - no) <= max(2, 0.001 * no)
    assert abs(cg - co) <= 1e-3, (cg, co)
    assert 0.5 < co <= 1.0


def test_largest_workload_4k_f16(bd):
    """3840x2160 (HD generator, disparities to 160 px), 12x12 patches at stride
    4, 6 levels, variance, FP16 pyramids: the largest single pair tested."""
    pair = synth.g1_pair(3840, 2160, 2, d0=10.0, d1=140.0, amp=20.0, sigma=240.0)
    m = {}
    _check_pair(bd, dict(patch=12, stride=4, levels=6, iters=8, variance=1, storage="f16"), pair, m)
    print("3840x2160 f16", m)
