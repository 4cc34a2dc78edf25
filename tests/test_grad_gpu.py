"""GPU adjoint of the differentiable finest level against the oracle's
analytic gradient (itself pinned to FP64 central differences on CPU), on the
same seeded float images, through the C ABI.

Tolerance: per element |g_gpu - g_oracle| <= 1e-4 * max|g_oracle| (+ a
FP32 floor).  The L1 terms of the loss have kinks (the sign of a residual,
or of a disparity difference at the tie threshold), where FP32 and FP64 can
take different sides at a handful of pixels.  The small cases therefore
compare the adjoint chain of both sides from the same dL/dD (the GPU's) on
every element, dL/dD itself away from kink-adjacent pixels, and the complete
gradients on most elements; at 640x480 the complete gradients are compared
on >= 99.9 % of the elements."""
import numpy as np
import pytest

import oracle
import synth
from parity import oracle_params

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def bd():
    import paper_2205_03133_gb300 as bd
    from paper_2205_03133_gb300 import build
    build.build()
    return bd


def _gpu(bd, kw, L32, R32, lam=0.1):
    import torch
    m = bd.BDIS(**kw)
    Lt = torch.from_numpy(L32).cuda()
    Rt = torch.from_numpy(R32).cuda()
    (d, v, ok), = m.match_f32([Lt], [Rt])
    g, = m.loss_and_grad(lam)
    torch.cuda.synchronize()
    rec = m.level_view(0, 0)["patches"]
    out = {k: t.cpu().numpy() for k, t in g.items()}
    out.update(disp=d.cpu().numpy(), valid=ok.cpu().numpy().astype(bool), rec=rec, params=m.params)
    m.close()
    return out


def _oracle(gp, L, R, lam=0.1):
    op = oracle_params(gp)
    o = oracle.match(op, L, R, trace=True)
    st = oracle.frozen_state(op, o)
    loss, gL, gR, gdk, gD = oracle.diff_grad(op, L, R, st, lam)
    return dict(loss=loss, g_left=gL, g_right=gR, g_patch=gdk, g_disp=gD, out=o, st=st)


def _kink_pixels(D, valid, L, R, lam_tie=1e-6, band=5e-6, rband=1e-4):
    """Pixels whose loss subgradient the two arithmetics may legitimately
    take on different sides: a reprojection residual within rband of 0, or a
    4-neighbour disparity difference within band of the tie threshold
    lam_tie (|D_p| + |D_q|) (reading r25).  FP32 rounding moves D by ~1e-6 px.
    Structural ties (differences that vanish in exact arithmetic, ~1e-15 in
    FP64) stay ties on both sides and are not kinks here."""
    h, w = D.shape
    out = np.zeros((h, w), bool)
    X = np.clip(np.arange(w)[None, :] - np.nan_to_num(D), 0, w - 1)
    x0 = np.floor(X).astype(int)
    x1 = np.minimum(x0 + 1, w - 1)
    t = X - x0
    rows = np.arange(h)[:, None]
    r = (1 - t) * R[rows, x0] + t * R[rows, x1] - L
    out |= valid & (np.abs(r) < rband)
    for dy, dx in ((0, 1), (1, 0)):
        a, b = D[: h - dy, : w - dx], D[dy:, dx:]
        both = valid[: h - dy, : w - dx] & valid[dy:, dx:]
        diff, thr = np.abs(a - b), lam_tie * (np.abs(a) + np.abs(b))
        near = both & (diff > 1e-9) & (np.abs(diff - thr) < band)
        out[: h - dy, : w - dx] |= near
        out[dy:, dx:] |= near
    return out


def _close(a, b, frac=1.0):
    scale = np.abs(b).max()
    err = np.abs(a.astype(np.float64) - b)
    ok = err <= REL * scale + 1e-9
    return ok.mean() >= frac, dict(frac_ok=float(ok.mean()), max_rel=float(err.max() / scale))


@pytest.mark.parametrize("kw", [
    dict(patch=8, stride=4, levels=3, iters=50),
    dict(patch=8, stride=4, levels=3, iters=50, sigma_r_mode="fixed"),
    dict(patch=12, stride=4, levels=2, iters=50, use_sgmm=0),
    # a window step other than 1/2 takes the general (per-offset split) adjoint
    dict(patch=8, stride=4, levels=2, iters=50, window_step=0.4),
])
def test_adjoint_matches_oracle_small(bd, kw):
    """Every element: the adjoint chain of both sides from the same dL/dD
    (the GPU's), and dL/dD itself away from the kinks of the L1 terms; the
    complete gradients agree on all but the kink-adjacent elements."""
    import torch
    pr = synth.g1_pair(64, 48, 3, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    L32, R32 = pr.left.astype(np.float32), pr.right.astype(np.float32)
    L, R = L32.astype(np.float64), R32.astype(np.float64)
    m = bd.BDIS(**kw)
    (d, _, ok), = m.match_f32([torch.from_numpy(L32).cuda()], [torch.from_numpy(R32).cuda()])
    g, = m.loss_and_grad(0.1)
    (aL, aR, adk), = m.backward([g["g_disp"]])     # the adjoint chain alone
    torch.cuda.synchronize()
    rec = m.level_view(0, 0)["patches"]
    gp = m.params
    g = {k: t.cpu().numpy() for k, t in g.items()}
    aL, aR, adk = aL.cpu().numpy(), aR.cpu().numpy(), adk.cpu().numpy()
    valid = ok.cpu().numpy().astype(bool)
    m.close()
    o = _oracle(gp, L, R)
    # same discrete state on both sides
    assert np.array_equal(valid, o["out"]["valid"])
    kept = o["st"]["kept"].astype(bool)
    assert np.array_equal(rec["flags"].ravel() == 0, kept)
    assert abs(float(g["loss"][0]) - o["loss"]) <= 1e-5 * o["loss"]
    oL, oR, odk = oracle.diff_adjoint(oracle_params(gp), L, R, o["st"], g["g_disp"])
    for key, a, b in (("adjoint g_left", aL, oL), ("adjoint g_right", aR, oR)):
        good, info = _close(a, b)
        assert good, (key, info)
    good, info = _close(adk.ravel()[kept], odk[kept])
    assert good, ("adjoint g_patch_disp", info)
    kinks = _kink_pixels(o["out"]["disp"], valid, L, R)
    assert kinks.mean() < 0.02, kinks.mean()
    good, info = _close(g["g_disp"][~kinks], o["g_disp"][~kinks])
    assert good, ("g_disp away from kinks", info, int(kinks.sum()))
    # the complete gradients: a kink pixel that the two sides take on
    # different sides reaches every element of the patches covering it (8x8
    # or larger, through their solves), a few hundred of the 3072 here
    for key in ("g_left", "g_right"):
        good, info = _close(g[key], o[key], frac=0.85)
        assert good, (key, info)


def test_adjoint_matches_oracle_640x480(bd):
    # a pair of the 16-pair differentiable workload: 640x480 G1, 8x8 patches,
    # stride 4, 3 levels, 8 Gauss-Newton iterations
    pr = synth.g1_pair(640, 480, 0)
    L32, R32 = pr.left.astype(np.float32), pr.right.astype(np.float32)
    kw = dict(patch=8, stride=4, levels=3, iters=8)
    g = _gpu(bd, kw, L32, R32)
    o = _oracle(g["params"], L32.astype(np.float64), R32.astype(np.float64))
    kept_g = g["rec"]["flags"].ravel() == 0
    kept_o = o["st"]["kept"].astype(bool)
    flips = int((kept_g != kept_o).sum())
    assert flips <= max(2, int(0.001 * kept_o.size))
    assert abs(float(g["loss"][0]) - o["loss"]) <= 1e-4 * o["loss"]
    for key in ("g_left", "g_right", "g_disp"):
        good, info = _close(g[key], o[key], frac=0.999)
        print(key, info, "flips", flips)
        assert good, (key, info)


def test_batched_backward_equals_per_pair(bd):
    import torch
    kw = dict(patch=8, stride=4, levels=2, iters=8)
    pairs = [synth.g1_pair(w, h, 40 + i, d0=1.0, d1=3.0, amp=1.0, as_float=True)
             for i, (w, h) in enumerate([(96, 64), (128, 80), (96, 64)])]
    Ls = [torch.from_numpy(p.left.astype(np.float32)).cuda() for p in pairs]
    Rs = [torch.from_numpy(p.right.astype(np.float32)).cuda() for p in pairs]
    m = bd.BDIS(**kw)
    m.match_f32(Ls, Rs)
    gb = m.loss_and_grad(0.1)
    torch.cuda.synchronize()
    gb = [{k: t.cpu().numpy() for k, t in g.items()} for g in gb]
    for i in range(3):
        m.match_f32([Ls[i]], [Rs[i]])
        g1, = m.loss_and_grad(0.1)
        torch.cuda.synchronize()
        for k in ("loss", "g_disp", "g_patch_disp"):
            np.testing.assert_allclose(g1[k].cpu().numpy(), gb[i][k], rtol=1e-5, atol=1e-9)
        for k in ("g_left", "g_right"):   # atomics: order of accumulation may differ
            a, b = g1[k].cpu().numpy(), gb[i][k]
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_autograd_function(bd):
    import torch
    pr = synth.g1_pair(96, 64, 7, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    L = torch.from_numpy(pr.left.astype(np.float32)).cuda().requires_grad_(True)
    R = torch.from_numpy(pr.right.astype(np.float32)).cuda().requires_grad_(True)
    m = bd.BDIS(patch=8, stride=4, levels=2, iters=30)
    d, valid = bd.disparity(m, L, R)
    w = torch.linspace(0, 1, d.shape[1], device=d.device)[None, :].expand_as(d)
    loss = (torch.nan_to_num(d, nan=0.0) * w).sum()
    loss.backward()
    # the same gradient from the C ABI with dL/dD = w on valid pixels
    m2 = bd.BDIS(patch=8, stride=4, levels=2, iters=30)
    m2.match_f32([L.detach()], [R.detach()])
    (gl, gr, _), = m2.backward([torch.where(valid.bool(), w, torch.zeros_like(w))])
    torch.cuda.synchronize()
    assert torch.allclose(L.grad, gl, rtol=1e-4, atol=1e-6 * gl.abs().max().item())
    assert torch.allclose(R.grad, gr, rtol=1e-4, atol=1e-6 * gr.abs().max().item())
    assert L.grad.abs().sum() > 0 and R.grad.abs().sum() > 0


def test_two_forwards_then_backward_of_the_first(bd):
    """Each disparity() forward keeps its state in its own caller-owned saved
    state (bdis_saved), held by the autograd graph: after a second forward on
    the same model, the first graph's backward still gives the first
    forward's gradient, equal to that of a lone forward on a fresh model."""
    import torch

    def leaf(a):
        return torch.from_numpy(a.astype(np.float32)).cuda().requires_grad_(True)

    prs = [synth.g1_pair(96, 64, 7, d0=1.0, d1=3.0, amp=1.0, as_float=True),
           synth.g1_pair(96, 64, 8, d0=1.5, d1=2.5, amp=1.0, as_float=True)]
    kw = dict(patch=8, stride=4, levels=2, iters=30)
    w = torch.linspace(0, 1, 96, device="cuda")[None, :].expand(64, 96)
    m = bd.BDIS(**kw)
    xs = [(leaf(p.left), leaf(p.right)) for p in prs]
    outs = [bd.disparity(m, L, R) for L, R in xs]       # two forwards, one model
    (torch.nan_to_num(outs[0][0], nan=0.0) * w).sum().backward()
    (torch.nan_to_num(outs[1][0], nan=0.0) * w).sum().backward()
    for (L, R), p in zip(xs, prs):
        m1 = bd.BDIS(**kw)
        L1, R1 = leaf(p.left), leaf(p.right)
        d1, _ = bd.disparity(m1, L1, R1)
        (torch.nan_to_num(d1, nan=0.0) * w).sum().backward()
        torch.cuda.synchronize()
        for a, b in ((L.grad, L1.grad), (R.grad, R1.grad)):
            assert b.abs().sum() > 0
            assert (a - b).abs().max().item() <= 1e-5 * b.abs().max().item()
        m1.close()
    m.close()


def test_saved_states_through_the_c_abi(bd):
    """bdis_match_batched_f32_saved keeps each forward in its own bdis_saved;
    bdis_loss / bdis_backward differentiate the one they are given (NULL:
    the handle's last call); a state of another handle is rejected."""
    import ctypes as C
    import torch
    lib = bd.B.lib()
    prs = [synth.g1_pair(96, 64, 11 + i, d0=1.0, d1=3.0, amp=1.0, as_float=True) for i in range(2)]
    ims = [(torch.from_numpy(p.left.astype(np.float32)).cuda(),
            torch.from_numpy(p.right.astype(np.float32)).cuda()) for p in prs]
    kw = dict(patch=8, stride=4, levels=2, iters=30)
    m = bd.BDIS(**kw)
    s1, s2 = m.saved_state(), m.saved_state()
    m.match_f32([ims[0][0]], [ims[0][1]], saved=s1)
    m.match_f32([ims[1][0]], [ims[1][1]], saved=s2)
    m.match_f32([ims[1][0]], [ims[0][1]])                  # a third forward, into the handle
    g1, = m.loss_and_grad(0.1, saved=s1)
    g2, = m.loss_and_grad(0.1, saved=s2)
    g3, = m.loss_and_grad(0.1)
    torch.cuda.synchronize()
    for g, (L, R) in zip((g1, g2, g3), (ims[0], ims[1], (ims[1][0], ims[0][1]))):
        ref = bd.BDIS(**kw)
        ref.match_f32([L], [R])
        gr, = ref.loss_and_grad(0.1)
        torch.cuda.synchronize()
        assert torch.equal(g["loss"], gr["loss"]) and torch.equal(g["g_disp"], gr["g_disp"])
        # sums reduced across blocks (the sigma_r chain) and float atomics
        # (image gradients): the last bits may differ from run to run
        for k in ("g_patch_disp", "g_left", "g_right"):
            assert (g[k] - gr[k]).abs().max() <= 1e-6 * gr[k].abs().max(), k
        ref.close()
    other = bd.BDIS(**kw)
    arr = bd._grad_table(m, [g1])
    rc = lib.bdis_backward(other._h, s1.handle, arr, None)
    assert rc == bd.B.BDIS_EINVAL
    empty = m.saved_state()
    assert lib.bdis_backward(m._h, empty.handle, arr, None) == bd.B.BDIS_EINVAL
    for sv in (s1, s2, empty):
        sv.destroy()
    other.close()
    m.close()


# ---------------------------------------------------------------- through every level

def _gpu_ml(bd, kw, L32, R32, lam=0.1):
    import torch
    m = bd.BDIS(**kw)
    m.set_option(bd.B.OPT_ADJOINT_LEVELS, 1)
    Lt = torch.from_numpy(L32).cuda()
    Rt = torch.from_numpy(R32).cuda()
    (d, v, ok), = m.match_f32([Lt], [Rt])
    g, = m.loss_and_grad(lam)
    (aL, aR, adk), = m.backward([g["g_disp"]])   # the adjoint chain alone
    torch.cuda.synchronize()
    recs = [m.level_view(0, l)["patches"] for l in range(m.params.levels)]
    out = {k: t.cpu().numpy() for k, t in g.items()}
    out["adjoint_g_left"], out["adjoint_g_right"] = aL.cpu().numpy(), aR.cpu().numpy()
    out["adjoint_g_patch_disp"] = adk.cpu().numpy()
    out.update(valid=ok.cpu().numpy().astype(bool), recs=recs, params=m.params)
    m.close()
    return out


@pytest.mark.parametrize("kw", [
    dict(patch=8, stride=4, levels=2, iters=50),
    dict(patch=8, stride=4, levels=3, iters=50),
    dict(patch=8, stride=4, levels=3, iters=50, sigma_r_mode="fixed"),
])
def test_adjoint_through_levels_matches_oracle_small(bd, kw):
    pr = synth.g1_pair(64, 48, 3, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    L32, R32 = pr.left.astype(np.float32), pr.right.astype(np.float32)
    L, R = L32.astype(np.float64), R32.astype(np.float64)
    g = _gpu_ml(bd, kw, L32, R32)
    op = oracle_params(g["params"])
    o = oracle.match(op, L, R, trace=True)
    st = oracle.frozen_state_ml(op, o)
    # same discrete state on both sides, every level
    assert np.array_equal(g["valid"], o["valid"])
    for l in range(op.levels):
        assert np.array_equal(g["recs"][l]["flags"].ravel() == 0, st["kept"][l].astype(bool)), l
    loss, gL, gR, gdk = oracle.mdiff_grad(op, L, R, st)
    assert abs(float(g["loss"][0]) - loss) <= 1e-5 * loss
    # every element of the adjoint chain from the GPU's own dL/dD
    oL, oR, odk = oracle.mdiff_adjoint(op, L, R, st, g["g_disp"])
    for key, ref in (("g_left", oL), ("g_right", oR)):
        good, info = _close(g["adjoint_" + key], ref)
        assert good, ("adjoint " + key, info)
    # the complete gradients: all but the elements a kink-adjacent pixel of
    # the L1 terms reaches
    for key, ref in (("g_left", gL), ("g_right", gR)):
        good, info = _close(g[key], ref, frac=0.9)
        assert good, (key, info)
    kept = st["kept"][0].astype(bool)
    good, info = _close(g["adjoint_g_patch_disp"].ravel()[kept], odk[kept])
    assert good, ("adjoint g_patch_disp", info)
    good, info = _close(g["g_patch_disp"].ravel()[kept], gdk[kept], frac=0.9)
    assert good, ("g_patch_disp", info)


def test_adjoint_through_levels_640x480(bd):
    pr = synth.g1_pair(640, 480, 0)
    L32, R32 = pr.left.astype(np.float32), pr.right.astype(np.float32)
    kw = dict(patch=8, stride=4, levels=3, iters=8)
    g = _gpu_ml(bd, kw, L32, R32)
    op = oracle_params(g["params"])
    L, R = L32.astype(np.float64), R32.astype(np.float64)
    o = oracle.match(op, L, R, trace=True)
    st = oracle.frozen_state_ml(op, o)
    flips = sum(int(((g["recs"][l]["flags"].ravel() == 0) != st["kept"][l].astype(bool)).sum())
                for l in range(op.levels))
    assert flips <= max(2, int(0.001 * st["kept"][0].size))
    loss, gL, gR, gdk = oracle.mdiff_grad(op, L, R, st)
    assert abs(float(g["loss"][0]) - loss) <= 1e-4 * loss
    for key, ref in (("g_left", gL), ("g_right", gR)):
        good, info = _close(g[key], ref, frac=0.999)
        print(key, info, "flips", flips)
        assert good, (key, info)
