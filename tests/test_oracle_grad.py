"""Pins for the oracle's analytic gradient of the differentiable form: the
frozen-state forward reproduces the full forward, and the analytic gradient
(implicit-function rule through each converged patch solve) matches FP64
central finite differences.  CPU only."""
import numpy as np
import pytest

import oracle
import synth


def _setup(seed=3, iters=50, levels=3, **kw):
    pr = synth.g1_pair(64, 48, seed, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    p = oracle.make_params(patch=8, stride=4, levels=levels, iters=iters, storage="f64", **kw)
    out = oracle.match(p, pr.left, pr.right, trace=True)
    return p, pr.left, pr.right, out, oracle.frozen_state(p, out)


def test_frozen_forward_reproduces_full_forward():
    for kw in (dict(iters=8), dict(iters=8, use_sgmm=0), dict(iters=8, sigma_r_mode="fixed")):
        p, L, R, out, st = _setup(**kw)
        loss, D, dk = oracle.diff_forward(p, L, R, st)
        v = out["valid"]
        assert v.mean() > 0.8
        np.testing.assert_allclose(D[v], out["disp"][v], rtol=0, atol=1e-10)
        rec = out["levels"][0]["patches"].ravel()
        kept = st["kept"].astype(bool)
        np.testing.assert_allclose(dk[kept], rec["d"][kept], atol=1e-12)
        assert loss > 0


def _fd_check(fun, x, idx, an, eps=1e-3):
    """central differences at indices idx of x; a point whose two step sizes
    disagree sits near a kink (|r| = 0, |dD| = 0, integer sample position)
    and is excluded and counted"""
    ok = bad = excluded = 0
    worst = 0.0
    for i in idx:
        def f(e):
            y = x.copy()
            y.flat[i] += e
            return fun(y)
        g1 = (f(eps) - f(-eps)) / (2 * eps)
        g2 = (f(eps / 2) - f(-eps / 2)) / eps
        scale = max(abs(an.flat[i]), 1e-7)
        if abs(g1 - g2) > 1e-5 * scale + 1e-12:
            excluded += 1
            continue
        err = abs(g1 - an.flat[i]) / scale
        worst = max(worst, err)
        if err <= 1e-4:
            ok += 1
        else:
            bad += 1
    return ok, bad, excluded, worst


@pytest.mark.parametrize("kw", [dict(), dict(sigma_r_mode="fixed"), dict(use_sgmm=0, use_c2f=0)])
def test_analytic_gradient_matches_finite_differences(kw):
    p, L, R, out, st = _setup(**kw)
    loss, gL, gR, gdk, gD = oracle.diff_grad(p, L, R, st)
    rng = np.random.default_rng(0)
    valid = out["valid"]
    # pixels whose value reaches the loss: inside valid regions
    cand = np.flatnonzero(valid.ravel())
    idx = rng.choice(cand, 120, replace=False)
    okL, badL, exL, wL = _fd_check(lambda y: oracle.diff_forward(p, y, R, st)[0], L, idx, gL)
    okR, badR, exR, wR = _fd_check(lambda y: oracle.diff_forward(p, L, y, st)[0], R, idx, gR)
    print("I_l", okL, badL, exL, wL, "I_r", okR, badR, exR, wR)
    assert badL == 0 and badR == 0
    assert okL >= 100 and okR >= 100


def test_patch_disparity_gradient_matches_finite_differences():
    p, L, R, out, st = _setup()
    loss, gL, gR, gdk, gD = oracle.diff_grad(p, L, R, st)
    _, _, dk = oracle.diff_forward(p, L, R, st)
    kept = np.flatnonzero(st["kept"])
    rng = np.random.default_rng(1)
    idx = rng.choice(kept, 40, replace=False)
    ok, bad, ex, worst = _fd_check(lambda y: oracle.diff_forward(p, L, R, st, d_override=y)[0],
                                   dk, idx, gdk)
    print("d_k", ok, bad, ex, worst)
    assert bad == 0 and ok >= 30


def test_gradient_invariances():
    # a constant added to both images changes nothing (mean-normalised search,
    # residual differences): the gradient sums to zero along (1, 1)
    p, L, R, out, st = _setup()
    loss, gL, gR, gdk, gD = oracle.diff_grad(p, L, R, st)
    scale = np.abs(gL).sum() + np.abs(gR).sum()
    assert abs(gL.sum() + gR.sum()) < 1e-9 * scale
    # with the pooled sigma_r, d, pi and D are invariant to scaling both
    # images, so the data term is homogeneous of degree 1 and the smoothness
    # term of degree 0: Euler's identity sum(I dL/dI) = data term checks every
    # chain term, including the one through sigma_r
    assert st["sr_const"] == 0
    data = oracle.diff_forward(p, L, R, st, lam=0.0)[0]
    assert data < loss
    assert abs((gL * L).sum() + (gR * R).sum() - data) < 1e-8 * data


def test_adjoint_alone_matches_finite_differences_of_a_linear_loss():
    # for a fixed weight map g, the adjoint chain of dL/dD = g is the gradient
    # of f(I) = sum g D(I) (the frozen forward's D): FD pins it independently
    p, L, R, out, st = _setup()
    rng = np.random.default_rng(12)
    g = rng.standard_normal(L.shape) * st["valid"]
    gL, gR, gdk = oracle.diff_adjoint(p, L, R, st, g)

    def f_left(x):
        return float((g * oracle.diff_forward(p, x, R, st)[1]).sum())

    def f_right(x):
        return float((g * oracle.diff_forward(p, L, x, st)[1]).sum())

    idx = rng.choice(L.size, 60, replace=False)
    for fun, x, an in ((f_left, L, gL), (f_right, R, gR)):
        ok, bad, excluded, worst = _fd_check(fun, x, idx, an)
        assert bad == 0 and ok >= 54, (ok, bad, excluded, worst)


def test_full_gradient_is_adjoint_plus_direct_loss_terms():
    # dL/dI = (direct terms of the loss) + adjoint(dL/dD); the direct terms of
    # the L1 reprojection are -sign(r)/(w h) on I_l and the interpolation
    # taps of sign(r)/(w h) on I_r
    p, L, R, out, st = _setup()
    loss, gL, gR, gdk, gD = oracle.diff_grad(p, L, R, st)
    aL, aR, adk = oracle.diff_adjoint(p, L, R, st, gD)
    _, D, _ = oracle.diff_forward(p, L, R, st)
    h, w = L.shape
    dL = np.zeros_like(L)
    dR = np.zeros_like(R)
    for y in range(h):
        for x in range(w):
            if not st["valid"][y, x]:
                continue
            X = min(max(x - D[y, x], 0.0), w - 1.0)
            x0 = int(np.floor(X))
            x1 = min(x0 + 1, w - 1)
            t = X - x0
            r = (1 - t) * R[y, x0] + t * R[y, x1] - L[y, x]
            s = np.sign(r) / (w * h)
            dL[y, x] -= s
            dR[y, x0] += s * (1 - t)
            dR[y, x1] += s * t
    np.testing.assert_allclose(gL, dL + aL, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gR, dR + aR, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gdk, adk, rtol=0, atol=1e-15)
