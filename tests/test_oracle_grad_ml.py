"""Pins for the oracle's gradient through every level (the coarse levels
reach the loss through the propagated probability of Eq. 10): the frozen
forward reproduces the full forward, the gradient reduces to the finest-level
one where the coarse levels cannot act, and it matches FP64 central finite
differences of the frozen forward -- where the finest-level gradient alone
does not.  CPU only."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_grad import _fd_check


def _setup(levels=3, seed=3, iters=50, **kw):
    pr = synth.g1_pair(64, 48, seed, d0=1.0, d1=3.0, amp=1.0, as_float=True)
    p = oracle.make_params(patch=8, stride=4, levels=levels, iters=iters, storage="f64", **kw)
    out = oracle.match(p, pr.left, pr.right, trace=True)
    return p, pr.left, pr.right, out


def test_frozen_forward_through_levels_reproduces_full_forward():
    p, L, R, out = _setup(iters=8)
    st = oracle.frozen_state_ml(p, out)
    loss, D, dk = oracle.mdiff_forward(p, L, R, st)
    v = out["valid"]
    np.testing.assert_allclose(D[v], out["disp"][v], rtol=0, atol=1e-10)
    loss1 = oracle.diff_forward(p, L, R, oracle.frozen_state(p, out))[0]
    assert abs(loss - loss1) < 1e-12


@pytest.mark.parametrize("kw,levels", [(dict(use_c2f=0), 3), (dict(), 1)])
def test_reduces_to_finest_level_gradient(kw, levels):
    # without coarse-to-fine propagation, or with one level, nothing upstream
    # of level 0 reaches the loss
    p, L, R, out = _setup(levels=levels, **kw)
    g1 = oracle.diff_grad(p, L, R, oracle.frozen_state(p, out))
    gm = oracle.mdiff_grad(p, L, R, oracle.frozen_state_ml(p, out))
    assert g1[0] == gm[0]
    for a, b in ((g1[1], gm[1]), (g1[2], gm[2]), (g1[3], gm[3])):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15 * np.abs(a).max())


@pytest.mark.parametrize("levels,kw", [(2, dict()), (3, dict()), (3, dict(sigma_r_mode="fixed"))])
def test_gradient_through_levels_matches_finite_differences(levels, kw):
    p, L, R, out = _setup(levels=levels, **kw)
    st = oracle.frozen_state_ml(p, out)
    loss, gL, gR, gdk = oracle.mdiff_grad(p, L, R, st)
    rng = np.random.default_rng(0)
    cand = np.flatnonzero(out["valid"].ravel())
    idx = rng.choice(cand, 120, replace=False)
    okL, badL, exL, wL = _fd_check(lambda y: oracle.mdiff_forward(p, y, R, st)[0], L, idx, gL)
    okR, badR, exR, wR = _fd_check(lambda y: oracle.mdiff_forward(p, L, y, st)[0], R, idx, gR)
    print("I_l", okL, badL, exL, wL, "I_r", okR, badR, exR, wR)
    assert badL == 0 and badR == 0
    assert okL >= 100 and okR >= 100


def test_finest_level_gradient_alone_misses_the_coarse_path():
    # the discriminating case: the finite differences of the full frozen
    # forward disagree with the finest-level gradient (coarse levels frozen)
    # somewhere, and agree everywhere with the gradient through the levels
    p, L, R, out = _setup(levels=3)
    st = oracle.frozen_state_ml(p, out)
    g1 = oracle.diff_grad(p, L, R, oracle.frozen_state(p, out))[1]
    gm = oracle.mdiff_grad(p, L, R, st)[1]
    # the pixels where the two gradients differ most
    idx = np.argsort(-np.abs(gm - g1).ravel())[:40]
    ok1, bad1, _, _ = _fd_check(lambda y: oracle.mdiff_forward(p, y, R, st)[0], L, idx, g1)
    okm, badm, _, _ = _fd_check(lambda y: oracle.mdiff_forward(p, y, R, st)[0], L, idx, gm)
    assert bad1 >= 10
    assert badm == 0 and okm >= 30


def test_adjoint_through_levels_alone_matches_finite_differences():
    # the adjoint through every level for a fixed dL/dD = g is the gradient of
    # f(I) = sum g D(I) of the frozen forward through every level
    p, L, R, out = _setup()
    st = oracle.frozen_state_ml(p, out)
    rng = np.random.default_rng(21)
    g = rng.standard_normal(L.shape) * st["valid"]
    gL, gR, gdk = oracle.mdiff_adjoint(p, L, R, st, g)

    def f_left(x):
        return float((g * oracle.mdiff_forward(p, x, R, st)[1]).sum())

    def f_right(x):
        return float((g * oracle.mdiff_forward(p, L, x, st)[1]).sum())

    idx = rng.choice(L.size, 40, replace=False)
    for fun, x, an in ((f_left, L, gL), (f_right, R, gR)):
        ok, bad, excluded, worst = _fd_check(fun, x, idx, an)
        assert bad == 0 and ok >= 34, (ok, bad, excluded, worst)
    # and the full gradient is this adjoint plus the loss's direct terms,
    # which are those of the finest-level form
    loss, fL, fR, fdk = oracle.mdiff_grad(p, L, R, st)
    _, _, _, _, gD = oracle.diff_grad(p, L, R, oracle.frozen_state(p, out))
    aL, aR, adk = oracle.mdiff_adjoint(p, L, R, st, gD)
    sL, sR, sdk = oracle.diff_adjoint(p, L, R, oracle.frozen_state(p, out), gD)
    d1 = oracle.diff_grad(p, L, R, oracle.frozen_state(p, out))
    np.testing.assert_allclose(fL - aL, d1[1] - sL, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fR - aR, d1[2] - sR, rtol=0, atol=1e-12)
