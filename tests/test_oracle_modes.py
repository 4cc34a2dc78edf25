"""Pins for the oracle's optional modes: the DIS fusion weights (Eq. 2), the
finest processed level with full-resolution upsampling (Sec. IV-A: finest
scale 2^1), the Gamma weights over the processed levels (Eq. 11) and
Schraudolph's exponential (Sec. IV, technical details).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Schraudolph exp

def test_fast_exp_within_published_bound():
    bound = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))["fast_exp_error_bound"]["value"]
    ys = np.linspace(-30.0, 8.0, 40001)
    v = np.array([oracle.exp_schraudolph(y) for y in ys])
    rel = v / np.exp(ys) - 1.0
    assert np.all(np.abs(rel) < bound)
    # the correction constant centres the error: over whole periods the mean
    # relative error is near zero (a missing correction leaves it near +3 %)
    assert abs(rel.mean()) < 0.005
    # exact powers of two where the fraction bits vanish: the approximation
    # is linear in y between consecutive multiples of ln 2
    assert oracle.exp_schraudolph(-100.0) == 0.0


def test_fast_exp_relative_error_has_period_ln2():
    ys = np.linspace(-10.0, 3.0, 301)
    r0 = np.array([oracle.exp_schraudolph(y) / math.exp(y) for y in ys])
    r1 = np.array([oracle.exp_schraudolph(y + math.log(2.0)) / math.exp(y + math.log(2.0)) for y in ys])
    np.testing.assert_allclose(r0, r1, atol=1e-6)


def test_fast_exp_is_monotone_and_piecewise_linear():
    ys = np.linspace(-5.0, 5.0, 10001)
    v = np.array([oracle.exp_schraudolph(y) for y in ys])
    assert np.all(np.diff(v) >= 0)
    # affine in y inside each octave: relative second differences vanish
    # except at the octave breaks (one per ln 2, 15 in this range)
    d2 = np.abs(np.diff(v, 2)) / v[1:-1]
    kinks = int((d2 > 1e-6).sum())
    assert 14 <= kinks <= 2 * 15


def test_fast_exp_posterior_close_to_exact():
    pr = synth.config_pair("plain_320x240")
    pe = oracle.make_params(patch=8, stride=4, levels=3, iters=8)
    pf = oracle.make_params(patch=8, stride=4, levels=3, iters=8, fast_exp=1)
    oe = oracle.match(pe, pr.left, pr.right, trace=True)
    of = oracle.match(pf, pr.left, pr.right, trace=True)
    re, rf = oe["levels"][2]["patches"], of["levels"][2]["patches"]  # coarsest: same inputs
    ok = re["flags"] == 0
    assert np.array_equal(re["flags"], rf["flags"])
    rel = rf["pi"][ok] / re["pi"][ok] - 1.0
    assert np.max(np.abs(rel)) < 0.08          # pi = 1 / sum of 5 terms each within 4 %
    assert np.max(np.abs(rel)) > 1e-4          # and the mode is in effect
    assert np.all(rf["pi"][ok] <= 1.0) and np.all(rf["pi"][ok] >= 0.2 * (1 - 0.08))


def test_fast_exp_posterior_special_cases():
    p = oracle.make_params(patch=8, stride=4, levels=1, fast_exp=1)
    rec = np.zeros((1, 3), dtype=oracle.PATCH_DTYPE)
    rec["E"][0, 0] = [50.0] * 5                     # flat window: every p_i equal
    rec["E"][0, 1] = [0.0, 1e9, 1e9, 1e9, 1e9]      # sharp minimum: the others vanish
    rec["E"][0, 2] = [10.0, 10.0, 1e9, 1e9, 1e9]    # two equal samples
    post = oracle.posterior(p, 0, rec, 1.0)
    assert post["pi"][0, 0] == 0.2
    assert post["pi"][0, 1] == 1.0
    assert post["pi"][0, 2] == 0.5


# ---------------------------------------------------------------- Gamma over the processed levels

@pytest.mark.parametrize("levels,finest", [(3, 0), (6, 1), (5, 2)])
def test_gamma_weights_over_processed_levels(levels, finest):
    g = [oracle.gamma_weight(n, levels, finest) for n in range(finest, levels)]
    assert abs(sum(g) - 1.0) < 1e-15
    for a, b in zip(g, g[1:]):
        assert b == 2.0 * a


# ---------------------------------------------------------------- DIS weights (Eq. 2)

def _two_patches(d_a, d_b, mu_a=0.0, mu_b=0.0):
    p = oracle.make_params(patch=8, stride=4, levels=1, weight_mode="dis")
    w, h = 12, 8                                # origins x: 0, 4; y: 0
    rec = np.zeros((1, 2), dtype=oracle.PATCH_DTYPE)
    rec["rho"] = 1.0
    rec[0, 0]["d"], rec[0, 1]["d"] = d_a, d_b
    rec[0, 0]["mu"], rec[0, 1]["mu"] = mu_a, mu_b
    return p, w, h, rec


def test_dis_weights_inverse_squared_residual_closed_form():
    # ramp images: I_l = alpha x, I_r(x) = alpha (x + d*), so the residual of
    # a patch at disparity d is alpha (d* - d) at every pixel (no clamping)
    alpha, dstar = 2.0, 1.0
    x = np.arange(12, dtype=float)
    L = np.tile(alpha * x, (8, 1))
    R = np.tile(alpha * (x + dstar), (8, 1))
    d_a, d_b = dstar + 0.25, dstar + 2.0        # residuals -0.5 and -4
    p, w, h, rec = _two_patches(d_a, d_b)
    D, Q, V, cnt = oracle.densify(p, rec, w, h, L=L, R=R)
    w_a, w_b = 1.0, 1.0 / 16.0                  # 1 / max(1, 0.25), 1 / 16
    np.testing.assert_allclose(D[:, 4:8], (w_a * d_a + w_b * d_b) / (w_a + w_b), atol=1e-13)
    # pixels covered by one patch take its disparity
    np.testing.assert_allclose(D[:, :4], d_a, atol=1e-13)
    np.testing.assert_allclose(D[:, 8:], d_b, atol=1e-13)
    assert np.all(cnt[:, 4:8] == 2)


def test_dis_weights_remove_the_patch_mean_offset():
    alpha, dstar = 2.0, 1.0
    x = np.arange(12, dtype=float)
    L = np.tile(alpha * x, (8, 1))
    R = np.tile(alpha * (x + dstar), (8, 1))
    d_a, d_b = dstar + 0.25, dstar + 2.0
    # with mu_b equal to patch b's constant residual its weight becomes 1
    p, w, h, rec = _two_patches(d_a, d_b, mu_b=alpha * (dstar - d_b))
    D, _, _, _ = oracle.densify(p, rec, w, h, L=L, R=R)
    np.testing.assert_allclose(D[:, 4:8], 0.5 * (d_a + d_b), atol=1e-13)


def test_search_records_mean_offset():
    # a brightness offset without a shift: the Gauss-Newton step is zero
    # (sum of the centred gradient vanishes) and the mean offset is recovered
    pr = synth.g1_pair(64, 32, 2)
    L = pr.left.astype(float)
    R = L + 5.0
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=8)
    G = oracle.sobel_x(L)
    rec = oracle.search_patch(p, L, R, G, 24, 12, 0.0)
    assert abs(rec["d"]) < 1e-9
    assert abs(rec["mu"] - 5.0) < 1e-9


def test_dis_mode_constant_shift_recovered():
    pr = synth.shift_pair(160, 120, 1, 4)
    p = oracle.make_params(patch=8, stride=4, levels=3, iters=8, weight_mode="dis")
    out = oracle.match(p, pr.left, pr.right)
    inner = (slice(None), slice(4 + 8, 160 - 8))
    v = out["valid"][inner]
    assert v.mean() > 0.99
    assert np.max(np.abs(out["disp"][inner][v] - 4)) < 1e-6


# ---------------------------------------------------------------- finest level + upsampling

def test_upsample_linear_map_is_exact():
    f, wf, hf = 1, 20, 12
    w, h = 40, 24
    Y, X = np.mgrid[0:hf, 0:wf].astype(float)
    Df = 0.3 * X - 0.2 * Y + 5.0
    Vf = np.full((hf, wf), 0.7)
    disp, var, valid = oracle.upsample_output(Df, Vf, np.ones((hf, wf)), f, w, h)
    assert valid.all()
    ys, xs = np.mgrid[0:h, 0:w].astype(float)
    Xf = np.clip((xs + 0.5) / 2 - 0.5, 0, wf - 1)
    Yf = np.clip((ys + 0.5) / 2 - 0.5, 0, hf - 1)
    np.testing.assert_allclose(disp, 2.0 * (0.3 * Xf - 0.2 * Yf + 5.0), atol=1e-12)
    np.testing.assert_allclose(var, 4.0 * 0.7, atol=1e-12)


@pytest.mark.parametrize("f", [1, 2])
def test_upsample_invalid_pixel_footprint(f):
    wf, hf = 16, 12
    w, h = wf << f, hf << f
    ok = np.ones((hf, wf))
    i, j = 7, 5
    ok[j, i] = 0
    _, _, valid = oracle.upsample_output(np.ones((hf, wf)), None, ok, f, w, h)
    s = 2 ** f
    # full-resolution pixels whose two bilinear neighbours per axis include i:
    # (x + 0.5) / s - 0.5 in (i - 1, i + 1)
    xs = [x for x in range(w) if i - 1 < (x + 0.5) / s - 0.5 < i + 1]
    ys = [y for y in range(h) if j - 1 < (y + 0.5) / s - 0.5 < j + 1]
    expect = np.ones((h, w), bool)
    expect[np.ix_(ys, xs)] = False
    assert np.array_equal(valid, expect)
    assert (~valid).sum() == (2 * s) ** 2


def test_paper_preset_recovers_even_integer_shift():
    # finest processed level 1 (scale 2^1) and upsampling: a shift of 4 px is
    # 2 px at level 1 exactly, so the upsampled result is 4 in the interior
    pr = synth.shift_pair(320, 240, 3, 4)
    p = oracle.make_params(patch=10, stride=4, levels=5, iters=12, finest_level=1)
    out = oracle.match(p, pr.left, pr.right, trace=True)
    inner = (slice(8, 232), slice(4 + 24, 320 - 24))
    v = out["valid"][inner]
    assert v.mean() > 0.99
    assert np.max(np.abs(out["disp"][inner][v] - 4.0)) < 1e-6
    assert out["levels"][0]["patches"]["flags"].size > 0  # level 0 untouched (zeros)
    assert np.all(out["levels"][0]["patches"]["d"] == 0)


def test_finest_level_checked():
    p = oracle.make_params(levels=3, finest_level=3)
    with pytest.raises(ValueError):
        oracle.match(p, np.zeros((64, 64)), np.zeros((64, 64)))
