"""Pins for the FP64 CPU oracle: closed forms, invariants, special cases
that reduce to library routines, and brute force on tiny inputs.  These fix
the oracle to the paper's definitions independently of the oracle itself and
of the CUDA path.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- storage

def test_round_f16_matches_numpy_half():
    # numpy's double -> binary16 conversion is an independent library routine
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.uniform(-300, 300, 4000),
        rng.uniform(-1e-3, 1e-3, 2000),          # includes subnormals
        rng.uniform(-7e-5, 7e-5, 1000),
        np.array([0.0, 65504.0, 65519.9, 65520.0, 1e6, -1e6]),
    ])
    # exact ties between binary16 neighbours (round half to even)
    ties = (np.arange(1, 400) + 0.5) * 2.0 ** -3   # spacing 1/8 above 64 -> ties at 1/16
    vals = np.concatenate([vals, ties + 64.0, (np.arange(1, 200) + 0.5) * 2.0 ** -24])
    for v in vals:
        a = oracle.round_f16(v)
        with np.errstate(over="ignore"):
            b = float(np.float64(v).astype(np.float16))
        assert a == b or (math.isinf(a) and math.isinf(b)), (v, a, b)


# ---------------------------------------------------------------- geometry

@pytest.mark.parametrize("n,P,S", [(320, 8, 4), (640, 12, 6), (1920, 12, 4), (61, 8, 4),
                                   (60, 12, 4), (34, 12, 4), (13, 10, 4), (12, 12, 5)])
def test_origins_cover_every_pixel(n, P, S):
    o = oracle.origins(n, P, S)
    assert o[0] == 0 and o[-1] == n - P
    assert np.all(np.diff(o) > 0) and np.all(np.diff(o)[:-1] == S)
    cover = np.zeros(n, int)
    for a in o:
        cover[a:a + P] += 1
    assert cover.min() >= 1
    # count: floor((n-P)/S) + 1 regular origins plus one extra if ragged
    assert len(o) == (n - P) // S + 1 + int((n - P) % S != 0)


def test_level_dims_ceil_halving():
    assert [oracle.level_dim(1080, l) for l in range(6)] == [1080, 540, 270, 135, 68, 34]
    assert [oracle.level_dim(1920, l) for l in range(6)] == [1920, 960, 480, 240, 120, 60]


def test_patch_counts_of_the_workloads():
    # (w, h, P, S, L) -> totals from the origin rule (also in the design notes)
    cases = {(320, 240, 8, 4, 3): [4661, 1131, 266],
             (640, 480, 12, 6, 4): [8374, 2067, 494, 117],
             (1920, 1080, 12, 4, 6): [128104, 31654, 7788, 1856, 420, 91]}
    for (w, h, P, S, L), want in cases.items():
        p = oracle.make_params(patch=P, stride=S, levels=L)
        got = [oracle.num_patches(p, w, h, l)[0] for l in range(L)]
        assert got == want


def test_gamma_weights():
    for L in range(1, 7):
        w = [oracle.gamma_weight(n, L) for n in range(L)]
        assert abs(sum(w) - 1.0) < 1e-15
        for n in range(L - 1):           # one level coarser doubles the weight
            assert abs(w[n + 1] / w[n] - 2.0) < 1e-14


# ---------------------------------------------------------------- pyramid / gradient

def _reflect101_conv_numpy(img, k):
    # separable correlation with numpy's 'reflect' padding (edge not repeated)
    r = len(k) // 2
    out = img
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="reflect")
        n = out.shape[axis]
        acc = np.zeros_like(out)
        for i, kv in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + n)
            acc = acc + kv * p[tuple(sl)]
        out = acc
    return out


@pytest.mark.parametrize("h,w", [(8, 8), (13, 17), (24, 31)])
def test_pyr_down_equals_blur_then_decimate(h, w):
    rng = np.random.default_rng(h * w)
    img = rng.uniform(0, 255, (h, w))
    k = np.array([1, 4, 6, 4, 1]) / 16.0
    want = _reflect101_conv_numpy(img, k)[::2, ::2]
    got = oracle.pyr_down(img)
    assert got.shape == ((h + 1) // 2, (w + 1) // 2)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_pyr_down_constant_linear_quadratic():
    h, w = 20, 30
    assert np.all(oracle.pyr_down(np.full((h, w), 77.0)) == 77.0)
    X = np.arange(w, dtype=float)[None, :].repeat(h, 0)
    lin = oracle.pyr_down(3.0 * X)
    # symmetric kernel keeps a linear ramp: level value at X is 3 * 2X (interior)
    want = np.broadcast_to(6.0 * np.arange(1, (w + 1) // 2 - 2)[None, :], lin[:, 1:-2].shape)
    np.testing.assert_allclose(lin[:, 1:-2], want, atol=1e-12)
    quad = oracle.pyr_down(X * X)
    # binomial [1 4 6 4 1]/16 has variance 1: blur(x^2) = x^2 + 1 in the interior
    Xc = np.arange((w + 1) // 2, dtype=float)
    want = np.broadcast_to((4 * Xc * Xc + 1)[None, 1:-2], quad[:, 1:-2].shape)
    # rows are constant (no y dependence), so only the x interior matters
    np.testing.assert_allclose(quad[:, 1:-2], want, atol=1e-9)


def test_pyr_down_f16_storage_rounds_each_level():
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 255, (16, 16))
    a = oracle.pyr_down(img, "f16")
    b = oracle.pyr_down(img, "f64").astype(np.float16).astype(np.float64)
    assert np.array_equal(a, b)


def test_sobel_matches_scipy():
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 255, (11, 14))
    want = scipy_ndimage.sobel(img, axis=1, mode="mirror") / 8.0  # 'mirror' = reflect-101
    np.testing.assert_allclose(oracle.sobel_x(img), want, atol=1e-12)


def test_sobel_of_ramp_and_quadratic():
    X = np.arange(20, dtype=float)[None, :].repeat(9, 0)
    g = oracle.sobel_x(2.5 * X + 7)
    np.testing.assert_allclose(g[:, 1:-1], 2.5, atol=1e-12)
    q = oracle.sobel_x(0.3 * X * X)
    np.testing.assert_allclose(q[:, 1:-1], (0.6 * X)[:, 1:-1], atol=1e-12)


# ---------------------------------------------------------------- GN search

def _quad_setup(beta, dstar, w=96, h=24):
    L = synth.quadratic_image(w, h, beta)
    R = synth.quadratic_image(w, h, beta, shift=dstar)  # R(x - d*) = L(x)
    return L, R, oracle.sobel_x(L)


@pytest.mark.parametrize("P", [8, 10, 12])
@pytest.mark.parametrize("beta,dstar,dinit", [(0.01, 2.3, 0.0), (0.05, 5.75, 3.0),
                                              (0.004, 1.1, 4.9), (0.02, 7.0, 7.6)])
def test_gn_lands_on_shift_in_one_step(P, beta, dstar, dinit):
    # I = beta x^2: the linear-interpolation error is constant over the patch
    # and removed by mean normalisation; Sobel/8 gives 2 beta x exactly; so one
    # inverse-compositional step is exact from any init.
    L, R, G = _quad_setup(beta, dstar)
    p = oracle.make_params(patch=P, stride=4, levels=1, iters=1, storage="f64")
    rec = oracle.search_patch(p, L, R, G, 40, 6, dinit)
    assert abs(rec["d"] - dstar) < 1e-9
    assert abs(rec["dlast"] - (dstar - dinit)) < 1e-9


@pytest.mark.parametrize("P", [8, 12])
def test_window_energies_quadratic_closed_form(P):
    beta, dstar = 0.03, 3.4
    L, R, G = _quad_setup(beta, dstar)
    p = oracle.make_params(patch=P, stride=4, levels=1, iters=3, storage="f64")
    rec = oracle.search_patch(p, L, R, G, 40, 6, 2.0)
    # sum over the patch of (x - xbar)^2: P rows of P (P^2 - 1) / 12
    S = P * (P * (P * P - 1) / 12.0)
    deltas = oracle.window_offsets(0.5)
    for k, dl in enumerate(deltas):
        want = 4 * beta ** 2 * (dstar - rec["d"] - dl) ** 2 * S
        assert abs(rec["E"][k] - want) < 1e-8 * max(1.0, want)
    assert rec["flags"] == 0


def test_window_offsets_are_the_papers_disturbances():
    d = oracle.window_offsets(0.5)
    assert d[0] == 0.0 and sorted(d) == [-1.0, -0.5, 0.0, 0.5, 1.0]


def test_gn_equals_brute_force_root_of_its_equation():
    # brute force on tiny inputs: scan d on a fine grid for the sign change of
    # F(d) = sum gt_i (s_i(d) - T_i), the inverse-compositional stationarity
    # condition, and compare with the converged GN estimate.
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=30, storage="f64")
    rng = np.random.default_rng(5)
    worst = 0.0
    for seed in range(4):
        dstar = rng.uniform(1.2, 3.8)
        tex = synth.gaussian_blur(np.random.default_rng(seed).standard_normal((16, 40)), 3.0)
        tex = tex / tex.std() * 40 + 128
        L = tex[:, :32]
        xs = np.arange(32) + dstar
        x0 = np.floor(xs).astype(int)
        t = xs - x0
        R = (1 - t) * tex[:, x0] + t * tex[:, x0 + 1]
        G = oracle.sobel_x(L)
        for oy in (0, 8):
            for ox in (8, 16, 24):
                rec = oracle.search_patch(p, L, R, G, ox, oy, float(round(dstar)))
                T = L[oy:oy + 8, ox:ox + 8]
                gt = G[oy:oy + 8, ox:ox + 8] - G[oy:oy + 8, ox:ox + 8].mean()
                rows = np.arange(oy, oy + 8)[:, None]
                cols = np.arange(ox, ox + 8)[None, :]
                ds = np.arange(dstar - 1, dstar + 1, 5e-5)
                F = []
                for d in ds:
                    X = np.clip(cols - d, 0, 31)
                    a0 = np.floor(X).astype(int)
                    a1 = np.minimum(a0 + 1, 31)
                    tt = X - a0
                    s = (1 - tt) * R[rows, a0] + tt * R[rows, a1]
                    F.append((gt * (s - T)).sum())
                F = np.array(F)
                roots = ds[np.where(np.sign(F[:-1]) != np.sign(F[1:]))[0]]
                r = roots[np.argmin(np.abs(roots - rec["d"]))]
                worst = max(worst, abs(r - rec["d"]))
    assert worst < 1e-3


def test_gn_matches_brute_force_ssd_on_integer_shift():
    pr = synth.shift_pair(40, 16, 3, 3)
    L, R = pr.left.astype(float), pr.right.astype(float)
    G = oracle.sobel_x(L)
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=10, storage="f64")
    for ox in (8, 16, 24):
        rec = oracle.search_patch(p, L, R, G, ox, 4, 2.4)
        T = L[4:12, ox:ox + 8]
        best = min(range(0, 8), key=lambda d: ((R[4:12, ox - d:ox - d + 8] - T) ** 2).sum()
                   if ox - d >= 0 else 1e18)
        assert best == 3 and abs(rec["d"] - 3.0) < 1e-6


def test_flat_patch_rejected_and_saddle_detected():
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=4, storage="f64")
    flat = np.full((16, 32), 50.0)
    rec = oracle.search_patch(p, flat, flat, oracle.sobel_x(flat), 8, 4, 0.0)
    assert rec["flags"] & oracle.F_FLAT
    # a patch pinned off the minimum: init far, zero iterations -> centre is
    # not the window minimum (saddle/unconverged rejection, Sec. IV)
    L, R, G = _quad_setup(0.02, 4.0)
    p0 = oracle.make_params(patch=8, stride=4, levels=1, iters=0, storage="f64")
    rec = oracle.search_patch(p0, L, R, G, 40, 6, 1.0)
    assert rec["flags"] & oracle.F_SADDLE


def test_out_of_image_samples_counted():
    L, R, G = _quad_setup(0.01, 2.0, w=40)
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=0, storage="f64")
    rec = oracle.search_patch(p, L, R, G, 0, 4, 3.0)   # x - 3 < 0 for x = 0, 1, 2
    assert rec["nout"] == 3 * 8
    rec = oracle.search_patch(p, L, R, G, 0, 4, 2.5)   # x - 2.5 < 0 for x = 0, 1, 2
    assert rec["nout"] == 3 * 8
    rec = oracle.search_patch(p, L, R, G, 32, 4, -1.0)  # x + 1 > 39 for x = 39
    assert rec["nout"] == 8
    p2 = oracle.make_params(patch=8, stride=4, levels=1, iters=0, storage="f64", valid_gamma=0.75)
    rec = oracle.search_patch(p2, L, R, G, 0, 4, 3.0)  # 24/64 out > 25%
    assert rec["flags"] & oracle.F_OUTSIDE


# ---------------------------------------------------------------- sigma_r, posterior

def test_sigma_r_pooled_recovers_noise_std():
    # zero disparity, right = left + N(0, sn^2): the pooled per-pixel residual
    # std estimates sn (up to the P^2/(P^2-1) mean-removal factor)
    rng = np.random.default_rng(7)
    tex = synth.gaussian_blur(rng.standard_normal((200, 200)), 2.0)
    L = tex / tex.std() * 40 + 128
    sn = 3.0
    R = L + rng.normal(0, sn, L.shape)
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=8, storage="f64", search_radius=4)
    rec = oracle.search_level(p, L, R, oracle.sobel_x(L))
    sr = oracle.sigma_r(p, rec)
    assert abs(sr - sn) / sn < 0.05


def test_sigma_r_modes():
    p = oracle.make_params(sigma_r_mode="fixed")
    rec = np.zeros((2, 2), dtype=oracle.PATCH_DTYPE)
    assert oracle.sigma_r(p, rec) == 8.0
    rec["flags"] = 1   # nothing valid -> floor
    assert oracle.sigma_r(oracle.make_params(), rec) == 0.5


def _records_with_E(E):
    rec = np.zeros((1, len(E)), dtype=oracle.PATCH_DTYPE)
    rec["E"][0] = np.asarray(E)
    return rec


def test_posterior_flat_window_is_one_fifth_and_textured_near_one():
    p = oracle.make_params(levels=1)
    post = oracle.posterior(p, 0, _records_with_E([[5.0] * 5, [0.0, 900, 900, 3600, 3600]]), 1.0)
    assert abs(post["pi"][0, 0] - 0.2) < 1e-15
    assert post["pi"][0, 1] > 0.99


def test_fig2_textured_vs_textureless_patch():
    # Fig. 2: a textured patch gives a peaked window posterior, a textureless
    # patch (constant + noise) an almost flat one.
    rng = np.random.default_rng(11)
    tex = synth.gaussian_blur(rng.standard_normal((40, 80)), 1.5)
    tex = tex / tex.std() * 40 + 128
    Lt = tex[:, :64]
    Rt = tex[:, 2:66] + rng.normal(0, 2, (40, 64))
    flat = 128 + rng.normal(0, 0.5, (40, 80))
    Lf, Rf = flat[:, :64], flat[:, 2:66] + rng.normal(0, 2, (40, 64))
    p = oracle.make_params(patch=12, stride=6, levels=1, iters=8, storage="f64")
    sr = 2.5
    rt = oracle.search_patch(p, Lt, Rt, oracle.sobel_x(Lt), 24, 12, 2.0)
    rf = oracle.search_patch(p, Lf, Rf, oracle.sobel_x(Lf), 24, 12, 2.0)
    pt = oracle.posterior(p, 0, rt.reshape(1, 1).copy(), sr)
    rf = rf.copy()
    rf["flags"] = 0
    pf = oracle.posterior(p, 0, rf.reshape(1, 1).copy(), sr)
    assert pt["pi"][0, 0] > 0.9
    assert pf["pi"][0, 0] < 0.3


def test_rho_adds_constant_coarse_probability():
    p = oracle.make_params(patch=8, stride=4, levels=3)
    rec = oracle.search_level(p, *[np.full((16, 16), 1.0)] * 3)
    rec["flags"] = 0
    rec["E"] = np.array([0.0, 10, 10, 40, 40])
    Qc = np.full((8, 8), 0.37)
    post = oracle.posterior(p, 1, rec, 1.0, Qc=Qc, w=16, h=16)
    w1 = oracle.gamma_weight(1, 3)
    np.testing.assert_allclose(post["rho"], w1 * post["pi"] + 0.37, atol=1e-14)
    post0 = oracle.posterior(p, 1, rec, 1.0)
    np.testing.assert_allclose(post0["rho"], w1 * post0["pi"], atol=1e-15)


# ---------------------------------------------------------------- PDF fit

def _lls(lnp, delta):
    # closed-form linear least squares of lnp against [1, -delta^2]
    A = np.stack([np.ones(5), -np.asarray(delta) ** 2], 1)
    (alpha, b), *_ = np.linalg.lstsq(A, lnp, rcond=None)
    return 1.0 / (2.0 * b)


@pytest.mark.parametrize("sig", [0.15, 0.3, 0.5, 0.8])
def test_pdf_fit_exact_gaussian(sig):
    delta = oracle.window_offsets(0.5)
    lp = -delta ** 2 / (2 * sig * sig)
    lnp = lp - np.log(np.exp(lp).sum())
    r = oracle.pdf_fit(lnp, delta, iters=10, tau=8.0)
    assert r["flags"] == 0
    assert abs(r["sig2"] - sig * sig) < 1e-6 * sig * sig


def test_pdf_fit_equals_linear_least_squares_closed_form():
    rng = np.random.default_rng(3)
    delta = oracle.window_offsets(0.5)
    n_ok = 0
    for _ in range(300):
        sig = rng.uniform(0.2, 1.0)
        lp = -delta ** 2 / (2 * sig * sig) + rng.normal(0, 0.02, 5)
        lp[0] = max(lp[0], lp[1:].max() + 1e-3)
        lnp = lp - np.log(np.exp(lp).sum())
        r = oracle.pdf_fit(lnp, delta, iters=10, tau=8.0)
        if r["flags"]:
            continue
        n_ok += 1
        assert abs(r["sig2"] - min(_lls(lnp, delta), 64.0)) < 1e-6 * r["sig2"]
    assert n_ok > 250


def test_pdf_fit_quadratic_image_sigma_closed_form():
    # on I = beta x^2 after convergence E(delta) = 4 beta^2 delta^2 S, so
    # sigma_k^2 = sigma_r^2 s^2 / (4 beta^2 S) exactly (s = 5 window samples)
    P, beta = 8, 0.08
    L, R, G = _quad_setup(beta, 3.3)
    p = oracle.make_params(patch=P, stride=4, levels=1, iters=2, storage="f64", variance=1)
    rec = oracle.search_patch(p, L, R, G, 40, 6, 2.5).reshape(1, 1).copy()
    sr = 0.5
    post = oracle.posterior(p, 0, rec, sr)
    S = P * (P * (P * P - 1) / 12.0)
    want = sr ** 2 * 25 / (4 * beta ** 2 * S)
    assert post["pdf_flags"][0, 0] == 0
    assert abs(post["sig2"][0, 0] - want) < 1e-6 * want


def test_pdf_fit_exceptions():
    delta = oracle.window_offsets(0.5)
    flat = np.full(5, np.log(0.2))          # ramp image: all energies equal
    r = oracle.pdf_fit(flat, delta, tau=8.0)
    assert r["flags"] & oracle.PDF_NOT_PEAK and r["sig2"] == 64.0
    bumpy = np.log(np.array([0.4, 0.05, 0.3, 0.2, 0.05]))  # non-Gaussian
    r = oracle.pdf_fit(bumpy, delta, tau=8.0)
    assert r["flags"] & oracle.PDF_RESIDUAL and r["sig2"] == 64.0


def test_ramp_image_has_no_texture():
    # I = alpha x: all window energies vanish and the patch is rejected as flat
    L = synth.ramp_image(48, 16, 1.7, 20)
    R = synth.ramp_image(48, 16, 1.7, 20 + 1.7 * 2.2)
    p = oracle.make_params(patch=8, stride=4, levels=1, iters=4, storage="f64")
    rec = oracle.search_patch(p, L, R, oracle.sobel_x(L), 16, 4, 2.0)
    assert rec["flags"] & oracle.F_FLAT
    assert np.all(np.abs(rec["E"]) < 1e-9)


# ---------------------------------------------------------------- sGMM + fusion

@pytest.mark.parametrize("P,ss", [(8, 4.0), (12, 4.0), (10, 2.5)])
def test_sgmm_table_is_separable_and_symmetric(P, ss):
    M = oracle.sgmm_table(P, ss)
    a = np.arange(P)
    m = np.exp(-(a[:, None] - a[None, :]) ** 2 / (2 * ss * ss)).sum(1)
    np.testing.assert_allclose(M, np.outer(m, m), rtol=1e-13)
    np.testing.assert_allclose(M, M[::-1, ::-1], rtol=1e-13)
    assert M[P // 2, P // 2] > M[0, 0]  # centre weighs more than the corner


def _grid_records(p, w, h):
    npx = len(oracle.origins(w, p.patch, p.stride))
    npy = len(oracle.origins(h, p.patch, p.stride))
    rec = np.zeros((npy, npx), dtype=oracle.PATCH_DTYPE)
    rec["flags"] = 1
    return rec


def test_densify_single_patch_and_constant_disparity():
    p = oracle.make_params(patch=8, stride=4, levels=1)
    w, h = 40, 24
    rec = _grid_records(p, w, h)
    rec[2, 3]["flags"] = 0
    rec[2, 3]["d"] = 4.25
    rec[2, 3]["rho"] = 0.3
    D, Q, V, cnt = oracle.densify(p, rec, w, h)
    ox, oy = 12, 8
    assert np.all(D[oy:oy + 8, ox:ox + 8] == 4.25)
    assert np.allclose(Q[oy:oy + 8, ox:ox + 8], 0.3, atol=1e-15)
    assert cnt.sum() == 64
    rec["flags"] = 0
    rec["d"] = 7.5
    rec["rho"] = np.random.default_rng(0).uniform(0.2, 1.0, rec.shape)
    D, Q, V, cnt = oracle.densify(p, rec, w, h)
    assert np.all(cnt >= 1)
    # normalised weights sum to one: a constant field is reproduced
    np.testing.assert_allclose(D, 7.5, atol=1e-13)


def test_densify_weights_and_variance_bounds():
    rng = np.random.default_rng(4)
    p = oracle.make_params(patch=12, stride=6, levels=1)
    w, h = 50, 38
    rec = _grid_records(p, w, h)
    rec["flags"] = (rng.uniform(size=rec.shape) < 0.3).astype(np.uint32)
    rec["d"] = rng.uniform(0, 10, rec.shape)
    rec["rho"] = rng.uniform(0.2, 1.0, rec.shape)
    rec["sig2"] = rng.uniform(0.01, 2.0, rec.shape)
    D, Q, V, cnt = oracle.densify(p, rec, w, h)
    ox, oy = oracle.origins(w, 12, 6), oracle.origins(h, 12, 6)
    M = oracle.sgmm_table(12, 4.0)
    for (y, x) in [(0, 0), (5, 7), (20, 30), (37, 49), (13, 44)]:
        ks = [(ky, kx) for ky in range(len(oy)) for kx in range(len(ox))
              if oy[ky] <= y < oy[ky] + 12 and ox[kx] <= x < ox[kx] + 12 and rec[ky, kx]["flags"] == 0]
        if not ks:
            assert cnt[y, x] == 0
            continue
        om = np.array([rec[k]["rho"] * M[y - oy[k[0]], x - ox[k[1]]] for k in ks])
        wn = om / om.sum()
        d = np.array([rec[k]["d"] for k in ks])
        s2 = np.array([rec[k]["sig2"] for k in ks])
        assert abs(D[y, x] - (wn * d).sum()) < 1e-12
        assert d.min() - 1e-12 <= D[y, x] <= d.max() + 1e-12
        assert s2.min() / len(ks) - 1e-12 <= V[y, x] <= s2.max() + 1e-12


def test_densify_uncovered_pixels_take_upsampled_coarse_disparity():
    p = oracle.make_params(patch=8, stride=4, levels=2)
    w, h = 24, 16
    rec = _grid_records(p, w, h)          # nothing valid
    Dc = np.full((8, 12), 3.0)
    D, Q, V, cnt = oracle.densify(p, rec, w, h, Dc=Dc)
    assert np.all(D == 6.0) and np.all(Q == 0.0) and np.all(cnt == 0)


# ---------------------------------------------------------------- end to end

@pytest.mark.parametrize("shift", [2, 4, 6])
def test_integer_shift_recovered_at_interior_pixels(shift):
    pr = synth.shift_pair(160, 120, 1, shift)
    p = oracle.make_params(patch=8, stride=4, levels=3, iters=8)
    out = oracle.match(p, pr.left, pr.right)
    P = 8
    inner = (slice(None), slice(shift + P, 160 - P))
    v = out["valid"][inner]
    assert v.mean() > 0.99
    assert np.max(np.abs(out["disp"][inner][v] - shift)) < 1e-6


def test_smooth_ground_truth_warp_epe():
    # within the LK basin (1-3 px, no noise) the dense result stays within a
    # small end-point error of the left-grid ground truth
    pr = synth.g1_pair(320, 240, 0, d0=1.0, d1=3.0, amp=1.0, noise=0.0)
    gt = pr.gt_left()
    p = oracle.make_params(patch=8, stride=4, levels=3, iters=8)
    out = oracle.match(p, pr.left, pr.right)
    v = out["valid"]
    e = np.abs(out["disp"][v] - gt[v])
    assert v.mean() > 0.98
    assert e.mean() < 0.03 and np.median(e) < 0.02


def test_match_trace_consistency():
    pr = synth.config_pair("plain_320x240")
    p = oracle.make_params(patch=8, stride=4, levels=3, iters=8, variance=1)
    out = oracle.match(p, pr.left, pr.right, trace=True)
    lv0 = out["levels"][0]
    assert np.array_equal(lv0["L"], pr.left.astype(float))
    # the pyramid stored in the trace is the blur/decimate of the level above
    np.testing.assert_allclose(out["levels"][1]["L"], oracle.pyr_down(lv0["L"], "f32"), atol=0)
    assert np.all(np.isnan(out["disp"][~out["valid"]]))
    assert np.all(np.isfinite(out["var"][out["valid"]]))
    assert np.all(out["var"][out["valid"]] >= 0)
    # at the finest level every valid pixel passed the pixel threshold
    assert np.all(lv0["Q"][out["valid"]] >= 0.15)
    for l in range(3):
        rec = out["levels"][l]["patches"]
        ok = rec["flags"] == 0
        assert np.all((rec["pi"][ok] >= 0.2 - 1e-12) & (rec["pi"][ok] <= 1 + 1e-12))


def test_default_parameters_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    p = oracle.make_params()
    assert p.sigma_s == g["sigma_s"]["value"]
    assert p.window_step == g["window_disturbances_px"]["value"][0]
    assert 2 * p.window_step == g["window_disturbances_px"]["value"][1]
    assert 5 == g["window_samples"]["value"]
    assert p.conv_eps == g["early_stopping"]["value"][0]
    assert p.valid_gamma == g["valid_gamma"]["value"]
    assert p.pix_thresh == g["pixel_threshold"]["value"]
    assert p.sigma_r_fixed == g["fixed_sigma_r_ablation"]["value"]
    assert p.pdf_iters == g["pdf_iterations"]["value"]
    assert p.pdf_resid == g["pdf_residual_threshold"]["value"]


# ---------------------------------------------------------------- coarse-to-fine lookup

# Coarse pixel X of level n+1 stands for the fine pixels 2X and 2X+1 of level
# n (Fig. 1: each level halves the resolution), so its centre sits at fine
# coordinate 2X + 1/2.  A disparity field that is linear at the fine level,
# sampled at the coarse centres and halved (a disparity measured in coarse
# pixels is half the fine one), must come back exactly from any coarse-to-
# fine lookup that interpolates bilinearly: bilinear interpolation reproduces
# linear functions.  A wrong coordinate map (x/2 instead of the centre
# convention), a missing factor 2 or a patch centre other than the mean of
# the patch's pixel coordinates all change the recovered values.

def _fine_plane(a, b, c):
    return lambda x, y: a * x + b * y + c


def _coarse_samples(f, wc, hc, scale):
    X = np.arange(wc, dtype=float)[None, :]
    Y = np.arange(hc, dtype=float)[:, None]
    return np.ascontiguousarray(f(2 * X + 0.5, 2 * Y + 0.5) * scale * np.ones((hc, wc)))


def _interior(n_fine, n_coarse):
    # fine coordinates whose coarse coordinate (x + 0.5)/2 - 0.5 lies in
    # [0, n_coarse - 1]: no clamping
    return lambda v: (v >= 0.5) & (v <= 2 * n_coarse - 1.5)


@pytest.mark.parametrize("a,b,c", [(0.37, -0.21, 5.0), (-1.3, 0.8, 20.0)])
def test_densify_fallback_recovers_linear_fine_field(a, b, c):
    # nothing valid at this level: every pixel takes 2 * bilinear(D^(n+1))
    p = oracle.make_params(patch=8, stride=4, levels=2)
    w, h = 26, 18
    wc, hc = (w + 1) // 2, (h + 1) // 2
    f = _fine_plane(a, b, c)
    Dc = _coarse_samples(f, wc, hc, 0.5)
    rec = _grid_records(p, w, h)
    D, Q, V, cnt = oracle.densify(p, rec, w, h, Dc=Dc)
    xs, ys = np.meshgrid(np.arange(w, dtype=float), np.arange(h, dtype=float))
    inner = _interior(w, wc)(xs) & _interior(h, hc)(ys)
    assert inner.sum() > 0.7 * w * h
    np.testing.assert_allclose(D[inner], f(xs, ys)[inner], rtol=0, atol=1e-12)
    assert np.all(Q == 0.0) and np.all(cnt == 0)


@pytest.mark.parametrize("P", [7, 8])
def test_search_init_is_linear_coarse_field_at_patch_centre(P):
    # the initial estimate of every patch is the fine field at the patch
    # centre: the mean of its pixel coordinates, origin + (P - 1)/2
    p = oracle.make_params(patch=P, stride=3, levels=2, iters=0, storage="f64")
    w, h = 40, 27
    wc, hc = (w + 1) // 2, (h + 1) // 2
    f = _fine_plane(0.11, 0.29, 2.5)
    Dc = _coarse_samples(f, wc, hc, 0.5)
    rng = np.random.default_rng(P)
    L = rng.uniform(0, 255, (h, w))
    rec = oracle.search_level(p, L, L, oracle.sobel_x(L), Dc=Dc)
    ox, oy = oracle.origins(w, P, 3), oracle.origins(h, P, 3)
    cx = ox + (P - 1) / 2.0
    cy = oy + (P - 1) / 2.0
    CX, CY = np.meshgrid(cx, cy)
    inner = _interior(w, wc)(CX) & _interior(h, hc)(CY)
    assert inner.sum() >= 0.6 * inner.size
    np.testing.assert_allclose(rec["dinit"][inner], f(CX, CY)[inner], rtol=0, atol=1e-12)
    # with zero iterations the estimate is the initial value
    np.testing.assert_allclose(rec["d"], rec["dinit"], rtol=0, atol=0)


@pytest.mark.parametrize("P", [7, 8])
def test_inherited_probability_is_linear_coarse_map_at_patch_centre(P):
    # Eq. 10 (reading): rho_k = Gamma_n pi_k + Q^(n+1)(centre); a probability
    # carries no resolution factor, so the coarse map is sampled unscaled
    p = oracle.make_params(patch=P, stride=3, levels=3)
    w, h = 40, 27
    wc, hc = (w + 1) // 2, (h + 1) // 2
    g = _fine_plane(0.004, -0.003, 0.42)
    Qc = _coarse_samples(g, wc, hc, 1.0)
    rec = _grid_records(p, w, h)
    rec["flags"] = 0
    rec["E"] = np.array([0.0, 30, 30, 120, 120])
    post = oracle.posterior(p, 1, rec, 1.0, Qc=Qc, w=w, h=h)
    ox, oy = oracle.origins(w, P, 3), oracle.origins(h, P, 3)
    CX, CY = np.meshgrid(ox + (P - 1) / 2.0, oy + (P - 1) / 2.0)
    inner = _interior(w, wc)(CX) & _interior(h, hc)(CY)
    w1 = oracle.gamma_weight(1, 3)
    np.testing.assert_allclose(post["prop"][inner], g(CX, CY)[inner], rtol=0, atol=1e-14)
    np.testing.assert_allclose((post["rho"] - w1 * post["pi"])[inner], g(CX, CY)[inner],
                               rtol=0, atol=1e-14)


# ---------------------------------------------------------------- sigma_r exact

def _checker_quadratic(beta, dstar, c, w=96, h=24):
    # left I = beta x^2; right = the left shifted by the integer d* plus the
    # checkerboard c (-1)^(x+y).  With an even patch side every column of a
    # patch holds as many +c as -c, so the checkerboard is orthogonal to the
    # centred gradient 2 beta (x - xbar) (which has no y dependence) at any
    # sample position, and the search converges on d* as without it.  At d*
    # the residual is the checkerboard itself: E(0) = c^2 P^2 exactly.  At
    # half-pixel offsets linear interpolation cancels the checkerboard, so
    # E(+-1/2) = beta^2 S (the closed form of the quadratic image), which
    # keeps the patch when beta^2 S > c^2 P^2.
    L = synth.quadratic_image(w, h, beta)
    X, Y = np.meshgrid(np.arange(w), np.arange(h))
    R = synth.quadratic_image(w, h, beta, shift=dstar) + c * (-1.0) ** (X + Y)
    return L, R, oracle.sobel_x(L)


@pytest.mark.parametrize("c", [0.75, 1.5, 2.5])
def test_sigma_r_pooled_exact_on_noise_free_checkerboard(c):
    P, beta, dstar = 8, 1.2, 3
    S = P * (P * (P * P - 1) / 12.0)
    assert beta ** 2 * S > c * c * P * P
    L, R, G = _checker_quadratic(beta, dstar, c)
    p = oracle.make_params(patch=P, stride=4, levels=1, iters=3, storage="f64")
    recs = []
    for oy in (0, 4, 8, 16):
        for ox in range(16, 80, 4):
            r = oracle.search_patch(p, L, R, G, ox, oy, 2.0)
            assert abs(r["d"] - dstar) < 1e-9
            assert r["flags"] == 0, r["flags"]
            assert abs(r["E"][0] - c * c * P * P) < 1e-6
            assert abs(r["E"][1] - beta ** 2 * S) < 1e-6 * beta ** 2 * S
            recs.append(r)
    rec = np.array(recs, dtype=oracle.PATCH_DTYPE)
    # pooled reading: sqrt(sum E_k(0) / (N P^2)) = c exactly (a P^2 - 1 in
    # the denominator would give c * sqrt(64/63))
    assert abs(oracle.sigma_r(p, rec) - c) < 1e-9
    # a rejected patch with a large energy does not enter the sum
    bad = rec[:1].copy()
    bad["flags"] = oracle.F_SADDLE
    bad["E"][0, 0] = 1e6
    assert abs(oracle.sigma_r(p, np.concatenate([rec, bad])) - c) < 1e-9


def test_sigma_r_literal_is_population_std_of_kept_energies():
    p = oracle.make_params(sigma_r_mode="literal", sigma_r_floor=0.5)
    rec = np.zeros(3, dtype=oracle.PATCH_DTYPE)
    rec["E"][:, 0] = [10.0, 30.0, 5000.0]
    rec["flags"] = [0, 0, oracle.F_MOVED]
    # two kept patches: population std |E1 - E2| / 2 (the sample std would
    # be |E1 - E2| / sqrt(2))
    assert abs(oracle.sigma_r(p, rec) - 10.0) < 1e-12
    rec["flags"] = 0
    rec["E"][:, 0] = [1.0, 2.0, 6.0]
    assert abs(oracle.sigma_r(p, rec) - float(np.std([1.0, 2.0, 6.0]))) < 1e-12
    # equal energies: std 0, so the floor applies
    rec["E"][:, 0] = 7.0
    assert oracle.sigma_r(p, rec) == 0.5


# ---------------------------------------------------------------- depth (Eq. 13, Eq. 17)

def test_depth_is_inverse_disparity_and_variance_its_first_order_propagation():
    rng = np.random.default_rng(9)
    d = rng.uniform(0.5, 120.0, 400)
    v = rng.uniform(0.0, 3.0, 400)
    fb = 512.0 * 0.0042
    z, zv = oracle.depth(d, v, fb)
    # Eq. 13: z d = f b for every pixel
    np.testing.assert_allclose(z * d, fb, rtol=1e-15)
    # Eq. 17's depth factor is the squared slope of z(d): compare with the
    # slope of the oracle's own depth by central differences (step 1e-5 d)
    h = 1e-5 * d
    zp, _ = oracle.depth(d + h, None, fb)
    zm, _ = oracle.depth(d - h, None, fb)
    slope = (zp - zm) / (2 * h)
    np.testing.assert_allclose(zv, slope ** 2 * v, rtol=1e-8)
    # doubling the disparity divides the depth by 2 and its variance by 16
    z2, zv2 = oracle.depth(2 * d, v, fb)
    np.testing.assert_allclose(z2, z / 2, rtol=1e-15)
    np.testing.assert_allclose(zv2, zv / 16, rtol=1e-14)
    # d = f b gives unit depth and unchanged variance / (f b)^2
    z1, zv1 = oracle.depth(np.array([fb]), np.array([0.7]), fb)
    assert z1[0] == 1.0 and abs(zv1[0] - 0.7 / fb ** 2) < 1e-15


def test_depth_invalid_pixels_are_nan():
    d = np.array([np.nan, 0.0, -3.0, np.inf, 5.0])
    v = np.ones(5)
    z, zv = oracle.depth(d, v, 10.0)
    assert np.all(np.isnan(z[:4])) and np.all(np.isnan(zv[:4]))
    assert z[4] == 2.0 and zv[4] == 100.0 / 625.0


# ---------------------------------------------------------------- 8-bit storage

def test_round_u8_is_numpy_rint_clipped():
    # numpy's rint rounds half to even; the stored value is clipped to 0..255
    vals = np.concatenate([np.arange(-3, 259, 0.25), np.arange(0, 256) + 0.5,
                           np.random.default_rng(1).uniform(-10, 270, 3000)])
    for v in vals:
        assert oracle.round_u8(v) == float(np.clip(np.rint(v), 0, 255)), v


def test_pyr_down_u8_storage_rounds_each_level_and_gradient_is_exact_f16():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, (18, 22)).astype(float)
    a = oracle.pyr_down(img, "u8")
    b = np.clip(np.rint(oracle.pyr_down(img, "f64")), 0, 255)
    assert np.array_equal(a, b)
    # Sobel/8 of an 8-bit image is a multiple of 1/8 within +-127.5, which
    # binary16 holds exactly: the stored gradient equals the exact one
    np.testing.assert_array_equal(oracle.sobel_x(a, "u8"), oracle.sobel_x(a, "f64"))
