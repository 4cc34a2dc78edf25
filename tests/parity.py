"""Helpers that run the CUDA path and the FP64 oracle on the same seeded
inputs and compare them element by element.

Tolerances (the gate, stated once here and used by every parity test):
  * disparity: |d_gpu - d_oracle| <= 1e-3 px on >= 99.9% of the pixels valid
    in both, and <= 0.05 px on every such pixel not covered by a level-0
    patch whose discrete decision (kept / rejected, PDF exception) differs
    between the two sides in a way that changes its estimate ("flipped");
  * variance: relative difference <= 1e-3 on the same pixels;
  * validity masks equal outside the footprints of flipped patches;
  * the kept / rejected decision of each patch equal on >= 99.9% of the
    patches of every level (at most 2 disagreements on small levels).
Where a floating-point comparison decides an integer (a rejection flag),
both sides take it in their own arithmetic (FP32 on the GPU, FP64 in the
oracle); the rare disagreements are counted as flips and reported.
"""
from __future__ import annotations

import numpy as np

import oracle

D_TOL = 1e-3
D_FRAC = 0.999
D_MAX = 0.05
V_RTOL = 1e-3
# With the DIS weights of Eq. 2 the weight 1 / max(1, r^2) of a patch depends
# on its disparity through the residual r = I_r(x - d) - I_l(x) - mu, with
# d omega / omega = -2 g dd / r for |r| > 1 (g the image slope).  A disparity
# difference dd between the two arithmetics (up to ~1e-5 px, the disparity
# gate allows 1e-3) thus moves the weights by 2 |g| dd / |r|, about 1e-3 for
# |g| ~ 50 DN/px at |r| = 1, and V = sum omega^2 sig^2 / (sum omega)^2 by
# twice that: the variance gate of this mode is 5e-3.
V_RTOL_DIS = 5e-3

STORE_NAMES = {0: "f32", 1: "f16", 2: "u8"}


def oracle_params(gp, storage_override=None):
    """Oracle parameters equal to a GPU bdis_params (field by field)."""
    st = storage_override or STORE_NAMES[gp.storage]
    return oracle.make_params(
        patch=gp.patch, stride=gp.stride, levels=gp.levels, iters=gp.iters,
        sigma_s=gp.sigma_s, window_step=gp.window_step, conv_eps=gp.conv_eps,
        valid_gamma=gp.valid_gamma, pix_thresh=gp.pix_thresh, search_radius=gp.search_radius,
        sigma_r_mode={0: "pooled", 1: "literal", 2: "fixed"}[gp.sigma_r_mode],
        sigma_r_floor=gp.sigma_r_floor, sigma_r_fixed=gp.sigma_r_fixed, variance=gp.variance,
        pdf_iters=gp.pdf_iters, pdf_resid=gp.pdf_resid, storage=st, hess_eps=gp.hess_eps,
        use_sgmm=gp.use_sgmm, use_c2f=gp.use_c2f, weight_mode=gp.weight_mode,
        finest_level=gp.finest_level, fast_exp=gp.fast_exp)


def footprint(mask_patches, w, h, P, S):
    """Pixels covered by the patches marked in the (npy, npx) mask."""
    ox = oracle.origins(w, P, S)
    oy = oracle.origins(h, P, S)
    out = np.zeros((h, w), bool)
    for ky, kx in zip(*np.nonzero(mask_patches)):
        out[oy[ky]:oy[ky] + P, ox[kx]:ox[kx] + P] = True
    return out


def upsampled_footprint(mask_f, f, w, h):
    """Full-resolution pixels whose bilinear sources (level-f coordinate
    (x + 0.5) / 2^f - 0.5) include a pixel of the level-f mask."""
    if f == 0:
        return mask_f
    hf, wf = mask_f.shape
    s = 2.0 ** f

    def src(n, nf):
        X = np.clip((np.arange(n) + 0.5) / s - 0.5, 0, nf - 1)
        a = np.floor(X).astype(int)
        return a, np.minimum(a + 1, nf - 1)

    xa, xb = src(w, wf)
    ya, yb = src(h, hf)
    out = np.zeros((h, w), bool)
    for yy in (ya, yb):
        for xx in (xa, xb):
            out |= mask_f[yy][:, xx]
    return out


def compare_outputs(gp, o, disp, var, valid, rec_gpu0):
    """Final-output comparison; returns a metrics dict.  rec_gpu0: the GPU
    records of the finest processed level."""
    h, w = disp.shape
    P, S = gp.patch, gp.stride
    F = gp.finest_level
    rec_o0 = o["levels"][F]["patches"]
    flip = (rec_o0["flags"] == 0) != (rec_gpu0["flags"] == 0)
    both_kept = (rec_o0["flags"] == 0) & (rec_gpu0["flags"] == 0)
    if gp.variance:
        # a PDF exception on one side only counts when it changes sigma_k
        # (an exception and a fit capped at tau both give sigma_k = tau)
        s2o = rec_o0["sig2"].astype(np.float64)
        s2g = rec_gpu0["sig2"].astype(np.float64)
        differs = np.abs(s2g - s2o) > V_RTOL * np.maximum(s2o, 1e-12)
        flip |= both_kept & ((rec_o0["pdf_flags"] != 0) != (rec_gpu0["pdf_flags"] != 0)) & differs
    wf, hf = oracle.level_dim(w, F), oracle.level_dim(h, F)
    fp = upsampled_footprint(footprint(flip, wf, hf, P, S), F, w, h)
    vo = o["valid"]
    vg = valid.astype(bool)
    both = vo & vg
    dd = np.abs(disp.astype(np.float64) - o["disp"])
    m = dict(
        pixels=w * h, valid_oracle=int(vo.sum()), valid_gpu=int(vg.sum()),
        mask_mismatch=int((vo != vg).sum()), mask_mismatch_outside_flips=int(((vo != vg) & ~fp).sum()),
        flipped_patches=int(flip.sum()), patches=int(flip.size),
        frac_within_tol=float((dd[both] <= D_TOL).mean()) if both.any() else 1.0,
        max_dd=float(dd[both].max()) if both.any() else 0.0,
        max_dd_outside_flips=float(dd[both & ~fp].max()) if (both & ~fp).any() else 0.0,
        # reported, not gated: the pixels a flipped patch covers and the
        # largest differences there (a flip moves a whole footprint)
        flip_footprint_pixels=int(fp.sum()),
        max_dd_inside_flips=float(dd[both & fp].max()) if (both & fp).any() else 0.0,
    )
    if gp.variance:
        vv = np.abs(var.astype(np.float64) - o["var"]) / np.maximum(np.abs(o["var"]), 1e-12)
        sel = both & ~fp
        m["var_max_rel_outside_flips"] = float(vv[sel].max()) if sel.any() else 0.0
        m["var_max_rel_inside_flips"] = float(vv[both & fp].max()) if (both & fp).any() else 0.0
        m["var_frac_within"] = float((vv[both] <= V_RTOL).mean()) if both.any() else 1.0
    return m


def assert_gate(m, v_rtol=V_RTOL):
    assert m["frac_within_tol"] >= D_FRAC, m
    assert m["max_dd_outside_flips"] <= D_MAX, m
    assert m["mask_mismatch_outside_flips"] == 0, m
    assert m["flipped_patches"] <= max(2, int(0.001 * m["patches"])), m
    if "var_max_rel_outside_flips" in m:
        assert m["var_max_rel_outside_flips"] <= v_rtol, m


def compare_records(rg, ro):
    """Per-patch comparison at one level.  The decision that reaches the
    outputs is kept / rejected; which rejection bits are set on a patch both
    sides reject (e.g. a flat patch whose window energies tie) is reported
    but not gated."""
    fg, fo = rg["flags"], ro["flags"]
    decision_flips = (fg == 0) != (fo == 0)
    both = (fg == 0) & (fo == 0)
    dd = np.abs(rg["d"].astype(np.float64) - ro["d"])
    return dict(patches=int(fg.size), decision_flips=int(decision_flips.sum()),
                flag_bits_agree=float((fg == fo).mean()),
                kept_gpu=int((fg == 0).sum()), kept_oracle=int((fo == 0).sum()),
                d_frac_within=float((dd[both] <= D_TOL).mean()) if both.any() else 1.0,
                d_max=float(dd[both].max()) if both.any() else 0.0)
