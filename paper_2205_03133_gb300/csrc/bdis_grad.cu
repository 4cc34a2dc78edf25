// bdis_grad.cu -- adjoint kernels of the differentiable finest level.
//
// The function differentiated is the level-0 pipeline of a forward pass on
// float images with its discrete state frozen (kept patches, their initial
// estimates and inherited coarse probabilities, valid pixels, whether sigma_r
// sat at its floor):
//   g = Sobel-x/8(I_l); d_k solves F_k(d) = sum_i gt_i (I_r(x_i - d) - T_i) = 0
//   (Eq. 1); E_k(delta) window energies; sigma_r pooled; pi_k (Eq. 5-6);
//   rho_k = Gamma_0 pi_k + prop_k (Eq. 10-11); D = sum omega d / sum omega (Eq. 12).
// The loss is L1 photometric reprojection plus lambda times first-order
// smoothness, both summed over valid pixels and divided by w h.  The patch
// adjoint is the implicit-function rule dd/dtheta = -(dF/dd)^-1 dF/dtheta.
//
// Image gradients are accumulated with float atomics (the sample positions
// of different patches overlap), so their last bits depend on the order in
// which the hardware serves the atomics.
#include "bdis_device.cuh"

namespace bdis {
namespace {

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// subgradient of |D_p - D_q|: 0 at a tie (pixels covered by the same patches
// along one axis have equal D in exact arithmetic; a difference within
// 1e-6 (|D_p| + |D_q|) is a tie)
__device__ __forceinline__ float sgn_tie(float dp, float dq) {
    const float a = dp - dq;
    return fabsf(a) <= 1e-6f * (fabsf(dp) + fabsf(dq)) ? 0.f : sgnf(a);
}

// Sample of a row at x - d = base + t (clamped linear interpolation), its
// taps and the right-sided slope (0 where the coordinate is clamped).
struct Tap {
    int x0, x1;
    float t, v, slope;
};

__device__ __forceinline__ Tap tap_row(const float *__restrict__ row, int w, int base, float t) {
    Tap q;
    if (base < 0) {
        q.x0 = q.x1 = 0;
        q.t = 0.f;
        q.v = __ldg(row);
        q.slope = 0.f;
    } else if (base >= w - 1) {
        q.x0 = q.x1 = w - 1;
        q.t = 0.f;
        q.v = __ldg(row + w - 1);
        q.slope = 0.f;
    } else {
        q.x0 = base;
        q.x1 = base + 1;
        q.t = t;
        const float a = __ldg(row + base), b = __ldg(row + base + 1);
        q.v = fmaf(t, b - a, a);
        q.slope = b - a;
    }
    return q;
}

// tap of the sample x - d of pixel x
__device__ __forceinline__ Tap tap_at(const float *__restrict__ row, int w, int x, float d) {
    int off;
    float t;
    split_shift(d, off, t);
    return tap_row(row, w, x + off, t);
}

__device__ __forceinline__ int find_pair_g(const GradDesc *d, int n, int unit, int kind) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].work_begin[kind] <= unit) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float ldg_grad(const GradDesc &g, int row, int col) {
    const size_t i = (size_t)row * g.gpitch + col;
    return g.gtype == E_F16 ? __half2float(__ldg((const __half *)g.G + i))
                            : __ldg((const float *)g.G + i);
}

__device__ __forceinline__ float block_sum256(float v, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// ---------------------------------------------------------------- loss (K6)

// Per pixel: loss terms, dL/dD, the direct dL/dI_l (written) and dL/dI_r
// (scattered into a zeroed buffer); one loss partial per block.
__global__ void __launch_bounds__(256) k_loss(GradArgs a) {
    __shared__ float red[32];
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const int pi = find_pair_g(a.descs, a.npairs, unit, G_PIX);
        const GradDesc &g = a.descs[pi];
        const int local = unit - g.work_begin[G_PIX];
        const int idx = local * blockDim.x + threadIdx.x;
        float part = 0.f;
        if (idx < g.w * g.h) {
            const int x = idx % g.w, y = idx / g.w;
            const float inv = 1.f / ((float)g.w * (float)g.h);
            float gD = 0.f, gLd = 0.f;
            if (g.valid[idx]) {
                const float D = g.disp[idx];
                const float *rrow = g.R + (size_t)y * g.pitch;
                const Tap q = tap_at(rrow, g.w, x, D);
                const float r = q.v - __ldg(g.L + (size_t)y * g.pitch + x);
                const float s = sgnf(r) * inv;
                part += fabsf(r);
                gD -= s * q.slope;
                gLd = -s;
                atomicAdd(g.gR + (size_t)y * g.w + q.x0, s * (1.f - q.t));
                atomicAdd(g.gR + (size_t)y * g.w + q.x1, s * q.t);
                const float li = a.lambda * inv;
                if (x + 1 < g.w && g.valid[idx + 1]) {
                    part += a.lambda * fabsf(D - g.disp[idx + 1]);
                    gD += li * sgn_tie(D, g.disp[idx + 1]);
                }
                if (y + 1 < g.h && g.valid[idx + g.w]) {
                    part += a.lambda * fabsf(D - g.disp[idx + g.w]);
                    gD += li * sgn_tie(D, g.disp[idx + g.w]);
                }
                if (x > 0 && g.valid[idx - 1]) gD += li * sgn_tie(D, g.disp[idx - 1]);
                if (y > 0 && g.valid[idx - g.w]) gD += li * sgn_tie(D, g.disp[idx - g.w]);
            }
            g.gDisp[idx] = gD;
            g.gL[(size_t)y * g.w + x] = gLd;
        }
        const float bs = block_sum256(part, red);
        if (threadIdx.x == 0) g.loss_part[local] = bs;
    }
}

// Zeroes every pair's dL/dI_r buffer (w h floats) before k_loss scatters
// into it: one launch over the pixels of all pairs.
__global__ void __launch_bounds__(256) k_zero_gr(GradArgs a) {
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_PIX)];
        const int idx = (unit - g.work_begin[G_PIX]) * blockDim.x + threadIdx.x;
        if (idx < g.w * g.h) g.gR[idx] = 0.f;
    }
}

// One block per pair: loss = sum of the partials / (w h), in a fixed order.
__global__ void __launch_bounds__(256) k_loss_reduce(GradArgs a) {
    __shared__ float red[32];
    for (int pair = blockIdx.x; pair < a.npairs; pair += gridDim.x) {
        const GradDesc &g = a.descs[pair];
        const int n = (g.w * g.h + 255) / 256;
        float s = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += g.loss_part[i];
        const float t = block_sum256(s, red);
        if (threadIdx.x == 0 && g.loss) *g.loss = t / ((float)g.w * (float)g.h);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- fusion adjoint

// Per pixel, divided by the weight sum saved by the forward's fusion:
// level 0 dL/dD (0 at invalid pixels), coarser levels dL/dQ.
__global__ void __launch_bounds__(256) k_bwd_pix(GradArgs a) {
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_PIX)];
        const int idx = (unit - g.work_begin[G_PIX]) * blockDim.x + threadIdx.x;
        if (idx >= g.w * g.h) continue;
        const float sw = __ldg(g.wsum + idx);
        float v = 0.f;
        if (a.level == 0) {
            if (g.valid[idx]) v = sw > 0.f ? g.gDisp[idx] / sw : 0.f;
        } else {
            v = sw > 0.f ? g.gQ[idx] / sw : 0.f;
        }
        g.gDw[idx] = v;
    }
}

// Per kept patch: dL/dd_k = sum_x gDw rho_k M, dL/drho_k = sum_x gDw M (d_k - D)
// at level 0 (D = sum omega d / sum omega, Eq. 12); at coarser levels, from the
// fused probability Q = sum omega rho / sum omega, dL/drho_k = sum_x gQw M (2 rho_k
// - Q).  Then dL/dpi_k = Gamma_n dL/drho_k, the bilinear transpose of rho's
// coarse term (Eq. 10) into the next level's dL/dQ, and the patch's share of
// dL/dsigma_r (block partials).  A group of lanes per patch, lane = patch row,
// so the pixel reads are row segments.
template <int P>
__device__ __forceinline__ void bwd_dens_unit(const GradArgs &a, int unit, float *red) {
    constexpr int G = P <= 8 ? 8 : 16;
    const int S = a.S;
    const int pi = find_pair_g(a.descs, a.npairs, unit, G_GROUP);
    const GradDesc &g = a.descs[pi];
    const int local = unit - g.work_begin[G_GROUP];
    const int ngrp = blockDim.x / G;
    const int gl = threadIdx.x & (G - 1);
    const int k = local * ngrp + (int)threadIdx.x / G;
    const int np = g.npx * g.npy;
    const int kk = min(k, np - 1);
    const bdis_patch_record &rc = g.rec[kk];
    const bool kept = k < np && rc.flags == 0u;
    float gd = 0.f, grho = 0.f;
    if (kept && gl < P) {
        const int ox = origin(kk % g.npx, g.w, P, S, g.kxreg);
        const int oy = origin(kk / g.npx, g.h, P, S, g.kyreg);
        const float my = a.use_sgmm ? a.m[gl] : 1.f;
        const size_t row = (size_t)(oy + gl) * g.w + ox;
        const bool fine = a.level == 0;
        const float *mp = fine ? g.disp : g.Q;
        float wv[P], dv[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {  // all loads first
            wv[c] = __ldg(g.gDw + row + c);
            dv[c] = __ldg(mp + row + c);
        }
#pragma unroll
        for (int c = 0; c < P; ++c) {
            if (wv[c] == 0.f) continue;  // invalid pixel (disp may be NaN)
            const float M = my * (a.use_sgmm ? a.m[c] : 1.f);
            if (fine) {
                gd = fmaf(wv[c] * rc.rho, M, gd);
                grho = fmaf(wv[c] * M, rc.d - dv[c], grho);
            } else {
                grho = fmaf(wv[c] * M, 2.f * rc.rho - dv[c], grho);
            }
        }
    }
    gd = group_sum<G>(gd);
    grho = group_sum<G>(grho);
    float gsr = 0.f, cnt = 0.f;
    if (gl == 0 && k < np) {
        float gpi = 0.f;
        if (kept) {
            gpi = a.use_c2f ? a.gamma_w * grho : grho;
            // rho_k = Gamma_n pi_k + Q^(n+1)(centre): bilinear transpose
            if (a.use_c2f && g.gQn != nullptr && grho != 0.f) {
                const float cx = (float)origin(kk % g.npx, g.w, P, S, g.kxreg) + 0.5f * (float)(P - 1);
                const float cy = (float)origin(kk / g.npx, g.h, P, S, g.kyreg) + 0.5f * (float)(P - 1);
                float X = (cx + 0.5f) * 0.5f - 0.5f, Y = (cy + 0.5f) * 0.5f - 0.5f;
                X = fminf(fmaxf(X, 0.f), (float)(g.wn - 1));
                Y = fminf(fmaxf(Y, 0.f), (float)(g.hn - 1));
                const int x0 = (int)floorf(X), y0 = (int)floorf(Y);
                const int x1 = min(x0 + 1, g.wn - 1), y1 = min(y0 + 1, g.hn - 1);
                const float fx = X - (float)x0, fy = Y - (float)y0;
                atomicAdd(g.gQn + (size_t)y0 * g.wn + x0, grho * (1.f - fx) * (1.f - fy));
                atomicAdd(g.gQn + (size_t)y0 * g.wn + x1, grho * fx * (1.f - fy));
                atomicAdd(g.gQn + (size_t)y1 * g.wn + x0, grho * (1.f - fx) * fy);
                atomicAdd(g.gQn + (size_t)y1 * g.wn + x1, grho * fx * fy);
            }
            // dpi/dsigma_r = (2 pi / sigma_r) sum_i pi_i e_i
            const float sr = __ldg(g.sigma_r);
            const float S2 = 2.f * sr * sr * (float)(kWindow * kWindow);
            float e[5], Z = 1.f;
            e[0] = 0.f;
#pragma unroll
            for (int i = 1; i < 5; ++i) {
                e[i] = -rc.E[i] / S2;
                Z += expf(e[i]);
            }
            float se = 0.f;
#pragma unroll
            for (int i = 1; i < 5; ++i) se += expf(e[i]) / Z * e[i];
            gsr = gpi * (2.f * rc.pi / sr) * se;
            cnt = 1.f;
        } else {
            gd = 0.f;
        }
        g.gd[k] = gd;
        g.gpi[k] = gpi;
    }
    const float s1 = block_sum256(gsr, red);
    const float s2 = block_sum256(cnt, red);
    if (threadIdx.x == 0) {
        g.sig_part[2 * local] = s1;
        g.sig_part[2 * local + 1] = s2;
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_bwd_dens(GradArgs a) {
    __shared__ float red[32];
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) bwd_dens_unit<P>(a, unit, red);
}

// One block per pair: dL/dsigma_r -> the coefficient added to every kept
// patch's dL/dE(0) (pooled sigma_r: dsigma_r/dE_k(0) = 1/(2 sigma_r N P^2)).
__global__ void __launch_bounds__(256) k_bwd_sigma(GradArgs a) {
    __shared__ float red[32];
    for (int pair = blockIdx.x; pair < a.npairs; pair += gridDim.x) {
        const GradDesc &g = a.descs[pair];
        const int ngrp = 256 / (a.P <= 8 ? 8 : 16);
        const int n = (g.npx * g.npy + ngrp - 1) / ngrp;
        float s = 0.f, c = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            s += g.sig_part[2 * i];
            c += g.sig_part[2 * i + 1];
        }
        const float S = block_sum256(s, red);
        const float Cn = block_sum256(c, red);
        if (threadIdx.x == 0) {
            const float sr = *g.sigma_r;
            const bool free_sr = a.sigma_r_mode == BDIS_SIGMA_R_POOLED && sr > a.sigma_r_floor &&
                                 Cn > 0.f;
            *g.coefE0 = free_sr ? S / (2.f * sr * Cn * (float)(a.P * a.P)) : 0.f;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- patch adjoint

// A group of G lanes per kept patch, lane = patch row (as in the search).
// Window energies and the implicit-function rule through F_k.
// Right-image values one lane stages for its patch row: the columns
// lo .. lo + P + kSegExtra - 1 (lo = leftmost tap of the window), clamped to
// the image like every sample.
constexpr int kSegExtra = 6;
template <int P>
__host__ __device__ constexpr int seg_stride() { return (P + kSegExtra) | 1; }  // odd: distinct banks

// Per-row tap of the staged segment at column j + S (S = offset of the
// window sample's integer part from lo): value and right-sided slope, equal
// to tap_row() on the image (a clamped tap reads equal neighbours: slope 0).
__device__ __forceinline__ void seg_tap(const float *seg, int k, float t, float &v, float &slope) {
    const float a = seg[k], b = seg[k + 1];
    slope = b - a;
    v = fmaf(t, slope, a);
}

// dL/dE_i of a kept patch from dL/dpi_k (through the window posterior) and
// the sigma_r coefficient of E(0).
__device__ __forceinline__ void grad_energies(const GradDesc &g, const bdis_patch_record &rc,
                                              int kk, float gE[5]) {
    const float sr = __ldg(g.sigma_r);
    const float S2 = 2.f * sr * sr * (float)(kWindow * kWindow);
    float pik[5], Z = 1.f;
    pik[0] = 1.f;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        pik[i] = expf(-rc.E[i] / S2);
        Z += pik[i];
    }
    const float gpi = g.gpi[kk];
    gE[0] = __ldg(g.coefE0);
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        gE[i] = gpi * rc.pi * (pik[i] / Z) / S2;
        gE[0] -= gE[i];
    }
}

// Window step 1/2: the samples of the row at d + delta for delta in
// {0, -1/2, +1/2, -1, +1} come from two clamped value rows, v0 (columns
// base0 - 1 .. base0 + P + 1, phase t0 of d) and vp (columns basep ..
// basep + P + 1, phase tp of d + 1/2): d -+ 1 is the d row one column over
// and d - 1/2 is the d + 1/2 row one column over.  Every tap, slope and tap
// adjoint then has a compile-time register index.
template <int P, int G>
__device__ __forceinline__ void patch_adjoint_half(const GradDesc &g, const bdis_patch_record &rc,
                                                   int k, int kk, bool active_patch, int gl,
                                                   bool row_on, int ox, int row,
                                                   const float *Rrow, const float (&T)[P],
                                                   const float (&gt)[P]) {
    constexpr float invN = 1.f / (float)(P * P);
    const float d = rc.d;
    int off0, offp;
    float t0, tp;
    split_shift(d, off0, t0);
    split_shift(d + 0.5f, offp, tp);
    const int b0 = ox + off0 - 1;
    // the d + 1/2 row starts at b0 + 1 (offp == off0) or b0 (offp == off0 - 1):
    // its values are the d row's, one column over or not
    const bool right = offp == off0;
    float v0[P + 3], vp[P + 2];
#pragma unroll
    for (int q = 0; q < P + 3; ++q) v0[q] = __ldg(Rrow + clampi(b0 + q, 0, g.w - 1));
#pragma unroll
    for (int q = 0; q < P + 2; ++q) vp[q] = right ? v0[q + 1] : v0[q];
    // tap (value, slope) of offset i at pixel j: row, first index, phase
    auto tap = [&](int i, int j, float &v, float &sl) {
        const float *r = (i == 1 || i == 2) ? vp : v0;
        const int q = i == 0 ? j + 1 : i == 1 ? j + 1 : i == 2 ? j : i == 3 ? j + 2 : j;
        const float t = (i == 1 || i == 2) ? tp : t0;
        sl = r[q + 1] - r[q];
        v = fmaf(t, sl, r[q]);
    };
    // means of the window residuals (the centre one is the residual mean of
    // the solve) and dF/dd
    float abar[5], dEdd[5], fd = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float sa = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            float v, sl;
            tap(i, j, v, sl);
            sa += row_on ? v - T[j] : 0.f;
            if (i == 0) fd -= gt[j] * sl;
        }
        abar[i] = group_sum<G>(sa) * invN;
    }
    const float mres = abar[0];
    const float Fd = group_sum<G>(fd);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float sd = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            float v, sl;
            tap(i, j, v, sl);
            sd += row_on ? 2.f * (v - T[j] - abar[i]) * (-sl) : 0.f;
        }
        dEdd[i] = group_sum<G>(sd);
    }
    float gE[5];
    grad_energies(g, rc, kk, gE);
    float gdt = g.gd[kk];
#pragma unroll
    for (int i = 0; i < 5; ++i) gdt = fmaf(gE[i], dEdd[i], gdt);
    const float vF = -gdt / Fd;
    // a rejected patch does not reach the output: its gradient is 0
    if (k < g.npx * g.npy && gl == 0 && g.gPatch) g.gPatch[kk] = active_patch ? gdt : 0.f;
    const int P2 = P * P;
    float *cLrow = g.cpatch + ((size_t)kk * 2 * P + (row_on ? gl : 0)) * P;
    float *cGrow = cLrow + P2;
    if (k < g.npx * g.npy && row_on && !active_patch) {
#pragma unroll
        for (int j = 0; j < P; ++j) {
            cLrow[j] = 0.f;
            cGrow[j] = 0.f;
        }
    }
    if (!(active_patch && row_on)) return;
    float a0[P + 3], ap[P + 3];
#pragma unroll
    for (int q = 0; q < P + 3; ++q) a0[q] = ap[q] = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        float tsum = 0.f, v00 = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float v, sl;
            tap(i, j, v, sl);
            if (i == 0) v00 = v;
            const float c = gE[i] * 2.f * (v - T[j] - abar[i]);
            tsum += c;
            const int q = i == 0 ? j + 1 : i == 1 ? j + 1 : i == 2 ? j : i == 3 ? j + 2 : j;
            const float t = (i == 1 || i == 2) ? tp : t0;
            float *acc = (i == 1 || i == 2) ? ap : a0;
            acc[q] = fmaf(c, 1.f - t, acc[q]);
            acc[q + 1] = fmaf(c, t, acc[q + 1]);
        }
        const float cF = vF * gt[j];
        a0[j + 1] = fmaf(cF, 1.f - t0, a0[j + 1]);
        a0[j + 2] = fmaf(cF, t0, a0[j + 2]);
        cLrow[j] = -tsum - cF;
        cGrow[j] = vF * ((v00 - T[j]) - mres);
    }
    // one atomic per column: the d + 1/2 row starts one column right of
    // the d row's first column (offp == off0) or at it (offp == off0 - 1,
    // the half pixel moving the split left), so its adjoints add onto the
    // d row's columns b0 .. b0 + P + 2.  A clamped column's weight lands on
    // the edge column, as in tap_row().
    float *gRrow = g.gR + (size_t)row * g.w;
#pragma unroll
    for (int c = 0; c < P + 3; ++c) {
        const float pr = c >= 1 ? ap[c - 1] : 0.f;
        const float pl = c < P + 2 ? ap[c] : 0.f;
        const float v = a0[c] + (right ? pr : pl);
        if (v != 0.f) atomicAdd(gRrow + clampi(b0 + c, 0, g.w - 1), v);
    }
}

// P <= 8: three blocks per SM (80 registers, a few spilled values) hide more
// of the record and row-load latency than two without spills; larger patches
// keep two (128 registers).
template <int P>
__global__ void __launch_bounds__(256, (P <= 8 ? 3 : 2)) k_bwd_patch(GradArgs a) {
    constexpr int G = P <= 8 ? 8 : 16;
    constexpr int N = P * P;
    constexpr int SEGN = P + kSegExtra;
    constexpr float invN = 1.f / (float)N;
    extern __shared__ float bsm[];
    float *seg = bsm + (size_t)threadIdx.x * 2 * seg_stride<P>();  // lane-private
    float *acc = seg + seg_stride<P>();
    const int tid = threadIdx.x;
    const int gl = tid & (G - 1);
    const int grp = tid / G;
    const int ngrp = blockDim.x / G;
    const bool row_on = gl < P;
    const float h = a.window_step;
    const float dl[5] = {0.f, -h, h, -2.f * h, 2.f * h};
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_GROUP)];
        const int k = (unit - g.work_begin[G_GROUP]) * ngrp + grp;
        const bool active_patch = k < g.npx * g.npy && g.rec[min(k, g.npx * g.npy - 1)].flags == 0u;
        const int kk = min(k, g.npx * g.npy - 1);
        const bdis_patch_record rc = g.rec[kk];
        const int ox = origin(kk % g.npx, g.w, P, a.S, g.kxreg);
        const int oy = origin(kk / g.npx, g.h, P, a.S, g.kyreg);
        const int row = oy + (row_on ? gl : 0);
        const float *Lrow = g.L + (size_t)row * g.pitch + ox;
        const float *Rrow = g.R + (size_t)row * g.pitch;
        float T[P], gt[P];
        float gs = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            T[j] = __ldg(Lrow + j);
            gt[j] = row_on ? ldg_grad(g, row, ox + j) : 0.f;
            gs += gt[j];
        }
        const float gbar = group_sum<G>(gs) * invN;
#pragma unroll
        for (int j = 0; j < P; ++j) gt[j] = row_on ? gt[j] - gbar : 0.f;
        if (h == 0.5f) {
            patch_adjoint_half<P, G>(g, rc, k, kk, active_patch, gl, row_on, ox, row, Rrow, T, gt);
            continue;
        }
        const float d = rc.d;
        // every sample of the row at offset delta_i is split_shift(d + delta_i):
        // taps ox + j + off_i and the next column, weights (1 - t_i), t_i
        int offs[5], sh[5];
        float ts[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) split_shift(d + dl[i], offs[i], ts[i]);
        int omin = offs[0], omax = offs[0];
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            omin = min(omin, offs[i]);
            omax = max(omax, offs[i]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) sh[i] = offs[i] - omin;
        const int lo = ox + omin;
        // taps reach column j + sh_i + 1 <= P + (omax - omin); a wider
        // window (window_step > 1.25) takes the per-tap path below
        const bool staged = omax - omin <= kSegExtra - 1;
        if (staged && row_on) {
#pragma unroll
            for (int q = 0; q < SEGN; ++q) {
                seg[q] = __ldg(Rrow + clampi(lo + q, 0, g.w - 1));
                acc[q] = 0.f;
            }
        }
        auto tap = [&](int i, int j, float &v, float &slope) {
            if (staged) {
                seg_tap(seg, j + sh[i], ts[i], v, slope);
            } else {
                const Tap q = tap_row(Rrow, g.w, ox + j + offs[i], ts[i]);
                v = q.v;
                slope = q.slope;
            }
        };
        // residual at d, and dF/dd
        float sres = 0.f, fd = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            float v, sl;
            tap(0, j, v, sl);
            sres += row_on ? v - T[j] : 0.f;
            fd -= gt[j] * sl;
        }
        const float mres = group_sum<G>(sres) * invN;
        const float Fd = group_sum<G>(fd);
        // dE_i/dd and the means of the window residuals
        float abar[5], dEdd[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float sa = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                float v, sl;
                tap(i, j, v, sl);
                sa += row_on ? v - T[j] : 0.f;
            }
            abar[i] = group_sum<G>(sa) * invN;
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float sd = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                float v, sl;
                tap(i, j, v, sl);
                sd += row_on ? 2.f * (v - T[j] - abar[i]) * (-sl) : 0.f;
            }
            dEdd[i] = group_sum<G>(sd);
        }
        // dL/dE_i from dL/dpi_k and sigma_r
        const float sr = __ldg(g.sigma_r);
        const float S2 = 2.f * sr * sr * (float)(kWindow * kWindow);
        float pik[5], Z = 1.f;
        pik[0] = 1.f;
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            pik[i] = expf(-rc.E[i] / S2);
            Z += pik[i];
        }
        const float gpi = g.gpi[kk];
        float gE[5];
        gE[0] = __ldg(g.coefE0);
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            gE[i] = gpi * rc.pi * (pik[i] / Z) / S2;
            gE[0] -= gE[i];
        }
        float gdt = g.gd[kk];
#pragma unroll
        for (int i = 0; i < 5; ++i) gdt = fmaf(gE[i], dEdd[i], gdt);
        const float vF = -gdt / Fd;
        // a rejected patch does not reach the output: its gradient is 0
        if (k < g.npx * g.npy && gl == 0 && g.gPatch) g.gPatch[kk] = active_patch ? gdt : 0.f;
        // this row's template and gradient-image terms (gathered per pixel
        // by k_bwd_gather); a rejected patch contributes zeros
        float *cLrow = g.cpatch + ((size_t)kk * 2 * P + (row_on ? gl : 0)) * P;
        float *cGrow = cLrow + P * P;
        if (k < g.npx * g.npy && row_on && !active_patch) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                cLrow[j] = 0.f;
                cGrow[j] = 0.f;
            }
        }
        if (!(active_patch && row_on)) continue;
        // scatter: window energies and the solve F into the right image (the
        // adjoint of each tap), the template into the left image, the solve
        // into the gradient image
        float *gRrow = g.gR + (size_t)row * g.w;
        if (staged) {
            // per-row sums over the staged columns, then one atomic per column
#pragma unroll
            for (int j = 0; j < P; ++j) {
                float tsum = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    float v, sl;
                    seg_tap(seg, j + sh[i], ts[i], v, sl);
                    const float c = gE[i] * 2.f * (v - T[j] - abar[i]);
                    acc[j + sh[i]] = fmaf(c, 1.f - ts[i], acc[j + sh[i]]);
                    acc[j + sh[i] + 1] = fmaf(c, ts[i], acc[j + sh[i] + 1]);
                    tsum += c;
                }
                float v0, sl0;
                seg_tap(seg, j + sh[0], ts[0], v0, sl0);
                const float cF = vF * gt[j];
                acc[j + sh[0]] = fmaf(cF, 1.f - ts[0], acc[j + sh[0]]);
                acc[j + sh[0] + 1] = fmaf(cF, ts[0], acc[j + sh[0] + 1]);
                cLrow[j] = -tsum - cF;
                cGrow[j] = vF * ((v0 - T[j]) - mres);
            }
            // a clamped tap's weight lands on the edge column, as in tap_row()
#pragma unroll
            for (int q = 0; q < SEGN; ++q)
                if (acc[q] != 0.f) atomicAdd(gRrow + clampi(lo + q, 0, g.w - 1), acc[q]);
        } else {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                float tsum = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const Tap q = tap_at(Rrow, g.w, ox + j, d + dl[i]);
                    const float c = gE[i] * 2.f * (q.v - T[j] - abar[i]);
                    atomicAdd(gRrow + q.x0, c * (1.f - q.t));
                    atomicAdd(gRrow + q.x1, c * q.t);
                    tsum += c;
                }
                const Tap q = tap_at(Rrow, g.w, ox + j, d);
                atomicAdd(gRrow + q.x0, vF * gt[j] * (1.f - q.t));
                atomicAdd(gRrow + q.x1, vF * gt[j] * q.t);
                cLrow[j] = -tsum - vF * gt[j];
                cGrow[j] = vF * ((q.v - T[j]) - mres);
            }
        }
    }
}

// dL/dg -> dL/dI_l through Sobel-x/8 (reflect-101), scattered.
// Per pixel: the template and gradient-image terms of the covering patches
// (no atomics): gG = sum of the gradient-image terms, gL += sum of the
// template terms.
__global__ void __launch_bounds__(256) k_bwd_gather(GradArgs a) {
    const int P = a.P, S = a.S;
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_PIX)];
        const int idx = (unit - g.work_begin[G_PIX]) * blockDim.x + threadIdx.x;
        if (idx >= g.w * g.h) continue;
        const int y = idx / g.w, x = idx - y * g.w;
        // x, y < 2^22: exact divisions by S through its rounded reciprocal
        const float rS = recip(S);
        const int kxlo = x - P + 1 > 0 ? udiv_small(x - P + S, rS) : 0;
        const int kxhi = min(g.kxreg - 1, udiv_small(x, rS));
        const bool kxext = g.npx > g.kxreg && x >= g.w - P;
        const int kylo = y - P + 1 > 0 ? udiv_small(y - P + S, rS) : 0;
        const int kyhi = min(g.kyreg - 1, udiv_small(y, rS));
        const bool kyext = g.npy > g.kyreg && y >= g.h - P;
        const int nkx = kxhi - kxlo + 1 + (kxext ? 1 : 0);
        const int nky = kyhi - kylo + 1 + (kyext ? 1 : 0);
        float sL = 0.f, sG = 0.f;
        for (int iy = 0; iy < nky; ++iy) {
            const int ky = (kylo + iy <= kyhi) ? kylo + iy : g.npy - 1;
            const int r = y - origin(ky, g.h, P, S, g.kyreg);
            for (int ix = 0; ix < nkx; ++ix) {
                const int kx = (kxlo + ix <= kxhi) ? kxlo + ix : g.npx - 1;
                const int c = x - origin(kx, g.w, P, S, g.kxreg);
                const float *cp = g.cpatch + ((size_t)(ky * g.npx + kx) * 2 * P + r) * P + c;
                sL += __ldg(cp);
                sG += __ldg(cp + P * P);
            }
        }
        g.gG[idx] = sG;
        g.gL[idx] += sL;
    }
}

// Sources of fine index x in the blur-and-decimate of a row of n pixels into
// nc coarse ones (coarse X reads fine refl(2X + i), i = -2..2, weight
// k[i + 2]): up to 3 (coarse index, weight) pairs.  Away from the borders
// they follow from the parity of x; near a border the reflected taps are
// enumerated.
__device__ __forceinline__ int pyr_sources(int x, int n, int nc, int (&X)[4], float (&wt)[4]) {
    if (x >= 3 && x <= n - 4) {
        if ((x & 1) == 0) {
            X[0] = x / 2 - 1; wt[0] = 1.f / 16;
            X[1] = x / 2;     wt[1] = 6.f / 16;
            X[2] = x / 2 + 1; wt[2] = 1.f / 16;
            return 3;
        }
        X[0] = (x - 1) / 2; wt[0] = 4.f / 16;
        X[1] = (x + 1) / 2; wt[1] = 4.f / 16;
        return 2;
    }
    const float k5[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
    int cnt = 0;
    const int lo = max(0, x / 2 - 2), hi = min(nc - 1, x / 2 + 2);
    for (int c = lo; c <= hi; ++c) {
        float s = 0.f;
#pragma unroll
        for (int i = -2; i <= 2; ++i)
            if (refl(2 * c + i, n) == x) s += k5[i + 2];
        if (s != 0.f && cnt < 4) {
            X[cnt] = c;
            wt[cnt] = s;
            ++cnt;
        }
    }
    return cnt;
}

// Pyramid transpose (a gather, no atomics): the image gradients of level n+1
// flow back to level n through the blur-and-decimate that made level n+1.
__global__ void __launch_bounds__(256) k_bwd_pyr(GradArgs a) {
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_PIX)];
        const int idx = (unit - g.work_begin[G_PIX]) * blockDim.x + threadIdx.x;
        if (idx >= g.w * g.h || g.gLc == nullptr) continue;
        const int x = idx % g.w, y = idx / g.w;
        int Xs[4], Ys[4];
        float wx[4], wy[4];
        const int nx = pyr_sources(x, g.w, g.wn, Xs, wx);
        const int ny = pyr_sources(y, g.h, g.hn, Ys, wy);
        float sL = 0.f, sR = 0.f;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t o = (size_t)Ys[j] * g.wn + Xs[i];
                const float wgt = wy[j] * wx[i];
                sL = fmaf(wgt, __ldg(g.gLc + o), sL);
                sR = fmaf(wgt, __ldg(g.gRc + o), sR);
            }
        g.gL[idx] += sL;
        g.gR[idx] += sR;
    }
}

__global__ void __launch_bounds__(256) k_bwd_sobel(GradArgs a) {
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const GradDesc &g = a.descs[find_pair_g(a.descs, a.npairs, unit, G_PIX)];
        const int idx = (unit - g.work_begin[G_PIX]) * blockDim.x + threadIdx.x;
        if (idx >= g.w * g.h) continue;
        const float v = g.gG[idx];
        if (v == 0.f) continue;
        const int x = idx % g.w, y = idx / g.w;
        const int xp = refl(x + 1, g.w), xm = refl(x - 1, g.w);
#pragma unroll
        for (int j = -1; j <= 1; ++j) {
            const float wgt = (j == 0 ? 2.f : 1.f) * 0.125f * v;
            float *row = g.gL + (size_t)refl(y + j, g.h) * g.w;
            atomicAdd(row + xp, wgt);
            atomicAdd(row + xm, -wgt);
        }
    }
}

int grad_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int ggrid(int total) {
    const int cap = grad_sms() * 8;
    return total < 1 ? 1 : (total < cap ? total : cap);
}

}  // namespace

cudaError_t launch_loss(const GradArgs &a, cudaStream_t s) {
    k_zero_gr<<<ggrid(a.total), 256, 0, s>>>(a);
    cudaError_t z = cudaGetLastError();
    if (z != cudaSuccess) return z;
    k_loss<<<ggrid(a.total), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss_reduce<<<ggrid(a.npairs), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_pix(const GradArgs &a, cudaStream_t s) {
    k_bwd_pix<<<ggrid(a.total), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_dens(const GradArgs &a, cudaStream_t s) {
    const int grid = ggrid(a.total);
    switch (a.P) {
        case 4: k_bwd_dens<4><<<grid, 256, 0, s>>>(a); break;
        case 5: k_bwd_dens<5><<<grid, 256, 0, s>>>(a); break;
        case 6: k_bwd_dens<6><<<grid, 256, 0, s>>>(a); break;
        case 7: k_bwd_dens<7><<<grid, 256, 0, s>>>(a); break;
        case 8: k_bwd_dens<8><<<grid, 256, 0, s>>>(a); break;
        case 9: k_bwd_dens<9><<<grid, 256, 0, s>>>(a); break;
        case 10: k_bwd_dens<10><<<grid, 256, 0, s>>>(a); break;
        case 11: k_bwd_dens<11><<<grid, 256, 0, s>>>(a); break;
        case 12: k_bwd_dens<12><<<grid, 256, 0, s>>>(a); break;
        case 13: k_bwd_dens<13><<<grid, 256, 0, s>>>(a); break;
        case 14: k_bwd_dens<14><<<grid, 256, 0, s>>>(a); break;
        case 15: k_bwd_dens<15><<<grid, 256, 0, s>>>(a); break;
        case 16: k_bwd_dens<16><<<grid, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bwd_sigma<<<ggrid(a.npairs), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_bwd_patch_p(const GradArgs &a, int grid, cudaStream_t s) {
    const size_t smem = sizeof(float) * 256 * 2 * seg_stride<P>();
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_bwd_patch<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_bwd_patch<P><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_patch(const GradArgs &a, cudaStream_t s) {
    const int grid = ggrid(a.total);
    switch (a.P) {
        case 4: return launch_bwd_patch_p<4>(a, grid, s);
        case 5: return launch_bwd_patch_p<5>(a, grid, s);
        case 6: return launch_bwd_patch_p<6>(a, grid, s);
        case 7: return launch_bwd_patch_p<7>(a, grid, s);
        case 8: return launch_bwd_patch_p<8>(a, grid, s);
        case 9: return launch_bwd_patch_p<9>(a, grid, s);
        case 10: return launch_bwd_patch_p<10>(a, grid, s);
        case 11: return launch_bwd_patch_p<11>(a, grid, s);
        case 12: return launch_bwd_patch_p<12>(a, grid, s);
        case 13: return launch_bwd_patch_p<13>(a, grid, s);
        case 14: return launch_bwd_patch_p<14>(a, grid, s);
        case 15: return launch_bwd_patch_p<15>(a, grid, s);
        case 16: return launch_bwd_patch_p<16>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bwd_pyr(const GradArgs &a, cudaStream_t s) {
    k_bwd_pyr<<<ggrid(a.total), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_gather(const GradArgs &a, cudaStream_t s) {
    k_bwd_gather<<<ggrid(a.total), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_sobel(const GradArgs &a, cudaStream_t s) {
    k_bwd_sobel<<<ggrid(a.total), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bdis
