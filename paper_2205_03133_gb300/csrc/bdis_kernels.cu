// bdis_kernels.cu -- sm_103a kernels of the BDIS pipeline.
//
// Every kernel processes one pyramid level of a whole batch of pairs: work
// units are flattened over the pairs through LevelDesc::work_begin, and each
// block strides over the units (grid sized to the SM count), so the plain
// single-pair call and the batched call run the same code.
//
// Stage map (arXiv 2205.03133):
//   k_pyramid   image pyramid + Sobel-x/8 of the left image (Sec. III-A)
//   k_search    inverse-compositional GN per patch (Eq. 1), window energies
//               and rejection flags (Sec. III-B, Sec. IV technical details)
//   k_sigma_r   dynamic sigma_r^(n) (text after Eq. 6)
//   k_posterior window posterior (Eq. 5-6), coarse-to-fine rho (Eq. 10-11),
//               PDF fit (Eq. 14-16)
//   k_densify   sGMM fusion gather (Eq. 8-9, Eq. 12) and pixel variance (Eq. 17)
#include <cfloat>
#include <cmath>

#include "bdis_device.cuh"

namespace bdis {
namespace {

// ---------------------------------------------------------------- pyramid

// One thread per pixel (X, Y) of the half-resolution grid of level l:
// Sobel-x/8 of the left image at the 2x2 block (2X.., 2Y..) of level l and,
// when a coarser level is requested, the [1 4 6 4 1]/16 blur of L and R at
// (2X, 2Y), reflect-101 borders.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_pyramid(LaunchArgs a) {
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_PYR)];
        const int wq = (D.w + 1) >> 1, hq = (D.h + 1) >> 1;
        const int idx = (unit - D.work_begin[W_PYR]) * blockDim.x + threadIdx.x;
        if (idx >= wq * hq) continue;
        const int X = idx % wq, Y = idx / wq;
        const TI *L = (const TI *)D.L;
        const TI *R = (const TI *)D.R;
        const int w = D.w, h = D.h, pitch = D.pitch;
        TO *G = (TO *)D.G;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int y = 2 * Y + j;
            if (y >= h) break;
            const TI *r0 = L + (size_t)refl(y - 1, h) * pitch;
            const TI *r1 = L + (size_t)y * pitch;
            const TI *r2 = L + (size_t)refl(y + 1, h) * pitch;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int x = 2 * X + i;
                if (x >= w) break;
                const int xm = refl(x - 1, w), xp = refl(x + 1, w);
                float acc = (ldf(r0 + xp) - ldf(r0 + xm)) + 2.f * (ldf(r1 + xp) - ldf(r1 + xm)) +
                            (ldf(r2 + xp) - ldf(r2 + xm));
                stf(G + (size_t)y * D.gpitch + x, acc * 0.125f);
            }
        }
        if (D.Ln != nullptr) {
            const float k[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
            int xs[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) xs[i] = refl(2 * X + i - 2, w);
            float accL = 0.f, accR = 0.f;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const size_t ro = (size_t)refl(2 * Y + j - 2, h) * pitch;
                float sl = 0.f, sr = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    sl += k[i] * ldf(L + ro + xs[i]);
                    sr += k[i] * ldf(R + ro + xs[i]);
                }
                accL += k[j] * sl;
                accR += k[j] * sr;
            }
            stf((TO *)D.Ln + (size_t)Y * D.pitchn + X, accL * (1.f / 256.f));
            stf((TO *)D.Rn + (size_t)Y * D.pitchn + X, accR * (1.f / 256.f));
        }
    }
}

// ---------------------------------------------------------------- patch search

// A block owns one chunk of consecutive patches of one patch row.  It stages
// the P right-image rows of that patch row over the full level width (any
// estimate d samples inside them after clamping), and the left image and
// gradient over the chunk's columns, in shared memory.  A group of G lanes
// handles one patch, lane r owning patch row r; reductions are xor shuffles
// inside the group.  The iteration count is fixed, so every lane of a warp
// executes the same instruction stream.
template <int P, typename TI, typename TG>
__global__ void __launch_bounds__(256) k_search(LaunchArgs a) {
    constexpr int G = P <= 8 ? 8 : 16;
    constexpr int N = P * P;
    constexpr float invN = 1.f / (float)N;
    extern __shared__ float smem[];
    const int bp = a.band_pitch, cp = a.chunk_pitch;
    float *Rb = smem;
    float *Lb = Rb + P * bp;
    float *Gb = Lb + P * cp;
    const int tid = threadIdx.x;
    const int gl = tid & (G - 1);
    const int grp = tid / G;
    const int ngrp = blockDim.x / G;
    const bool row_on = gl < P;
    const int S = a.S;
    const float h = a.window_step;
    const float dl[4] = {-h, h, -2.f * h, 2.f * h};

    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_SEARCH)];
        const int u = unit - D.work_begin[W_SEARCH];
        const int py = u / D.nchunks, ch = u - py * D.nchunks;
        const int oy = origin(py, D.h, P, S, D.kyreg);
        const int k0 = ch * a.chunk;
        const int k1 = min(k0 + a.chunk, D.npx);
        const int cx0 = origin(k0, D.w, P, S, D.kxreg);
        const int cw = origin(k1 - 1, D.w, P, S, D.kxreg) + P - cx0;
        const int w = D.w;
        const TI *R = (const TI *)D.R;
        const TI *L = (const TI *)D.L;
        const TG *Gi = (const TG *)D.G;

        __syncthreads();  // the previous unit's readers are done with smem
        for (int i = tid; i < P * w; i += blockDim.x) {
            const int r = i / w, c = i - r * w;
            Rb[r * bp + c] = ldf(R + (size_t)(oy + r) * D.pitch + c);
        }
        for (int i = tid; i < P * cw; i += blockDim.x) {
            const int r = i / cw, c = i - r * cw;
            Lb[r * cp + c] = ldf(L + (size_t)(oy + r) * D.pitch + cx0 + c);
            Gb[r * cp + c] = ldf(Gi + (size_t)(oy + r) * D.gpitch + cx0 + c);
        }
        __syncthreads();

        for (int kk = grp; kk < a.chunk; kk += ngrp) {
            const bool active = k0 + kk < k1;
            const int kx = min(k0 + kk, k1 - 1);
            const int ox = origin(kx, w, P, S, D.kxreg);
            const int rr = row_on ? gl : 0;
            const float *Lrow = Lb + rr * cp + (ox - cx0);
            const float *Grow = Gb + rr * cp + (ox - cx0);
            const float *Rrow = Rb + rr * bp;

            // template, centred gradient, Hessian (computed once, Sec. III-A)
            float T[P], gt[P];
            float gs = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                T[j] = Lrow[j];
                gt[j] = row_on ? Grow[j] : 0.f;
                gs += gt[j];
            }
            const float gbar = group_sum<G>(gs) * invN;
            float hp = 0.f, cp_ = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                gt[j] = row_on ? gt[j] - gbar : 0.f;
                hp = fmaf(gt[j], gt[j], hp);
                cp_ = fmaf(gt[j], T[j], cp_);
            }
            const float H = group_sum<G>(hp);
            const float cT = group_sum<G>(cp_);
            const bool flat = !(H >= a.hess_eps * (float)N);

            const float cxp = (float)ox + 0.5f * (float)(P - 1);
            const float cyp = (float)oy + 0.5f * (float)(P - 1);
            const float dinit = D.Dc != nullptr ? 2.f * coarse_bilin(D.Dc, D.wc, D.hc, cxp, cyp) : 0.f;
            const float dlim = (float)w + 2.f * (float)P;

            // Gauss-Newton: d <- d + (sum gt_i s_i - cT) / H, s_i = I_r(x_i - d)
            float d = dinit, dlast = 0.f;
            for (int it = 0; it < a.iters; ++it) {
                int off;
                float t;
                split_shift(d, off, t);
                const int base = ox + off;
                float A = 0.f, B = 0.f;
                float v = Rrow[clampi(base, 0, w - 1)];
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const float vn = Rrow[clampi(base + j + 1, 0, w - 1)];
                    A = fmaf(gt[j], v, A);
                    B = fmaf(gt[j], vn, B);
                    v = vn;
                }
                const float s = group_sum<G>(fmaf(t, B - A, A));
                if (!flat) {
                    const float delta = (s - cT) / H;
                    d = fminf(fmaxf(d + delta, -dlim), dlim);
                    dlast = delta;
                }
            }

            // window energies.  E(0) in two passes; for the four offsets the
            // differences dE_k = E(delta_k) - E(0) directly from the sample
            // differences u_j = s_kj - s_0j (the template cancels):
            //   dE_k = sum u^2 - (sum u)^2 / N + 2 sum u (a_0j - mean a_0),
            // which keeps full relative precision when dE_k << E(0).
            int off0;
            float t0;
            split_shift(d, off0, t0);
            const int base0 = ox + off0;
            float s0[P];
            float sa = 0.f;
            int nout = 0;
            {
                float v = Rrow[clampi(base0, 0, w - 1)];
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const float vn = Rrow[clampi(base0 + j + 1, 0, w - 1)];
                    s0[j] = fmaf(t0, vn - v, v);
                    sa += row_on ? s0[j] - T[j] : 0.f;
                    const int xi = base0 + j;
                    nout += (row_on && (xi < 0 || xi > w - 1 || (xi == w - 1 && t0 > 0.f))) ? 1 : 0;
                    v = vn;
                }
            }
            const float mean0 = group_sum<G>(sa) * invN;
            float e0 = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const float q = row_on ? (s0[j] - T[j]) - mean0 : 0.f;
                e0 = fmaf(q, q, e0);
            }
            float su[4], suu[4], suc[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int off;
                float t;
                split_shift(d + dl[k], off, t);
                const int base = ox + off;
                float v = Rrow[clampi(base, 0, w - 1)];
                float p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const float vn = Rrow[clampi(base + j + 1, 0, w - 1)];
                    const float u = row_on ? fmaf(t, vn - v, v) - s0[j] : 0.f;
                    const float c = row_on ? (s0[j] - T[j]) - mean0 : 0.f;
                    p1 += u;
                    p2 = fmaf(u, u, p2);
                    p3 = fmaf(u, c, p3);
                    v = vn;
                }
                su[k] = p1;
                suu[k] = p2;
                suc[k] = p3;
            }
            float E[5];  // E[0] = E(0); E[k] = E(delta_k) - E(0)
            E[0] = group_sum<G>(e0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float S1 = group_sum<G>(su[k]);
                const float S2 = group_sum<G>(suu[k]);
                const float S3 = group_sum<G>(suc[k]);
                E[k + 1] = fmaxf(S2 - S1 * S1 * invN, 0.f) + 2.f * S3;
            }
            const int nout_all = (int)group_sum<G>((float)nout);

            if (active && gl == 0) {
                uint32_t f = 0;
                if (flat) f |= BDIS_F_FLAT;
                if (!isfinite(d) || !isfinite(H)) f |= BDIS_F_NONFINITE;
                if (fabsf(dlast) > a.conv_eps) f |= BDIS_F_UNCONVERGED;
                if (fabsf(d - dinit) > a.tau) f |= BDIS_F_MOVED;
                if ((float)(N - nout_all) < a.valid_gamma * (float)N) f |= BDIS_F_OUTSIDE;
                // saddle: E(0) above the smallest off-centre energy (a tie keeps)
                const float dmin = fminf(fminf(E[1], E[2]), fminf(E[3], E[4]));
                if (dmin < 0.f) f |= BDIS_F_SADDLE;
                bdis_patch_record rec;
                rec.d = d;
                rec.dinit = dinit;
                rec.dlast = dlast;
                rec.H = H;
#pragma unroll
                for (int k = 0; k < 5; ++k) rec.E[k] = E[k];
                rec.cT = cT;
                rec.flags = f;
                rec.nout = nout_all;
                rec.pi = 0.f;
                rec.rho = 0.f;
                rec.sig2 = 0.f;
                rec.pdf_flags = 0u;
                D.rec[(size_t)py * D.npx + kx] = rec;
            }
        }
    }
}

// ---------------------------------------------------------------- sigma_r

__device__ __forceinline__ float block_sum(float v, float *red) {
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
    return s;  // valid in thread 0
}

// One block per pair: sigma_r of this level from the kept patches
// (deterministic order: fixed per-thread partial sums, then a tree).
__global__ void __launch_bounds__(256) k_sigma_r(LaunchArgs a) {
    __shared__ float red[32];
    __shared__ float bc[2];
    for (int pair = blockIdx.x; pair < a.npairs; pair += gridDim.x) {
        const LevelDesc &D = a.descs[pair];
        const int n = D.npx * D.npy;
        float s = 0.f, c = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const bdis_patch_record &r = D.rec[i];
            if (r.flags == 0u) { s += r.E[0]; c += 1.f; }
        }
        const float S = block_sum(s, red);
        const float C = block_sum(c, red);
        if (threadIdx.x == 0) { bc[0] = S; bc[1] = C; }
        __syncthreads();
        float sr;
        if (a.sigma_r_mode == BDIS_SIGMA_R_FIXED) {
            sr = a.sigma_r_fixed;
        } else if (bc[1] == 0.f) {
            sr = 0.f;
        } else if (a.sigma_r_mode == BDIS_SIGMA_R_LITERAL) {
            const float mean = bc[0] / bc[1];
            float v = 0.f;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const bdis_patch_record &r = D.rec[i];
                if (r.flags == 0u) v += (r.E[0] - mean) * (r.E[0] - mean);
            }
            const float V = block_sum(v, red);
            sr = sqrtf(V / bc[1]);
        } else {
            sr = sqrtf(bc[0] / (bc[1] * (float)(a.P * a.P)));
        }
        if (a.sigma_r_mode != BDIS_SIGMA_R_FIXED) sr = fmaxf(sr, a.sigma_r_floor);
        if (threadIdx.x == 0) *D.sigma_r = sr;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- posterior + PDF

// Gauss-Newton fit of ln c - 1/2 ln(2 pi sigma^2) - delta^2/(2 sigma^2) to
// the window log-probabilities, state (sigma, c) from (sqrt(0.1), 1), steps
// halved to keep sigma, c > 0 (Sec. III-E, Eq. 16).  The 2x2 normal
// equations J^T J step = -J^T r are solved exactly, but through the centred
// abscissa q_i = delta_i^2 - mean(delta^2) instead of a Cholesky factor: with
// J_sigma = a + b delta^2 (a = -1/sigma, b = 1/sigma^3) and J_c = 1/c the
// system decouples into b dsigma = -sum q r / sum q^2 and
// (a + b mean) dsigma + dc / c = -mean r.  Same step in exact arithmetic; in
// FP32 it avoids the cancellation of the nearly collinear columns when the
// window is flat (sigma large).
__device__ float pdf_fit(const float lnp[5], const float dlt[5], int iters, float resid_max,
                         float tau, uint32_t &flags) {
    flags = 0u;
#pragma unroll
    for (int i = 1; i < 5; ++i)
        if (!(lnp[0] > lnp[i])) flags |= BDIS_PDF_NOT_PEAK;
    const float ln2pi = 1.8378770664093453f;  // ln(2 pi)
    float d2[5], mu = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        d2[i] = dlt[i] * dlt[i];
        mu += d2[i];
    }
    mu *= 0.2f;
    float qq = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) qq = fmaf(d2[i] - mu, d2[i] - mu, qq);
    float sg = sqrtf(0.1f), c = 1.f;
    for (int it = 0; it < iters; ++it) {
        const float lc = logf(c), ls = logf(sg * sg);
        const float inv2s2 = 1.f / (2.f * sg * sg);
        float rbar = 0.f, qr = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float r = (lc - 0.5f * (ln2pi + ls) - d2[i] * inv2s2) - lnp[i];
            rbar += r;
            qr = fmaf(d2[i] - mu, r, qr);
        }
        rbar *= 0.2f;
        const float a = -1.f / sg, b = 1.f / (sg * sg * sg);
        float ds = -qr / (b * qq);
        float dc = c * (-rbar - (a + b * mu) * ds);
        if (!isfinite(ds) || !isfinite(dc)) { flags |= BDIS_PDF_FAILED; break; }
        int halv = 0;
        while (!(sg + ds > 0.f && c + dc > 0.f) && halv < 60) {
            ds *= 0.5f;
            dc *= 0.5f;
            ++halv;
        }
        if (!(sg + ds > 0.f && c + dc > 0.f)) { flags |= BDIS_PDF_FAILED; break; }
        sg += ds;
        c += dc;
        if (!isfinite(sg) || !isfinite(c)) { flags |= BDIS_PDF_FAILED; break; }
    }
    float ss = 0.f;
    {
        const float lc = logf(c), ls = logf(sg * sg);
        const float inv2s2 = 1.f / (2.f * sg * sg);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float r = (lc - 0.5f * (ln2pi + ls) - d2[i] * inv2s2) - lnp[i];
            ss = fmaf(r, r, ss);
        }
    }
    const float rms = sqrtf(ss / 5.f);
    if (!isfinite(rms)) flags |= BDIS_PDF_FAILED;
    else if (rms > resid_max) flags |= BDIS_PDF_RESIDUAL;
    const float s = flags != 0u ? tau : fminf(sg, tau);
    return s * s;
}

// One thread per patch: pi_k = p_0 / sum_i p_i with p_i = exp(-E_i/(2 sigma_r^2 s^2)),
// rho_k = Gamma_n pi_k + Q^(n+1)(centre), and at the finest level with
// variance on the PDF fit.  Writes the compact fusion record.
__global__ void __launch_bounds__(256) k_posterior(LaunchArgs a) {
    const float h = a.window_step;
    const float dlt[5] = {0.f, -h, h, -2.f * h, 2.f * h};
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_POST)];
        const int idx = (unit - D.work_begin[W_POST]) * blockDim.x + threadIdx.x;
        const int n = D.npx * D.npy;
        if (idx >= n) continue;
        bdis_patch_record *rec = D.rec + idx;
        const uint32_t flags = rec->flags;
        if (flags != 0u) {
            rec->pi = rec->rho = rec->sig2 = 0.f;
            rec->pdf_flags = 0u;
            D.fuse[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float sr = __ldg(D.sigma_r);
        const float scale = 2.f * sr * sr * (float)(kWindow * kWindow);
        // ln p_i - ln p_0 = -(E_i - E_0) / (2 sigma_r^2 s^2); the record holds E_i - E_0
        float e[5], Z = 1.f;
        e[0] = 0.f;
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            e[i] = -rec->E[i] / scale;
            Z += expf(e[i]);
        }
        const float pi = 1.f / Z;
        float rho;
        if (a.use_c2f) {
            float prop = 0.f;
            if (D.Qc != nullptr) {
                const int kx = idx % D.npx, ky = idx / D.npx;
                const float cx = (float)origin(kx, D.w, a.P, a.S, D.kxreg) + 0.5f * (float)(a.P - 1);
                const float cy = (float)origin(ky, D.h, a.P, a.S, D.kyreg) + 0.5f * (float)(a.P - 1);
                prop = coarse_bilin(D.Qc, D.wc, D.hc, cx, cy);
            }
            rho = a.gamma_w * pi + prop;
        } else {
            rho = pi;
        }
        float sig2 = 0.f;
        uint32_t pf = 0u;
        if (a.level == 0 && a.variance) {
            const float lnZ = logf(Z);
            float lnp[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) lnp[i] = e[i] - lnZ;
            sig2 = pdf_fit(lnp, dlt, a.pdf_iters, a.pdf_resid, a.tau0, pf);
        }
        rec->pi = pi;
        rec->rho = rho;
        rec->sig2 = sig2;
        rec->pdf_flags = pf;
        D.fuse[idx] = make_float4(rec->d, rho, sig2, 1.f);
    }
}

// ---------------------------------------------------------------- densify

// One thread per pixel: gather the kept patches covering it (no atomics):
// omega_k = rho_k m[x - ox] m[y - oy], D = sum omega d / sum omega,
// Q = sum omega rho / sum omega, V = sum omega^2 sig2 / (sum omega)^2.
__global__ void __launch_bounds__(256) k_densify(LaunchArgs a) {
    const int P = a.P, S = a.S;
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) {
        const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_DENSE)];
        const int idx = (unit - D.work_begin[W_DENSE]) * blockDim.x + threadIdx.x;
        if (idx >= D.w * D.h) continue;
        const int x = idx % D.w, y = idx / D.w;
        // covering origins: regular k with kS <= x < kS + P, plus the ragged one
        const int kxlo = x - P + 1 > 0 ? (x - P + 1 + S - 1) / S : 0;
        const int kxhi = min(D.kxreg - 1, x / S);
        const bool kxext = D.npx > D.kxreg && x >= D.w - P;
        const int kylo = y - P + 1 > 0 ? (y - P + 1 + S - 1) / S : 0;
        const int kyhi = min(D.kyreg - 1, y / S);
        const bool kyext = D.npy > D.kyreg && y >= D.h - P;
        float sw = 0.f, swd = 0.f, swr = 0.f, sw2 = 0.f;
        int n = 0;
        const int nky = kyhi - kylo + 1 + (kyext ? 1 : 0);
        const int nkx = kxhi - kxlo + 1 + (kxext ? 1 : 0);
        for (int iy = 0; iy < nky; ++iy) {
            const int ky = (kylo + iy <= kyhi) ? kylo + iy : D.npy - 1;
            const int oy = origin(ky, D.h, P, S, D.kyreg);
            const float my = a.use_sgmm ? a.m[y - oy] : 1.f;
            for (int ix = 0; ix < nkx; ++ix) {
                const int kx = (kxlo + ix <= kxhi) ? kxlo + ix : D.npx - 1;
                const int ox = origin(kx, D.w, P, S, D.kxreg);
                const float4 f = __ldg(D.fuse + (size_t)ky * D.npx + kx);
                if (f.w == 0.f) continue;
                const float mx = a.use_sgmm ? a.m[x - ox] : 1.f;
                const float om = f.y * (my * mx);
                sw += om;
                swd = fmaf(om, f.x, swd);
                swr = fmaf(om, f.y, swr);
                sw2 = fmaf(om * om, f.z, sw2);
                ++n;
            }
        }
        float Dv, Qv, Vv;
        if (n > 0 && sw > 0.f) {
            Dv = swd / sw;
            Qv = swr / sw;
            Vv = sw2 / (sw * sw);
        } else {
            Dv = D.Dc != nullptr ? 2.f * coarse_bilin(D.Dc, D.wc, D.hc, (float)x, (float)y) : 0.f;
            Qv = 0.f;
            Vv = 0.f;
            n = 0;
        }
        if (a.level == 0) {
            const bool ok = n > 0 && Qv >= a.pix_thresh;
            D.valid[idx] = ok ? 1 : 0;
            D.disp[idx] = ok ? Dv : __int_as_float(0x7fc00000);
            if (D.var != nullptr && a.variance) D.var[idx] = ok ? Vv : __int_as_float(0x7fc00000);
        } else {
            D.D[idx] = Dv;
            D.Q[idx] = Qv;
        }
    }
}

// ---------------------------------------------------------------- dispatch

// (image type, gradient type): (u8, f32), (u8, f16), (f32, f32), (f32, f16), (f16, f16)
template <int P>
const void *search_fn(int in_type, int g_type) {
    if (in_type == E_U8)
        return g_type == E_F32 ? (const void *)k_search<P, uint8_t, float>
                               : (const void *)k_search<P, uint8_t, __half>;
    if (in_type == E_F32)
        return g_type == E_F32 ? (const void *)k_search<P, float, float>
                               : (const void *)k_search<P, float, __half>;
    if (in_type == E_F16 && g_type == E_F16) return (const void *)k_search<P, __half, __half>;
    return nullptr;
}

const void *search_kernel(int P, int in_type, int g_type) {
    switch (P) {
        case 4: return search_fn<4>(in_type, g_type);
        case 5: return search_fn<5>(in_type, g_type);
        case 6: return search_fn<6>(in_type, g_type);
        case 7: return search_fn<7>(in_type, g_type);
        case 8: return search_fn<8>(in_type, g_type);
        case 9: return search_fn<9>(in_type, g_type);
        case 10: return search_fn<10>(in_type, g_type);
        case 11: return search_fn<11>(in_type, g_type);
        case 12: return search_fn<12>(in_type, g_type);
        case 13: return search_fn<13>(in_type, g_type);
        case 14: return search_fn<14>(in_type, g_type);
        case 15: return search_fn<15>(in_type, g_type);
        case 16: return search_fn<16>(in_type, g_type);
        default: return nullptr;
    }
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int grid_for(int total, int per_sm) {
    const int cap = num_sms() * per_sm;
    return total < cap ? (total > 0 ? total : 1) : cap;
}

}  // namespace

bool search_supported(int P) { return P >= kMinPatch && P <= kMaxPatch; }
int search_group(int P) { return P <= 8 ? 8 : 16; }
int search_chunk(int P) { return 2 * (256 / search_group(P)); }

cudaError_t prepare_search(int P, size_t smem_bytes) {
    const int combos[5][2] = {{E_U8, E_F32}, {E_U8, E_F16}, {E_F32, E_F32}, {E_F32, E_F16},
                              {E_F16, E_F16}};
    for (const auto &c : combos) {
        const void *f = search_kernel(P, c[0], c[1]);
        if (f == nullptr) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int search_occupancy(int P, int in_type, int g_type, size_t smem_bytes) {
    int nb = 0;
    const void *f = search_kernel(P, in_type, g_type);
    if (f == nullptr) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem_bytes) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_pyramid(const LaunchArgs &a, int in_type, int out_type, cudaStream_t s) {
    const int grid = grid_for(a.total, 8);
    if (out_type == E_F32) {
        if (in_type == E_U8) k_pyramid<uint8_t, float><<<grid, 256, 0, s>>>(a);
        else k_pyramid<float, float><<<grid, 256, 0, s>>>(a);
    } else {
        if (in_type == E_U8) k_pyramid<uint8_t, __half><<<grid, 256, 0, s>>>(a);
        else if (in_type == E_F32) k_pyramid<float, __half><<<grid, 256, 0, s>>>(a);
        else k_pyramid<__half, __half><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_search(const LaunchArgs &a, int in_type, int g_type, size_t smem, int grid,
                          cudaStream_t s) {
    const void *f = search_kernel(a.P, in_type, g_type);
    if (f == nullptr) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3(grid), dim3(256), args, smem, s);
}

cudaError_t launch_sigma_r(const LaunchArgs &a, cudaStream_t s) {
    k_sigma_r<<<grid_for(a.npairs, 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_posterior(const LaunchArgs &a, cudaStream_t s) {
    k_posterior<<<grid_for(a.total, 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_densify(const LaunchArgs &a, cudaStream_t s) {
    k_densify<<<grid_for(a.total, 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bdis
