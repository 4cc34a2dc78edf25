/*
 * bdis_oracle.c -- plain, slow FP64 CPU restatement of BDIS
 * (Bayesian Dense Inverse Search, arXiv 2205.03133).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the CUDA
 * path and the timed CPU baseline.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Every step follows the paper's order and notation, in plain loops, FP64:
 *   pyramid + x-gradient (Sec. III, Fig. 1; Sec. III-A)
 *   fast inverse-compositional LK per patch (Sec. III-A, Eq. 1)
 *   window energies, saddle / unconverged rejection (Sec. III-B, Eq. 4-6;
 *     Sec. IV technical details)
 *   dynamic sigma_r (Sec. III-B, text after Eq. 6)
 *   patch posterior in the small window (Eq. 5, Eq. 6)
 *   coarse-to-fine propagation (Sec. III-D, Eq. 10, Eq. 11)
 *   sGMM spatial kernel (Sec. III-C, Eq. 8, Eq. 9) and fusion (Eq. 12)
 *   optional PDF fit per patch (Sec. III-E, Eq. 14-16) and pixel variance
 *     (Eq. 17, disparity part)
 * Where the paper is silent the reading used is stated beside the code.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, invariants, brute force); agreement with the authors' own C++ is
 * unpinned (no code or data of theirs is available).
 *
 * Conventions: disparity d >= 0 with I_r(x - d, y) ~= I_l(x, y), i.e. the
 * paper's u = -d.  Level 0 is full resolution; level l+1 has ceil(n/2) pixels
 * per axis.  Images are row-major, dense (row stride = width).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OB_MAX_LEVELS 8

/* storage emulation for the pyramid and gradient images; U8: pyramid images
 * stored as 8-bit integers, gradients as binary16 */
enum { OB_STORE_F64 = 0, OB_STORE_F32 = 1, OB_STORE_F16 = 2, OB_STORE_U8 = 3 };
enum { OB_SIGMA_R_POOLED = 0, OB_SIGMA_R_LITERAL = 1, OB_SIGMA_R_FIXED = 2 };
/* fusion weights: BDIS (Eq. 12, sGMM x probability) or DIS (Eq. 2, inverse
 * photometric residual) */
enum { OB_WEIGHT_BDIS = 0, OB_WEIGHT_DIS = 1 };

/* patch rejection reasons (bit flags; a patch is valid iff flags == 0) */
enum {
    OB_F_FLAT = 1u << 0,        /* Hessian below threshold: no texture        */
    OB_F_UNCONVERGED = 1u << 1, /* last GN update above conv_eps              */
    OB_F_MOVED = 1u << 2,       /* |d - d_init| above the search radius       */
    OB_F_OUTSIDE = 1u << 3,     /* too few in-image samples (gamma)           */
    OB_F_SADDLE = 1u << 4,      /* centre not the window minimum              */
    OB_F_NONFINITE = 1u << 5
};
/* PDF-fit exceptions (Sec. III-E) */
enum {
    OB_PDF_NOT_PEAK = 1u << 0,  /* probability at u_k not the strict maximum */
    OB_PDF_FAILED = 1u << 1,    /* GN left the domain or produced non-finite  */
    OB_PDF_RESIDUAL = 1u << 2   /* RMS log residual above pdf_resid           */
};

typedef struct {
    int patch, stride, levels, iters;
    double sigma_s;        /* sGMM spatial sigma (px), paper: 4              */
    double window_step;    /* window offsets {0, +-h, +-2h}, paper: h = 0.5  */
    double conv_eps;       /* convergence threshold on |last update|, 0.05   */
    double valid_gamma;    /* minimum in-image sample ratio, 0.75            */
    double pix_thresh;     /* pixel threshold on the fused probability, 0.15 */
    double search_radius;  /* tau (px at each level); <= 0 means = patch     */
    int sigma_r_mode;
    double sigma_r_floor;
    double sigma_r_fixed;
    int variance, pdf_iters;
    double pdf_resid;
    int storage;
    double hess_eps;       /* per-pixel Hessian threshold: H < hess_eps*P^2  */
    int use_sgmm, use_c2f; /* ablation switches (Table VII)                  */
    int weight_mode;       /* OB_WEIGHT_BDIS | OB_WEIGHT_DIS                  */
    int finest_level;      /* finest processed level f; f > 0 upsamples       */
    int fast_exp;          /* 1: Schraudolph's exponential in the posterior   */
} ob_params;

typedef struct {
    double d, dinit, E[5], H, cT, dlast;
    int nout;
    uint32_t flags;
    double pi, rho, sig2;
    double prop;           /* coarse probability inherited at the centre (Eq. 10) */
    uint32_t pdf_flags;
    double mu;             /* patch mean of I_r(x - d) - T at the estimate    */
} ob_patch;

/* Per-level buffers the caller may ask for (any pointer may be NULL). */
typedef struct {
    double *L[OB_MAX_LEVELS], *R[OB_MAX_LEVELS], *G[OB_MAX_LEVELS];
    double *D[OB_MAX_LEVELS], *Q[OB_MAX_LEVELS];
    ob_patch *patches[OB_MAX_LEVELS];
    double sigma_r[OB_MAX_LEVELS];
} ob_trace;

/* ------------------------------------------------------------------ */
/* storage emulation                                                    */
/* ------------------------------------------------------------------ */

/* Round to the nearest IEEE-754 binary16 value, ties to even.  Written from
 * the format's definition: 10 fraction bits, normal exponents -14..15,
 * subnormal spacing 2^-24, overflow to infinity at >= 65520. */
double ob_round_f16(double v)
{
    if (isnan(v)) return v;
    double a = fabs(v);
    if (a >= 65520.0) return copysign(INFINITY, v);
    if (a == 0.0) return v;
    int e;
    frexp(a, &e);          /* a = m * 2^e, m in [0.5, 1): a in [2^(e-1), 2^e) */
    int E = e - 1;
    if (E < -14) E = -14;  /* subnormal range keeps the spacing of 2^-14 binade */
    double ulp = ldexp(1.0, E - 10);
    double q = nearbyint(a / ulp); /* default rounding mode: nearest, ties even */
    return copysign(q * ulp, v);
}

/* An 8-bit image value: the nearest integer, ties to even, clamped to
 * [0, 255]. */
double ob_round_u8(double v)
{
    double q = nearbyint(v); /* default rounding mode: nearest, ties even */
    return q < 0.0 ? 0.0 : (q > 255.0 ? 255.0 : q);
}

/* Rounding of a stored pyramid image value. */
double ob_round_storage(double v, int storage)
{
    if (storage == OB_STORE_F32) return (double)(float)v;
    if (storage == OB_STORE_F16) return ob_round_f16(v);
    if (storage == OB_STORE_U8) return ob_round_u8(v);
    return v;
}

/* Rounding of a stored gradient value (binary16 with 8-bit images). */
static double round_grad_storage(double v, int storage)
{
    return ob_round_storage(v, storage == OB_STORE_U8 ? OB_STORE_F16 : storage);
}

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

int ob_level_dim(int n, int l)
{
    for (int i = 0; i < l; ++i) n = (n + 1) / 2;
    return n;
}

static int reflect101(int i, int n)
{
    /* reflect about the edge pixel without repeating it: -1 -> 1, n -> n-2 */
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

/* Patch origins along one axis of length n: 0, S, 2S, ... <= n-P, plus one
 * extra origin at n-P when (n-P) is not a multiple of S, so every pixel is
 * covered (patch grid of Sec. III-A with overlap 1 - S/P). */
int ob_origins(int n, int P, int S, int *out)
{
    if (n < P) return 0;
    int k = 0;
    for (int o = 0; o <= n - P; o += S) {
        if (out) out[k] = o;
        ++k;
    }
    if ((n - P) % S != 0) {
        if (out) out[k] = n - P;
        ++k;
    }
    return k;
}

/* Gamma weight of level n (the formula following Eq. 11):
 * 2^n / sum_{m in N} 2^m, N the processed levels finest .. levels-1. */
double ob_gamma_weight_f(int n, int finest, int levels)
{
    double s = 0.0;
    for (int m = finest; m < levels; ++m) s += ldexp(1.0, m);
    return ldexp(1.0, n) / s;
}

double ob_gamma_weight(int n, int levels) { return ob_gamma_weight_f(n, 0, levels); }

/* Schraudolph's exponential (N. Schraudolph, "A fast, compact approximation
 * of the exponential function", Neural Computation 11(4), 1999), in the
 * single-precision form: the integer i = A y + (B - C), A = 2^23 / ln 2,
 * B = 127 * 2^23 (the exponent bias in place), C = 8 * 60801 (the published
 * RMS-optimal correction of the double-precision form, moved to the 23-bit
 * fraction), truncated, read as the bits of an IEEE-754 binary32 number.
 * Relative error within about 4 %.  Arguments below -87 (where i would leave
 * the normal range) give 0. */
double ob_exp_schraudolph(double y)
{
    if (y < -87.0) return 0.0;
    if (y > 88.0) y = 88.0;
    const double A = 8388608.0 / log(2.0);
    const double BC = 127.0 * 8388608.0 - 8.0 * 60801.0;
    int32_t i = (int32_t)floor(A * y + BC);
    float f;
    memcpy(&f, &i, sizeof f);
    return (double)f;
}

/* ------------------------------------------------------------------ */
/* pyramid and x-gradient                                               */
/* ------------------------------------------------------------------ */

/* One pyramid step: 5-tap binomial blur [1 4 6 4 1]/16 in both axes,
 * reflect-101 border, keep the even samples.  The paper does not state the
 * filter (it only says level n pixels stand for 2^n x 2^n patches, Sec. III-B);
 * this is the reading used. */
void ob_pyr_down(const double *src, int w, int h, double *dst, int storage)
{
    static const double k[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
    for (int Y = 0; Y < h2; ++Y)
        for (int X = 0; X < w2; ++X) {
            double acc = 0.0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i) {
                    int yy = reflect101(2 * Y + j, h), xx = reflect101(2 * X + i, w);
                    acc += k[j + 2] * k[i + 2] * src[(size_t)yy * w + xx];
                }
            dst[(size_t)Y * w2 + X] = ob_round_storage(acc, storage);
        }
}

/* x-gradient of the left image used as the fixed inverse-compositional
 * Jacobian (Sec. III-A): Sobel-x divided by 8 (columns [-1 0 1], rows
 * [1 2 1]), reflect-101 border. */
void ob_sobel_x(const double *src, int w, int h, double *g, int storage)
{
    static const double wr[3] = {1.0, 2.0, 1.0};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double acc = 0.0;
            for (int j = -1; j <= 1; ++j) {
                int yy = reflect101(y + j, h);
                acc += wr[j + 1] * (src[(size_t)yy * w + reflect101(x + 1, w)] -
                                    src[(size_t)yy * w + reflect101(x - 1, w)]);
            }
            g[(size_t)y * w + x] = round_grad_storage(acc / 8.0, storage);
        }
}

/* ------------------------------------------------------------------ */
/* sampling                                                             */
/* ------------------------------------------------------------------ */

/* Right image at (X, row) by linear interpolation along x; the coordinate
 * is clamped to [0, w-1] (rows are integer for rectified stereo, so the
 * bilinear lookup of Eq. 1 reduces to linear). */
static double sample_row(const double *img, int w, int row, double X)
{
    if (X < 0.0) X = 0.0;
    if (X > w - 1.0) X = w - 1.0;
    int x0 = (int)floor(X);
    double t = X - x0;
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
    const double *r = img + (size_t)row * w;
    return (1.0 - t) * r[x0] + t * r[x1];
}

/* Bilinear lookup of a coarse map at fine position (x, y) of the next finer
 * level: coarse coordinate = (x + 0.5)/2 - 0.5, clamped to the map. */
static double coarse_lookup(const double *m, int wc, int hc, double x, double y)
{
    double X = (x + 0.5) / 2.0 - 0.5, Y = (y + 0.5) / 2.0 - 0.5;
    if (X < 0.0) X = 0.0;
    if (X > wc - 1.0) X = wc - 1.0;
    if (Y < 0.0) Y = 0.0;
    if (Y > hc - 1.0) Y = hc - 1.0;
    int x0 = (int)floor(X), y0 = (int)floor(Y);
    int x1 = x0 + 1 < wc ? x0 + 1 : wc - 1, y1 = y0 + 1 < hc ? y0 + 1 : hc - 1;
    double fx = X - x0, fy = Y - y0;
    double a = (1.0 - fx) * m[(size_t)y0 * wc + x0] + fx * m[(size_t)y0 * wc + x1];
    double b = (1.0 - fx) * m[(size_t)y1 * wc + x0] + fx * m[(size_t)y1 * wc + x1];
    return (1.0 - fy) * a + fy * b;
}

static double search_radius(const ob_params *p)
{
    return p->search_radius > 0.0 ? p->search_radius : (double)p->patch;
}

/* ------------------------------------------------------------------ */
/* per-patch search (Sec. III-A, Eq. 1) and window energies (Eq. 6)     */
/* ------------------------------------------------------------------ */

/* Window offsets delta_i of the small window P' (Sec. III-B and the
 * parameter list of Sec. IV-A: 5 samples, disturbances 0.5 and 1 px):
 * index 0 is the converged estimate itself. */
void ob_window_offsets(double h, double *delta)
{
    delta[0] = 0.0;
    delta[1] = -h;
    delta[2] = h;
    delta[3] = -2.0 * h;
    delta[4] = 2.0 * h;
}

/* Search one patch with origin (ox, oy) at a level of size w x h.
 * L, R, G: left, right, left x-gradient of the level.
 * dinit: initial disparity (from the coarser level, 0 at the coarsest).
 *
 * Inverse compositional Gauss-Newton on the mean-normalised residual
 * r_i = (s_i - mean s) - (T_i - mean T), s_i = I_r(x_i - d): the template
 * warp is linearised once, with Jacobian the centred gradient
 * gt_i = g_i - mean g and scalar Hessian H = sum gt_i^2.  Because
 * sum gt_i = 0 the step is  delta = (sum gt_i s_i - sum gt_i T_i) / H  and the
 * warp update composes to d <- d + delta.  The iteration count is fixed. */
void ob_search_patch(const ob_params *p, const double *L, const double *R,
                     const double *G, int w, int h, int ox, int oy, double dinit,
                     ob_patch *out)
{
    const int P = p->patch;
    const int N = P * P;
    double *T = (double *)malloc(sizeof(double) * N);
    double *gt = (double *)malloc(sizeof(double) * N);
    double gbar = 0.0;
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            T[r * P + c] = L[(size_t)(oy + r) * w + ox + c];
            gt[r * P + c] = G[(size_t)(oy + r) * w + ox + c];
            gbar += gt[r * P + c];
        }
    gbar /= N;
    double H = 0.0, cT = 0.0;
    for (int i = 0; i < N; ++i) {
        gt[i] -= gbar;
        H += gt[i] * gt[i];
        cT += gt[i] * T[i];
    }
    memset(out, 0, sizeof(*out));
    out->H = H;
    out->cT = cT;
    out->dinit = dinit;
    double d = dinit, dlast = 0.0;
    const double dlim = (double)w + 2.0 * P; /* beyond this every sample is clamped */
    int flat = !(H >= p->hess_eps * N);
    if (!flat) {
        for (int it = 0; it < p->iters; ++it) {
            double acc = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c)
                    acc += gt[r * P + c] * sample_row(R, w, oy + r, (double)(ox + c) - d);
            double delta = (acc - cT) / H;
            d += delta;
            if (d > dlim) d = dlim;
            if (d < -dlim) d = -dlim;
            dlast = delta;
        }
    }
    out->d = d;
    out->dlast = dlast;

    /* window energies E(delta_i) = sum_j (a_j - mean a)^2 with
     * a_j = I_r(x_j - d - delta_i) - T_j (mean-normalised SSD, Eq. 6 numerator) */
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    double *a = (double *)malloc(sizeof(double) * N);
    for (int k = 0; k < 5; ++k) {
        double mean = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                a[r * P + c] = sample_row(R, w, oy + r, (double)(ox + c) - d - delta[k]) - T[r * P + c];
                mean += a[r * P + c];
            }
        mean /= N;
        double E = 0.0;
        for (int i = 0; i < N; ++i) E += (a[i] - mean) * (a[i] - mean);
        out->E[k] = E;
        if (k == 0) out->mu = mean;
    }
    int nout = 0;
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            double X = (double)(ox + c) - d;
            if (X < 0.0 || X > w - 1.0) ++nout;
        }
    out->nout = nout;

    uint32_t f = 0;
    if (flat) f |= OB_F_FLAT;
    if (!isfinite(d) || !isfinite(H)) f |= OB_F_NONFINITE;
    if (fabs(dlast) > p->conv_eps) f |= OB_F_UNCONVERGED;
    if (fabs(d - dinit) > search_radius(p)) f |= OB_F_MOVED;
    if ((double)(N - nout) < p->valid_gamma * N) f |= OB_F_OUTSIDE;
    double emin = out->E[1];
    for (int k = 2; k < 5; ++k) emin = out->E[k] < emin ? out->E[k] : emin;
    if (out->E[0] > emin) f |= OB_F_SADDLE; /* a tie keeps the patch */
    out->flags = f;
    free(a);
    free(T);
    free(gt);
}

/* ------------------------------------------------------------------ */
/* dynamic sigma_r (text after Eq. 6)                                   */
/* ------------------------------------------------------------------ */

/* The paper sets sigma_r^(n) to "the standard deviation" of the converged
 * patch residual.  Default reading (pooled): the standard deviation of the
 * per-pixel normalised residual pooled over the valid patches of the level,
 * sqrt(sum_k E_k(0) / (N_valid P^2)), floored.  LITERAL: population std of
 * E_k(0) over valid patches.  FIXED: the constant of the ablation (8). */
double ob_sigma_r(const ob_params *p, const ob_patch *pt, int n)
{
    if (p->sigma_r_mode == OB_SIGMA_R_FIXED) return p->sigma_r_fixed;
    double s = 0.0;
    long cnt = 0;
    for (int k = 0; k < n; ++k)
        if (pt[k].flags == 0) {
            s += pt[k].E[0];
            ++cnt;
        }
    double sr;
    if (cnt == 0) {
        sr = 0.0;
    } else if (p->sigma_r_mode == OB_SIGMA_R_LITERAL) {
        double mean = s / cnt, v = 0.0;
        for (int k = 0; k < n; ++k)
            if (pt[k].flags == 0) v += (pt[k].E[0] - mean) * (pt[k].E[0] - mean);
        sr = sqrt(v / cnt);
    } else {
        sr = sqrt(s / ((double)cnt * p->patch * p->patch));
    }
    return sr > p->sigma_r_floor ? sr : p->sigma_r_floor;
}

/* ------------------------------------------------------------------ */
/* PDF fit (Sec. III-E, Eq. 14-16)                                      */
/* ------------------------------------------------------------------ */

/* Fit  ln c - 1/2 ln(2 pi sigma^2) - delta_i^2 / (2 sigma^2)  to the window
 * log-probabilities lnp[i] by Gauss-Newton on (sigma, c), the 2x2 normal
 * equations solved by Cholesky, from (sqrt(0.1), 1), a fixed number of
 * iterations.  Reading: a step that would leave sigma > 0, c > 0 is halved
 * until it stays inside (the paper does not say how the state is kept in its
 * domain).  Exceptions (Sec. III-E): probability at the estimate not the
 * strict maximum, GN failure, RMS residual above pdf_resid -> sigma = tau.
 * A fitted sigma above tau is capped at tau.  Returns sigma_k^2. */
double ob_pdf_fit(const double *lnp, const double *delta, int iters, double resid_max,
                  double tau, uint32_t *flags_out, double *sigma_out, double *c_out,
                  double *rms_out)
{
    uint32_t flags = 0;
    for (int i = 1; i < 5; ++i)
        if (!(lnp[0] > lnp[i])) flags |= OB_PDF_NOT_PEAK;
    double sg = sqrt(0.1), c = 1.0;
    const double ln2pi = log(2.0 * M_PI);
    for (int it = 0; it < iters && !(flags & OB_PDF_FAILED); ++it) {
        double A11 = 0, A12 = 0, A22 = 0, b1 = 0, b2 = 0;
        for (int i = 0; i < 5; ++i) {
            double d2 = delta[i] * delta[i];
            double m = log(c) - 0.5 * (ln2pi + log(sg * sg)) - d2 / (2.0 * sg * sg);
            double r = m - lnp[i];
            double js = -1.0 / sg + d2 / (sg * sg * sg);
            double jc = 1.0 / c;
            A11 += js * js;
            A12 += js * jc;
            A22 += jc * jc;
            b1 -= js * r;
            b2 -= jc * r;
        }
        /* Cholesky A = L L^T */
        if (!(A11 > 0.0)) { flags |= OB_PDF_FAILED; break; }
        double l11 = sqrt(A11), l21 = A12 / l11, s22 = A22 - l21 * l21;
        if (!(s22 > 0.0)) { flags |= OB_PDF_FAILED; break; }
        double l22 = sqrt(s22);
        double y1 = b1 / l11, y2 = (b2 - l21 * y1) / l22;
        double dc = y2 / l22, ds = (y1 - l21 * dc) / l11;
        int halvings = 0;
        while (!(sg + ds > 0.0 && c + dc > 0.0) && halvings < 60) {
            ds *= 0.5;
            dc *= 0.5;
            ++halvings;
        }
        if (!(sg + ds > 0.0 && c + dc > 0.0)) { flags |= OB_PDF_FAILED; break; }
        sg += ds;
        c += dc;
        if (!isfinite(sg) || !isfinite(c)) { flags |= OB_PDF_FAILED; break; }
    }
    double ss = 0.0;
    for (int i = 0; i < 5; ++i) {
        double d2 = delta[i] * delta[i];
        double m = log(c) - 0.5 * (ln2pi + log(sg * sg)) - d2 / (2.0 * sg * sg);
        ss += (m - lnp[i]) * (m - lnp[i]);
    }
    double rms = sqrt(ss / 5.0);
    if (!isfinite(rms)) flags |= OB_PDF_FAILED;
    else if (rms > resid_max) flags |= OB_PDF_RESIDUAL;
    if (sigma_out) *sigma_out = sg;
    if (c_out) *c_out = c;
    if (rms_out) *rms_out = rms;
    if (flags_out) *flags_out = flags;
    double s = (flags != 0) ? tau : (sg < tau ? sg : tau);
    return s * s;
}

/* ------------------------------------------------------------------ */
/* posterior (Eq. 5, 6) and coarse-to-fine propagation (Eq. 10, 11)     */
/* ------------------------------------------------------------------ */

/* Window posterior of the converged estimate: with the Boltzmann prior of
 * Eq. 6, p_i = exp(-E_i / (2 sigma_r^2 s^2)) for the s = 5 window samples,
 * and Eq. 5 with r = 1:  pi_k = p_0 / sum_i p_i. */
void ob_posterior(const ob_params *p, int level, ob_patch *pt, int n, double sigma_r,
                  const double *Qc, int wc, int hc, const int *ox, const int *oy,
                  int npx)
{
    const double s = 5.0;
    const double scale = 2.0 * sigma_r * sigma_r * s * s;
    const double wl = ob_gamma_weight_f(level, p->finest_level, p->levels);
    const double tau0 = search_radius(p);
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    for (int k = 0; k < n; ++k) {
        ob_patch *q = &pt[k];
        q->pi = q->rho = q->sig2 = q->prop = 0.0;
        q->pdf_flags = 0;
        if (q->flags != 0) continue;
        double e[5], Z = 0.0, Zf = 0.0;
        for (int i = 0; i < 5; ++i) {
            e[i] = -(q->E[i] - q->E[0]) / scale; /* ln p_i - ln p_0 */
            Z += exp(e[i]);
            Zf += ob_exp_schraudolph(e[i]);
        }
        /* pi = p_0 / sum_i p_i; with fast_exp every p_i (p_0 included) is
         * Schraudolph's approximation.  The PDF fit below keeps the exact
         * log-probabilities. */
        q->pi = p->fast_exp ? ob_exp_schraudolph(0.0) / Zf : 1.0 / Z;
        if (p->use_c2f) {
            /* rho = Gamma_n pi + propagated probability of the coarser levels,
             * read from the fused coarse probability map at the patch centre
             * (reading of Eq. 10: a superposition over levels) */
            double prop = 0.0;
            if (Qc) {
                double cx = ox[k % npx] + (p->patch - 1) / 2.0;
                double cy = oy[k / npx] + (p->patch - 1) / 2.0;
                prop = coarse_lookup(Qc, wc, hc, cx, cy);
            }
            q->rho = wl * q->pi + prop;
            q->prop = prop;
        } else {
            q->rho = q->pi;
        }
        if (level == p->finest_level && p->variance) {
            double lnp[5], lnZ = log(Z);
            for (int i = 0; i < 5; ++i) lnp[i] = e[i] - lnZ;
            q->sig2 = ob_pdf_fit(lnp, delta, p->pdf_iters, p->pdf_resid, tau0,
                                 &q->pdf_flags, NULL, NULL, NULL);
        }
    }
}

/* ------------------------------------------------------------------ */
/* sGMM kernel (Eq. 8) and fusion (Eq. 12, Eq. 17)                      */
/* ------------------------------------------------------------------ */

/* M[b][a] = sum over the patch pixels x_i of exp(-|x - x_i|^2 / (2 sigma_s^2))
 * for x at offset (a, b) inside the patch: Eq. 8 written out literally. */
void ob_sgmm_table(int P, double sigma_s, double *M)
{
    for (int b = 0; b < P; ++b)
        for (int a = 0; a < P; ++a) {
            double s = 0.0;
            for (int j = 0; j < P; ++j)
                for (int i = 0; i < P; ++i) {
                    double dx = a - i, dy = b - j;
                    s += exp(-(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s));
                }
            M[b * P + a] = s;
        }
}

/* Fuse the valid patches of one level into dense maps.  For pixel x with
 * covering valid patches Omega(x): omega_k = rho_k M[x - o_k] (Eq. 12), or
 * with weight_mode DIS the inverse photometric residual of Eq. 2,
 * omega_k = 1 / max(1, r_k(x)^2) with r_k(x) = I_r(x - d_k) - I_l(x) - mu_k
 * (mean-normalised like the search; the floor of 1 DN^2 avoids a division
 * by zero at an exact match).  Then
 * D = sum omega_k d_k / sum omega_k, Q = sum omega_k rho_k / sum omega_k,
 * V = sum omega_k^2 sigma_k^2 / (sum omega_k)^2.  Pixels with no valid
 * covering patch take the upsampled coarser disparity (0 at the coarsest
 * level) and Q = 0, V = 0, and are marked invalid (cnt = 0).  L, R: the
 * level's images (read only in DIS mode; may be NULL otherwise). */
void ob_densify(const ob_params *p, const ob_patch *pt, const int *ox, int npx,
                const int *oy, int npy, int w, int h, const double *L, const double *R,
                const double *Dc, int wc, int hc, double *D, double *Q, double *V, int *cnt)
{
    const int P = p->patch;
    double *M = (double *)malloc(sizeof(double) * P * P);
    if (p->use_sgmm) {
        ob_sgmm_table(P, p->sigma_s, M);
    } else {
        for (int i = 0; i < P * P; ++i) M[i] = 1.0; /* equal pixel weights */
    }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double sw = 0.0, swd = 0.0, swr = 0.0, sw2s = 0.0;
            int n = 0;
            for (int ky = 0; ky < npy; ++ky) {
                if (!(oy[ky] <= y && y < oy[ky] + P)) continue;
                for (int kx = 0; kx < npx; ++kx) {
                    if (!(ox[kx] <= x && x < ox[kx] + P)) continue;
                    const ob_patch *q = &pt[ky * npx + kx];
                    if (q->flags != 0) continue;
                    double om;
                    if (p->weight_mode == OB_WEIGHT_DIS) {
                        double r = sample_row(R, w, y, (double)x - q->d) - L[(size_t)y * w + x] -
                                   q->mu;
                        om = 1.0 / (r * r > 1.0 ? r * r : 1.0);
                    } else {
                        om = q->rho * M[(y - oy[ky]) * P + (x - ox[kx])];
                    }
                    sw += om;
                    swd += om * q->d;
                    swr += om * q->rho;
                    sw2s += om * om * q->sig2;
                    ++n;
                }
            }
            size_t i = (size_t)y * w + x;
            if (n > 0 && sw > 0.0) {
                D[i] = swd / sw;
                Q[i] = swr / sw;
                if (V) V[i] = sw2s / (sw * sw);
            } else {
                D[i] = Dc ? 2.0 * coarse_lookup(Dc, wc, hc, x, y) : 0.0;
                Q[i] = 0.0;
                if (V) V[i] = 0.0;
                n = 0;
            }
            if (cnt) cnt[i] = n;
        }
    free(M);
}

/* ------------------------------------------------------------------ */
/* one level and the whole coarse-to-fine pipeline (Fig. 1)             */
/* ------------------------------------------------------------------ */

int ob_num_patches(const ob_params *p, int w, int h, int level, int *npx, int *npy)
{
    int wl = ob_level_dim(w, level), hl = ob_level_dim(h, level);
    int a = ob_origins(wl, p->patch, p->stride, NULL);
    int b = ob_origins(hl, p->patch, p->stride, NULL);
    if (npx) *npx = a;
    if (npy) *npy = b;
    return a * b;
}

int ob_check(const ob_params *p, int w, int h)
{
    if (p->patch < 2 || p->stride < 1 || p->levels < 1 || p->levels > OB_MAX_LEVELS ||
        p->iters < 0 || p->finest_level < 0 || p->finest_level >= p->levels)
        return 1;
    int wl = ob_level_dim(w, p->levels - 1), hl = ob_level_dim(h, p->levels - 1);
    if (wl < p->patch || hl < p->patch || wl < 3 || hl < 3) return 1;
    return 0;
}

/* Search all patches of one level given its images and the coarser fused
 * disparity Dc (NULL at the coarsest level). */
void ob_search_level(const ob_params *p, const double *L, const double *R, const double *G,
                     int w, int h, const double *Dc, int wc, int hc, ob_patch *out)
{
    int npx, npy;
    int *ox = (int *)malloc(sizeof(int) * (w + 2));
    int *oy = (int *)malloc(sizeof(int) * (h + 2));
    npx = ob_origins(w, p->patch, p->stride, ox);
    npy = ob_origins(h, p->patch, p->stride, oy);
    for (int ky = 0; ky < npy; ++ky)
        for (int kx = 0; kx < npx; ++kx) {
            double cx = ox[kx] + (p->patch - 1) / 2.0, cy = oy[ky] + (p->patch - 1) / 2.0;
            double dinit = Dc ? 2.0 * coarse_lookup(Dc, wc, hc, cx, cy) : 0.0;
            ob_search_patch(p, L, R, G, w, h, ox[kx], oy[ky], dinit, &out[ky * npx + kx]);
        }
    free(ox);
    free(oy);
}

/* Full-resolution output from the finest processed level f > 0 (the paper
 * stops at scale 2^1 and upsamples, Sec. IV-A).  For pixel x the level-f
 * coordinate is X = (x + 0.5) / 2^f - 0.5, clamped to the map; disp =
 * 2^f * bilinear(D_f), var = 4^f * bilinear(V_f) (a disparity scaled by s
 * has s^2 times the variance).  The pixel is valid iff every level-f pixel
 * with a non-zero bilinear weight is valid. */
void ob_upsample_output(const double *Df, const double *Vf, const uint8_t *okf, int wf, int hf,
                        int f, int w, int h, double *disp, double *var, uint8_t *valid)
{
    const double s = ldexp(1.0, f);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double X = (x + 0.5) / s - 0.5, Y = (y + 0.5) / s - 0.5;
            if (X < 0.0) X = 0.0;
            if (X > wf - 1.0) X = wf - 1.0;
            if (Y < 0.0) Y = 0.0;
            if (Y > hf - 1.0) Y = hf - 1.0;
            int x0 = (int)floor(X), y0 = (int)floor(Y);
            int x1 = x0 + 1 < wf ? x0 + 1 : wf - 1, y1 = y0 + 1 < hf ? y0 + 1 : hf - 1;
            double fx = X - x0, fy = Y - y0;
            int xs[4] = {x0, x1, x0, x1}, ys[4] = {y0, y0, y1, y1};
            double wt[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
            int ok = 1;
            double dv = 0.0, vv = 0.0;
            for (int i = 0; i < 4; ++i) {
                if (wt[i] == 0.0) continue;
                size_t j = (size_t)ys[i] * wf + xs[i];
                ok &= okf[j] != 0;
                dv += wt[i] * Df[j];
                if (Vf) vv += wt[i] * Vf[j];
            }
            size_t i = (size_t)y * w + x;
            valid[i] = (uint8_t)ok;
            disp[i] = ok ? s * dv : NAN;
            if (var) var[i] = (ok && Vf) ? s * s * vv : NAN;
        }
}

/* Full BDIS on one pair of level-0 images (values already in the storage
 * type; 8-bit inputs are exact in every storage type).
 * Outputs (w*h each): disp (NaN where invalid), var (NaN where invalid or
 * variance off; may be NULL), valid (0/1). */
int ob_match(const ob_params *p, const double *L0, const double *R0, int w, int h,
             double *disp, double *var, uint8_t *valid, ob_trace *tr)
{
    if (ob_check(p, w, h)) return 1;
    const int NL = p->levels;
    double *Lv[OB_MAX_LEVELS], *Rv[OB_MAX_LEVELS], *Gv[OB_MAX_LEVELS];
    int W[OB_MAX_LEVELS], Hh[OB_MAX_LEVELS];
    for (int l = 0; l < NL; ++l) {
        W[l] = ob_level_dim(w, l);
        Hh[l] = ob_level_dim(h, l);
        size_t n = (size_t)W[l] * Hh[l];
        Lv[l] = (double *)malloc(sizeof(double) * n);
        Rv[l] = (double *)malloc(sizeof(double) * n);
        Gv[l] = (double *)malloc(sizeof(double) * n);
    }
    memcpy(Lv[0], L0, sizeof(double) * w * h);
    memcpy(Rv[0], R0, sizeof(double) * w * h);
    for (int l = 0; l + 1 < NL; ++l) {
        ob_pyr_down(Lv[l], W[l], Hh[l], Lv[l + 1], p->storage);
        ob_pyr_down(Rv[l], W[l], Hh[l], Rv[l + 1], p->storage);
    }
    for (int l = 0; l < NL; ++l) ob_sobel_x(Lv[l], W[l], Hh[l], Gv[l], p->storage);

    double *Dprev = NULL, *Qprev = NULL;
    int wprev = 0, hprev = 0;
    const int F = p->finest_level;
    for (int l = NL - 1; l >= F; --l) {
        const int wl = W[l], hl = Hh[l];
        int *ox = (int *)malloc(sizeof(int) * (wl + 2));
        int *oy = (int *)malloc(sizeof(int) * (hl + 2));
        int npx = ob_origins(wl, p->patch, p->stride, ox);
        int npy = ob_origins(hl, p->patch, p->stride, oy);
        int np = npx * npy;
        ob_patch *pt = (ob_patch *)calloc((size_t)np, sizeof(ob_patch));
        ob_search_level(p, Lv[l], Rv[l], Gv[l], wl, hl, Dprev, wprev, hprev, pt);
        double sr = ob_sigma_r(p, pt, np);
        ob_posterior(p, l, pt, np, sr, Qprev, wprev, hprev, ox, oy, npx);
        size_t n = (size_t)wl * hl;
        double *D = (double *)malloc(sizeof(double) * n);
        double *Q = (double *)malloc(sizeof(double) * n);
        double *V = (l == F) ? (double *)malloc(sizeof(double) * n) : NULL;
        int *cnt = (int *)malloc(sizeof(int) * n);
        ob_densify(p, pt, ox, npx, oy, npy, wl, hl, Lv[l], Rv[l], Dprev, wprev, hprev, D, Q, V,
                   cnt);
        if (tr) {
            tr->sigma_r[l] = sr;
            if (tr->patches[l]) memcpy(tr->patches[l], pt, sizeof(ob_patch) * np);
            if (tr->D[l]) memcpy(tr->D[l], D, sizeof(double) * n);
            if (tr->Q[l]) memcpy(tr->Q[l], Q, sizeof(double) * n);
            if (tr->L[l]) memcpy(tr->L[l], Lv[l], sizeof(double) * n);
            if (tr->R[l]) memcpy(tr->R[l], Rv[l], sizeof(double) * n);
            if (tr->G[l]) memcpy(tr->G[l], Gv[l], sizeof(double) * n);
        }
        if (l == 0) {
            /* finest level: a pixel is valid iff it has a valid covering
             * patch and its fused probability reaches the pixel threshold */
            for (size_t i = 0; i < n; ++i) {
                int ok = cnt[i] > 0 && Q[i] >= p->pix_thresh;
                valid[i] = (uint8_t)ok;
                disp[i] = ok ? D[i] : NAN;
                if (var) var[i] = (ok && p->variance) ? V[i] : NAN;
            }
        } else if (l == F) {
            uint8_t *okf = (uint8_t *)malloc(n);
            for (size_t i = 0; i < n; ++i) okf[i] = (uint8_t)(cnt[i] > 0 && Q[i] >= p->pix_thresh);
            ob_upsample_output(D, p->variance ? V : NULL, okf, wl, hl, F, w, h, disp, var,
                               valid);
            free(okf);
        }
        free(Dprev);
        free(Qprev);
        free(V);
        free(cnt);
        free(pt);
        free(ox);
        free(oy);
        Dprev = D;
        Qprev = Q;
        wprev = wl;
        hprev = hl;
    }
    free(Dprev);
    free(Qprev);
    for (int l = 0; l < NL; ++l) {
        free(Lv[l]);
        free(Rv[l]);
        free(Gv[l]);
    }
    return 0;
}

/* 8-bit entry point: converts to double and runs ob_match. */
int ob_match_u8(const ob_params *p, const uint8_t *L, const uint8_t *R, int w, int h,
                double *disp, double *var, uint8_t *valid, ob_trace *tr)
{
    size_t n = (size_t)w * h;
    double *a = (double *)malloc(sizeof(double) * n), *b = (double *)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) {
        a[i] = L[i];
        b[i] = R[i];
    }
    int rc = ob_match(p, a, b, w, h, disp, var, valid, tr);
    free(a);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------ */
/* depth (Eq. 13) and depth variance (Eq. 17)                           */
/* ------------------------------------------------------------------ */

/* Depth of a rectified pair from the fused finest-level disparity, Eq. 13:
 * z = f b / d, with f the focal length (px) and b the baseline.  Its
 * variance, Eq. 17: the fused disparity variance sum_k omega_k^2 sigma_k^2
 * (the output var of ob_match) times (f b)^2 / d^4, the square of the slope
 * of z(d).  A pixel whose disparity is not a positive finite number (NaN
 * where the match is invalid) gets NaN in both.  var / depth_var may be
 * NULL. */
void ob_depth(const double *disp, const double *var, long n, double fb, double *depth,
              double *depth_var)
{
    for (long i = 0; i < n; ++i) {
        double d = disp[i];
        int ok = isfinite(d) && d > 0.0;
        depth[i] = ok ? fb / d : NAN;
        if (depth_var) depth_var[i] = ok ? (fb * fb) / (d * d * d * d) * var[i] : NAN;
    }
}

int ob_sizeof_patch(void) { return (int)sizeof(ob_patch); }
int ob_sizeof_params(void) { return (int)sizeof(ob_params); }

/* ================================================================== */
/* Differentiable form (finest level, discrete state frozen)           */
/* ================================================================== */
/*
 * The function differentiated, given float images I_l, I_r of level 0 and
 * the discrete state of a forward pass (which level-0 patches were kept,
 * each patch's initial disparity d_init and inherited coarse probability
 * prop, the valid pixels, and whether sigma_r sat at its floor):
 *   g     = Sobel-x/8 of I_l
 *   d_k   = `iters` Gauss-Newton steps from d_init (Eq. 1), kept patches
 *   E_k   = window energies at d_k + delta_i
 *   sigma_r (pooled, or the floor / fixed value as a constant)
 *   pi_k  = window posterior (Eq. 5-6), rho_k = Gamma_0 pi_k + prop_k
 *   D(x)  = sum_k omega_k d_k / sum_k omega_k over kept covering patches (Eq. 12)
 *   loss  = ( sum_{x valid} |I_r(x - D(x)) - I_l(x)|
 *           + lambda sum_{valid 4-neighbour pairs (p, q)} |D(p) - D(q)| ) / (w h)
 * The analytic gradient treats each d_k as the root of
 *   F_k(d) = sum_i gt_i (I_r(x_i - d) - T_i) = 0
 * (implicit-function rule dd/dtheta = -(dF/dd)^-1 dF/dtheta), which is exact
 * where the Gauss-Newton iterate has converged.
 */

/* right-sided slope of the clamped linear interpolation of a row at X */
static double slope_row(const double *img, int w, int row, double X)
{
    if (X < 0.0 || X >= w - 1.0) return 0.0;
    int x0 = (int)floor(X);
    const double *r = img + (size_t)row * w;
    return r[x0 + 1] - r[x0];
}

/* interpolation taps of a row sample at X (after clamping) */
static void taps_row(int w, double X, int *x0, int *x1, double *t)
{
    if (X < 0.0) X = 0.0;
    if (X > w - 1.0) X = w - 1.0;
    *x0 = (int)floor(X);
    *t = X - *x0;
    *x1 = *x0 + 1 < w ? *x0 + 1 : w - 1;
}

typedef struct {
    double d, E[5], e[5], pik[5], pi, rho, Fd, sigma_prop;
} ob_dpatch;

/* forward of the frozen level-0 function; fills the per-patch values, D,
 * the weight sums W and the loss.  d_override (may be NULL) replaces the
 * Gauss-Newton estimates (the patch disparities as free variables). */
static double diff_forward(const ob_params *p, const double *L, const double *R, int w, int h,
                           const uint8_t *kept, const double *dinit, const double *prop,
                           const uint8_t *valid, int sr_const, double lambda,
                           const double *d_override, double *G, ob_dpatch *dp, double *sr_out,
                           double *D, double *W, double *M)
{
    const int P = p->patch, N = P * P;
    int *ox = (int *)malloc(sizeof(int) * (w + 2)), *oy = (int *)malloc(sizeof(int) * (h + 2));
    int npx = ob_origins(w, P, p->stride, ox), npy = ob_origins(h, P, p->stride, oy);
    ob_sobel_x(L, w, h, G, OB_STORE_F64);
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    double *T = (double *)malloc(sizeof(double) * N), *gt = (double *)malloc(sizeof(double) * N);
    double sumE0 = 0.0;
    int nk = 0;
    for (int k = 0; k < npx * npy; ++k) {
        if (!kept[k]) continue;
        const int x0 = ox[k % npx], y0 = oy[k / npx];
        double gbar = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                T[r * P + c] = L[(size_t)(y0 + r) * w + x0 + c];
                gt[r * P + c] = G[(size_t)(y0 + r) * w + x0 + c];
                gbar += gt[r * P + c];
            }
        gbar /= N;
        double H = 0.0, cT = 0.0;
        for (int i = 0; i < N; ++i) {
            gt[i] -= gbar;
            H += gt[i] * gt[i];
            cT += gt[i] * T[i];
        }
        double d = dinit[k];
        if (d_override) {
            d = d_override[k];
        } else {
            const double dlim = (double)w + 2.0 * P;
            for (int it = 0; it < p->iters; ++it) {
                double acc = 0.0;
                for (int r = 0; r < P; ++r)
                    for (int c = 0; c < P; ++c)
                        acc += gt[r * P + c] * sample_row(R, w, y0 + r, (double)(x0 + c) - d);
                d += (acc - cT) / H;
                if (d > dlim) d = dlim;
                if (d < -dlim) d = -dlim;
            }
        }
        ob_dpatch *q = &dp[k];
        q->d = d;
        double Fd = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c)
                Fd -= gt[r * P + c] * slope_row(R, w, y0 + r, (double)(x0 + c) - d);
        q->Fd = Fd;
        for (int i = 0; i < 5; ++i) {
            double mean = 0.0, E = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c)
                    mean += sample_row(R, w, y0 + r, (double)(x0 + c) - d - delta[i]) - T[r * P + c];
            mean /= N;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    double a = sample_row(R, w, y0 + r, (double)(x0 + c) - d - delta[i]) -
                               T[r * P + c] - mean;
                    E += a * a;
                }
            q->E[i] = E;
        }
        sumE0 += q->E[0];
        ++nk;
    }
    double sr;
    if (sr_const || p->sigma_r_mode == OB_SIGMA_R_FIXED || nk == 0)
        sr = p->sigma_r_mode == OB_SIGMA_R_FIXED ? p->sigma_r_fixed : p->sigma_r_floor;
    else
        sr = sqrt(sumE0 / ((double)nk * P * P));
    *sr_out = sr;
    const double S2 = 2.0 * sr * sr * 25.0;
    const double w0 = ob_gamma_weight(0, p->levels);
    for (int k = 0; k < npx * npy; ++k) {
        if (!kept[k]) continue;
        ob_dpatch *q = &dp[k];
        double Z = 0.0;
        for (int i = 0; i < 5; ++i) {
            q->e[i] = -(q->E[i] - q->E[0]) / S2;
            Z += exp(q->e[i]);
        }
        for (int i = 0; i < 5; ++i) q->pik[i] = exp(q->e[i]) / Z;
        q->pi = 1.0 / Z;
        q->rho = p->use_c2f ? w0 * q->pi + prop[k] : q->pi;
    }
    if (p->use_sgmm) ob_sgmm_table(P, p->sigma_s, M);
    else for (int i = 0; i < N; ++i) M[i] = 1.0;
    for (size_t i = 0; i < (size_t)w * h; ++i) { D[i] = 0.0; W[i] = 0.0; }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            if (!valid[(size_t)y * w + x]) continue;
            double sw = 0.0, swd = 0.0;
            for (int ky = 0; ky < npy; ++ky) {
                if (!(oy[ky] <= y && y < oy[ky] + P)) continue;
                for (int kx = 0; kx < npx; ++kx) {
                    if (!(ox[kx] <= x && x < ox[kx] + P)) continue;
                    int k = ky * npx + kx;
                    if (!kept[k]) continue;
                    double om = dp[k].rho * M[(y - oy[ky]) * P + (x - ox[kx])];
                    sw += om;
                    swd += om * dp[k].d;
                }
            }
            D[(size_t)y * w + x] = sw > 0.0 ? swd / sw : 0.0;
            W[(size_t)y * w + x] = sw;
        }
    double loss = 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * w + x;
            if (!valid[i]) continue;
            loss += fabs(sample_row(R, w, y, x - D[i]) - L[i]);
            if (x + 1 < w && valid[i + 1]) loss += lambda * fabs(D[i] - D[i + 1]);
            if (y + 1 < h && valid[i + w]) loss += lambda * fabs(D[i] - D[i + w]);
        }
    free(T);
    free(gt);
    free(ox);
    free(oy);
    return loss / ((double)w * h);
}

static double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

/* Subgradient of |D_p - D_q| used for the smoothness term: 0 at a tie.
 * Pixels covered by the same patches along one axis have exactly equal D in
 * exact arithmetic (the common sGMM factor cancels, Eq. 12), so ties are
 * structural; a difference within 1e-6 (|D_p| + |D_q|) counts as a tie. */
static double sgn_tie(double a, double dp, double dq)
{
    return fabs(a) <= 1e-6 * (fabs(dp) + fabs(dq)) ? 0.0 : sgn(a);
}

/* Frozen-state forward: returns the loss; D (w*h) and dk (patches) may be NULL. */
double ob_diff_forward(const ob_params *p, const double *L, const double *R, int w, int h,
                       const uint8_t *kept, const double *dinit, const double *prop,
                       const uint8_t *valid, int sr_const, double lambda,
                       const double *d_override, double *D_out, double *dk_out)
{
    /* the differentiable form covers the default fusion at full resolution */
    if (p->weight_mode != OB_WEIGHT_BDIS || p->finest_level != 0 || p->fast_exp) return NAN;
    const int P = p->patch;
    int npx = ob_origins(w, P, p->stride, NULL), npy = ob_origins(h, P, p->stride, NULL);
    ob_dpatch *dp = (ob_dpatch *)calloc((size_t)npx * npy, sizeof(ob_dpatch));
    double *G = (double *)malloc(sizeof(double) * w * h), *D = (double *)malloc(sizeof(double) * w * h);
    double *W = (double *)malloc(sizeof(double) * w * h), *M = (double *)malloc(sizeof(double) * P * P);
    double sr;
    double loss = diff_forward(p, L, R, w, h, kept, dinit, prop, valid, sr_const, lambda, d_override,
                               G, dp, &sr, D, W, M);
    if (D_out) memcpy(D_out, D, sizeof(double) * w * h);
    if (dk_out)
        for (int k = 0; k < npx * npy; ++k) dk_out[k] = kept[k] ? dp[k].d : 0.0;
    free(dp);
    free(G);
    free(D);
    free(W);
    free(M);
    return loss;
}

/* Analytic gradient of ob_diff_forward with respect to I_l, I_r (w*h each,
 * overwritten) and to the patch disparities d_k as free variables (gdk,
 * patches).  gD (w*h, may be NULL) receives dloss/dD.  With gD_in given, the
 * loss step is replaced by that dloss/dD (read at valid pixels): the result
 * is the adjoint of the fusion, posterior, window and patch-solve chain
 * alone (steps 2-5 below), for any loss on D. */
static double diff_grad_impl(const ob_params *p, const double *L, const double *R, int w, int h,
                             const uint8_t *kept, const double *dinit, const double *prop,
                             const uint8_t *valid, int sr_const, double lambda,
                             const double *gD_in, double *gL, double *gR, double *gdk,
                             double *gD_out)
{
    /* the differentiable form covers the default fusion at full resolution */
    if (p->weight_mode != OB_WEIGHT_BDIS || p->finest_level != 0 || p->fast_exp) return NAN;
    const int P = p->patch, N = P * P;
    int *ox = (int *)malloc(sizeof(int) * (w + 2)), *oy = (int *)malloc(sizeof(int) * (h + 2));
    int npx = ob_origins(w, P, p->stride, ox), npy = ob_origins(h, P, p->stride, oy);
    const int np = npx * npy;
    ob_dpatch *dp = (ob_dpatch *)calloc((size_t)np, sizeof(ob_dpatch));
    double *G = (double *)malloc(sizeof(double) * w * h), *D = (double *)malloc(sizeof(double) * w * h);
    double *W = (double *)malloc(sizeof(double) * w * h), *M = (double *)malloc(sizeof(double) * N);
    double *gD = (double *)calloc((size_t)w * h, sizeof(double));
    double *gG = (double *)calloc((size_t)w * h, sizeof(double));
    double sr;
    const double loss = diff_forward(p, L, R, w, h, kept, dinit, prop, valid, sr_const, lambda, NULL,
                                     G, dp, &sr, D, W, M);
    const double inv = 1.0 / ((double)w * h);
    for (size_t i = 0; i < (size_t)w * h; ++i) { gL[i] = 0.0; gR[i] = 0.0; }

    /* 1. loss -> D, and the direct image terms (or the given dloss/dD) */
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * w + x;
            if (!valid[i]) continue;
            if (gD_in) {
                gD[i] = gD_in[i];
                continue;
            }
            double X = x - D[i];
            double r = sample_row(R, w, y, X) - L[i];
            double s = sgn(r) * inv;
            gD[i] += -s * slope_row(R, w, y, X);
            int a0, a1;
            double t;
            taps_row(w, X, &a0, &a1, &t);
            gR[(size_t)y * w + a0] += s * (1.0 - t);
            gR[(size_t)y * w + a1] += s * t;
            gL[i] += -s;
            if (x + 1 < w && valid[i + 1]) {
                double q = lambda * inv * sgn_tie(D[i] - D[i + 1], D[i], D[i + 1]);
                gD[i] += q;
                gD[i + 1] -= q;
            }
            if (y + 1 < h && valid[i + w]) {
                double q = lambda * inv * sgn_tie(D[i] - D[i + w], D[i], D[i + w]);
                gD[i] += q;
                gD[i + w] -= q;
            }
        }
    if (gD_out) memcpy(gD_out, gD, sizeof(double) * w * h);

    /* 2. fusion (Eq. 12) -> d_k and rho_k */
    double *gd = (double *)calloc((size_t)np, sizeof(double));
    double *gpi = (double *)calloc((size_t)np, sizeof(double));
    for (int k = 0; k < np; ++k) {
        if (!kept[k]) continue;
        const int x0 = ox[k % npx], y0 = oy[k / npx];
        double grho = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                size_t i = (size_t)(y0 + r) * w + x0 + c;
                if (!valid[i]) continue;
                double m = M[r * P + c];
                gd[k] += gD[i] * dp[k].rho * m / W[i];
                grho += gD[i] * m * (dp[k].d - D[i]) / W[i];
            }
        gpi[k] = p->use_c2f ? ob_gamma_weight(0, p->levels) * grho : grho;
    }

    /* 3. posterior (Eq. 5-6) -> window energies and sigma_r */
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    const double S2 = 2.0 * sr * sr * 25.0;
    int nk = 0;
    double gsr = 0.0;
    double *gE = (double *)calloc((size_t)np * 5, sizeof(double));
    for (int k = 0; k < np; ++k) {
        if (!kept[k]) continue;
        ++nk;
        const ob_dpatch *q = &dp[k];
        for (int i = 1; i < 5; ++i) {
            /* dpi/de_i = -pi pik_i; de_i/dE_i = -1/S2; de_i/dE_0 = 1/S2 */
            double g = gpi[k] * q->pi * q->pik[i] / S2;
            gE[k * 5 + i] += g;
            gE[k * 5 + 0] -= g;
            /* de_i/dsigma_r = -2 e_i / sigma_r */
            gsr += gpi[k] * (-q->pi * q->pik[i]) * (-2.0 * q->e[i] / sr);
        }
    }
    const int sr_free = !(sr_const || p->sigma_r_mode == OB_SIGMA_R_FIXED) && nk > 0;
    if (sr_free)
        for (int k = 0; k < np; ++k)
            if (kept[k]) gE[k * 5 + 0] += gsr / (2.0 * sr * (double)nk * P * P);

    /* 4. window energies and the patch solve (implicit function) -> images */
    double *T = (double *)malloc(sizeof(double) * N), *gt = (double *)malloc(sizeof(double) * N);
    double *a = (double *)malloc(sizeof(double) * N);
    for (int k = 0; k < np; ++k) {
        if (!kept[k]) continue;
        const int x0 = ox[k % npx], y0 = oy[k / npx];
        const double d = dp[k].d;
        double gbar = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                T[r * P + c] = L[(size_t)(y0 + r) * w + x0 + c];
                gt[r * P + c] = G[(size_t)(y0 + r) * w + x0 + c];
                gbar += gt[r * P + c];
            }
        gbar /= N;
        for (int i = 0; i < N; ++i) gt[i] -= gbar;
        double gdt = gd[k];
        for (int i = 0; i < 5; ++i) {
            const double ge = gE[k * 5 + i];
            double mean = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    a[r * P + c] = sample_row(R, w, y0 + r, (double)(x0 + c) - d - delta[i]) - T[r * P + c];
                    mean += a[r * P + c];
                }
            mean /= N;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    double X = (double)(x0 + c) - d - delta[i];
                    double dE_da = 2.0 * (a[r * P + c] - mean);
                    gdt += ge * dE_da * (-slope_row(R, w, y0 + r, X));
                    int a0, a1;
                    double t;
                    taps_row(w, X, &a0, &a1, &t);
                    gR[(size_t)(y0 + r) * w + a0] += ge * dE_da * (1.0 - t);
                    gR[(size_t)(y0 + r) * w + a1] += ge * dE_da * t;
                    gL[(size_t)(y0 + r) * w + x0 + c] += -ge * dE_da;
                }
        }
        gdk[k] = gdt;
        /* implicit function: v = -gdt / (dF/dd) */
        const double v = -gdt / dp[k].Fd;
        double mres = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c)
                mres += sample_row(R, w, y0 + r, (double)(x0 + c) - d) - T[r * P + c];
        mres /= N;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                double X = (double)(x0 + c) - d;
                int a0, a1;
                double t;
                taps_row(w, X, &a0, &a1, &t);
                gR[(size_t)(y0 + r) * w + a0] += v * gt[r * P + c] * (1.0 - t);
                gR[(size_t)(y0 + r) * w + a1] += v * gt[r * P + c] * t;
                gL[(size_t)(y0 + r) * w + x0 + c] += -v * gt[r * P + c];
                double res = sample_row(R, w, y0 + r, X) - T[r * P + c];
                gG[(size_t)(y0 + r) * w + x0 + c] += v * (res - mres);
            }
    }
    for (int k = 0; k < np; ++k)
        if (!kept[k]) gdk[k] = 0.0;

    /* 5. x-gradient (Sobel-x/8, reflect-101) -> I_l */
    static const double wr[3] = {1.0, 2.0, 1.0};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double g = gG[(size_t)y * w + x];
            if (g == 0.0) continue;
            for (int j = -1; j <= 1; ++j) {
                int yy = reflect101(y + j, h);
                gL[(size_t)yy * w + reflect101(x + 1, w)] += g * wr[j + 1] / 8.0;
                gL[(size_t)yy * w + reflect101(x - 1, w)] -= g * wr[j + 1] / 8.0;
            }
        }
    free(T);
    free(gt);
    free(a);
    free(gE);
    free(gd);
    free(gpi);
    free(dp);
    free(G);
    free(D);
    free(W);
    free(M);
    free(gD);
    free(gG);
    free(ox);
    free(oy);
    return loss;
}

double ob_diff_grad(const ob_params *p, const double *L, const double *R, int w, int h,
                    const uint8_t *kept, const double *dinit, const double *prop,
                    const uint8_t *valid, int sr_const, double lambda, double *gL, double *gR,
                    double *gdk, double *gD_out)
{
    return diff_grad_impl(p, L, R, w, h, kept, dinit, prop, valid, sr_const, lambda, NULL, gL, gR,
                          gdk, gD_out);
}

/* The adjoint chain alone (see diff_grad_impl) for a given dloss/dD. */
void ob_diff_adjoint(const ob_params *p, const double *L, const double *R, int w, int h,
                     const uint8_t *kept, const double *dinit, const double *prop,
                     const uint8_t *valid, int sr_const, const double *gD_in, double *gL,
                     double *gR, double *gdk)
{
    diff_grad_impl(p, L, R, w, h, kept, dinit, prop, valid, sr_const, 0.0, gD_in, gL, gR, gdk,
                   NULL);
}

/* ------------------------------------------------------------------ */
/* differentiable form through every level                              */
/* ------------------------------------------------------------------ */

/* The coarse levels reach the loss only through the propagated probability
 * (Eq. 10): rho_k^(n) = Gamma_n pi_k^(n) + Q^(n+1)(c_k), with
 * Q^(n+1) = sum omega rho / sum omega the fused probability of the coarser
 * level.  The coarse disparity maps only initialise the finer searches, and a
 * converged patch solve F_k(d) = 0 does not depend on its initial value, so
 * they carry no gradient.  The frozen state is per level: kept patches, the
 * Gauss-Newton starting values, whether sigma_r sat at its floor; plus the
 * valid pixels of level 0.  The pyramid is FP64 (no storage rounding). */
typedef struct {
    const uint8_t *kept[OB_MAX_LEVELS];
    const double *dinit[OB_MAX_LEVELS];
    int sr_const[OB_MAX_LEVELS];
    const uint8_t *valid;
} ob_mstate;

typedef struct {
    int w, h, npx, npy;
    int *ox, *oy;
    double *L, *R, *G, *W, *Q, *D;
    ob_dpatch *dp;
    double sr;
} ob_mlevel;

/* bilinear taps of the coarse map at fine position (x, y), as coarse_lookup */
static void coarse_taps(int wc, int hc, double x, double y, int ix[4], int iy[4], double wt[4])
{
    double X = (x + 0.5) / 2.0 - 0.5, Y = (y + 0.5) / 2.0 - 0.5;
    if (X < 0.0) X = 0.0;
    if (X > wc - 1.0) X = wc - 1.0;
    if (Y < 0.0) Y = 0.0;
    if (Y > hc - 1.0) Y = hc - 1.0;
    int x0 = (int)floor(X), y0 = (int)floor(Y);
    int x1 = x0 + 1 < wc ? x0 + 1 : wc - 1, y1 = y0 + 1 < hc ? y0 + 1 : hc - 1;
    double fx = X - x0, fy = Y - y0;
    ix[0] = x0; iy[0] = y0; wt[0] = (1.0 - fx) * (1.0 - fy);
    ix[1] = x1; iy[1] = y0; wt[1] = fx * (1.0 - fy);
    ix[2] = x0; iy[2] = y1; wt[2] = (1.0 - fx) * fy;
    ix[3] = x1; iy[3] = y1; wt[3] = fx * fy;
}

static void mlevels_free(ob_mlevel *lv, int NL)
{
    for (int n = 0; n < NL; ++n) {
        free(lv[n].ox); free(lv[n].oy);
        free(lv[n].L); free(lv[n].R); free(lv[n].G);
        free(lv[n].W); free(lv[n].Q); free(lv[n].D);
        free(lv[n].dp);
    }
}

/* One level of the frozen forward: patch solves, window energies, sigma_r,
 * posterior, rho with the coarser Q, and the fused W, Q (and D at level 0). */
static void mdiff_level(const ob_params *p, const ob_mstate *st, ob_mlevel *lv, int n, int NL,
                        const double *d_override)
{
    ob_mlevel *v = &lv[n];
    const int P = p->patch, N = P * P, w = v->w, h = v->h, npx = v->npx, npy = v->npy;
    const uint8_t *kept = st->kept[n];
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    double *T = (double *)malloc(sizeof(double) * N), *gt = (double *)malloc(sizeof(double) * N);
    double sumE0 = 0.0;
    int nk = 0;
    for (int k = 0; k < npx * npy; ++k) {
        if (!kept[k]) continue;
        const int x0 = v->ox[k % npx], y0 = v->oy[k / npx];
        double gbar = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                T[r * P + c] = v->L[(size_t)(y0 + r) * w + x0 + c];
                gt[r * P + c] = v->G[(size_t)(y0 + r) * w + x0 + c];
                gbar += gt[r * P + c];
            }
        gbar /= N;
        double H = 0.0, cT = 0.0;
        for (int i = 0; i < N; ++i) {
            gt[i] -= gbar;
            H += gt[i] * gt[i];
            cT += gt[i] * T[i];
        }
        double d = st->dinit[n][k];
        if (d_override) {
            d = d_override[k];
        } else {
            const double dlim = (double)w + 2.0 * P;
            for (int it = 0; it < p->iters; ++it) {
                double acc = 0.0;
                for (int r = 0; r < P; ++r)
                    for (int c = 0; c < P; ++c)
                        acc += gt[r * P + c] * sample_row(v->R, w, y0 + r, (double)(x0 + c) - d);
                d += (acc - cT) / H;
                if (d > dlim) d = dlim;
                if (d < -dlim) d = -dlim;
            }
        }
        ob_dpatch *q = &v->dp[k];
        q->d = d;
        double Fd = 0.0;
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c)
                Fd -= gt[r * P + c] * slope_row(v->R, w, y0 + r, (double)(x0 + c) - d);
        q->Fd = Fd;
        for (int i = 0; i < 5; ++i) {
            double mean = 0.0, E = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c)
                    mean += sample_row(v->R, w, y0 + r, (double)(x0 + c) - d - delta[i]) - T[r * P + c];
            mean /= N;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    double a = sample_row(v->R, w, y0 + r, (double)(x0 + c) - d - delta[i]) -
                               T[r * P + c] - mean;
                    E += a * a;
                }
            q->E[i] = E;
        }
        sumE0 += q->E[0];
        ++nk;
    }
    if (st->sr_const[n] || p->sigma_r_mode == OB_SIGMA_R_FIXED || nk == 0)
        v->sr = p->sigma_r_mode == OB_SIGMA_R_FIXED ? p->sigma_r_fixed : p->sigma_r_floor;
    else
        v->sr = sqrt(sumE0 / ((double)nk * P * P));
    const double S2 = 2.0 * v->sr * v->sr * 25.0;
    const double gw = ob_gamma_weight(n, NL);
    for (int k = 0; k < npx * npy; ++k) {
        if (!kept[k]) continue;
        ob_dpatch *q = &v->dp[k];
        double Z = 0.0;
        for (int i = 0; i < 5; ++i) {
            q->e[i] = -(q->E[i] - q->E[0]) / S2;
            Z += exp(q->e[i]);
        }
        for (int i = 0; i < 5; ++i) q->pik[i] = exp(q->e[i]) / Z;
        q->pi = 1.0 / Z;
        double prop = 0.0;
        if (p->use_c2f && n + 1 < NL) {
            const double cx = v->ox[k % npx] + (P - 1) / 2.0, cy = v->oy[k / npx] + (P - 1) / 2.0;
            prop = coarse_lookup(lv[n + 1].Q, lv[n + 1].w, lv[n + 1].h, cx, cy);
        }
        q->rho = p->use_c2f ? gw * q->pi + prop : q->pi;
    }
    double *M = (double *)malloc(sizeof(double) * N);
    if (p->use_sgmm) ob_sgmm_table(P, p->sigma_s, M);
    else for (int i = 0; i < N; ++i) M[i] = 1.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double sw = 0.0, swd = 0.0, swr = 0.0;
            for (int ky = 0; ky < npy; ++ky) {
                if (!(v->oy[ky] <= y && y < v->oy[ky] + P)) continue;
                for (int kx = 0; kx < npx; ++kx) {
                    if (!(v->ox[kx] <= x && x < v->ox[kx] + P)) continue;
                    int k = ky * npx + kx;
                    if (!kept[k]) continue;
                    double om = v->dp[k].rho * M[(y - v->oy[ky]) * P + (x - v->ox[kx])];
                    sw += om;
                    swd += om * v->dp[k].d;
                    swr += om * v->dp[k].rho;
                }
            }
            size_t i = (size_t)y * w + x;
            v->W[i] = sw;
            v->Q[i] = sw > 0.0 ? swr / sw : 0.0;
            if (v->D) v->D[i] = sw > 0.0 ? swd / sw : 0.0;
        }
    free(M);
    free(T);
    free(gt);
}

/* Builds the levels (FP64 pyramid, gradients, patch grids) and runs the
 * frozen forward coarse to fine; returns the loss. */
static double mdiff_forward(const ob_params *p, const double *L0, const double *R0, int w, int h,
                            const ob_mstate *st, double lambda, const double *d_override0,
                            ob_mlevel *lv)
{
    const int NL = p->levels, P = p->patch;
    memset(lv, 0, sizeof(ob_mlevel) * NL);
    for (int n = 0; n < NL; ++n) {
        ob_mlevel *v = &lv[n];
        v->w = ob_level_dim(w, n);
        v->h = ob_level_dim(h, n);
        size_t px = (size_t)v->w * v->h;
        v->L = (double *)malloc(sizeof(double) * px);
        v->R = (double *)malloc(sizeof(double) * px);
        v->G = (double *)malloc(sizeof(double) * px);
        v->W = (double *)malloc(sizeof(double) * px);
        v->Q = (double *)malloc(sizeof(double) * px);
        v->D = n == 0 ? (double *)malloc(sizeof(double) * px) : NULL;
        v->ox = (int *)malloc(sizeof(int) * (v->w + 2));
        v->oy = (int *)malloc(sizeof(int) * (v->h + 2));
        v->npx = ob_origins(v->w, P, p->stride, v->ox);
        v->npy = ob_origins(v->h, P, p->stride, v->oy);
        v->dp = (ob_dpatch *)calloc((size_t)v->npx * v->npy, sizeof(ob_dpatch));
        if (n == 0) {
            memcpy(v->L, L0, sizeof(double) * px);
            memcpy(v->R, R0, sizeof(double) * px);
        } else {
            ob_pyr_down(lv[n - 1].L, lv[n - 1].w, lv[n - 1].h, v->L, OB_STORE_F64);
            ob_pyr_down(lv[n - 1].R, lv[n - 1].w, lv[n - 1].h, v->R, OB_STORE_F64);
        }
        ob_sobel_x(v->L, v->w, v->h, v->G, OB_STORE_F64);
    }
    for (int n = NL - 1; n >= 0; --n) mdiff_level(p, st, lv, n, NL, n == 0 ? d_override0 : NULL);
    const ob_mlevel *v = &lv[0];
    double loss = 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * w + x;
            if (!st->valid[i]) continue;
            loss += fabs(sample_row(v->R, w, y, x - v->D[i]) - v->L[i]);
            if (x + 1 < w && st->valid[i + 1]) loss += lambda * fabs(v->D[i] - v->D[i + 1]);
            if (y + 1 < h && st->valid[i + w]) loss += lambda * fabs(v->D[i] - v->D[i + w]);
        }
    return loss / ((double)w * h);
}

double ob_mdiff_forward(const ob_params *p, const double *L, const double *R, int w, int h,
                        const ob_mstate *st, double lambda, const double *d_override,
                        double *D_out, double *dk_out)
{
    if (p->weight_mode != OB_WEIGHT_BDIS || p->finest_level != 0 || p->fast_exp) return NAN;
    ob_mlevel lv[OB_MAX_LEVELS];
    const double loss = mdiff_forward(p, L, R, w, h, st, lambda, d_override, lv);
    if (D_out) memcpy(D_out, lv[0].D, sizeof(double) * w * h);
    if (dk_out)
        for (int k = 0; k < lv[0].npx * lv[0].npy; ++k) dk_out[k] = lv[0].dp[k].d;
    mlevels_free(lv, p->levels);
    return loss;
}

/* Analytic gradient of ob_mdiff_forward with respect to both level-0 images
 * (and the level-0 patch disparities, images held fixed).  Reverse order:
 * the loss and the level-0 fusion; then per level, finest first, the Q-map
 * fusion adjoint (n >= 1), the posterior, sigma_r, the window energies and
 * the implicit-function adjoint of each solve into that level's images, the
 * Sobel transpose, and the bilinear transpose of rho's coarse term into the
 * next level's Q map; finally the pyramid transpose, coarsest first. */
static double mdiff_grad_impl(const ob_params *p, const double *L, const double *R, int w, int h,
                              const ob_mstate *st, double lambda, const double *gD_in,
                              double *gL_out, double *gR_out, double *gdk_out)
{
    if (p->weight_mode != OB_WEIGHT_BDIS || p->finest_level != 0 || p->fast_exp) return NAN;
    const int NL = p->levels, P = p->patch, N = P * P;
    ob_mlevel lv[OB_MAX_LEVELS];
    const double loss = mdiff_forward(p, L, R, w, h, st, lambda, NULL, lv);
    double *gLv[OB_MAX_LEVELS], *gRv[OB_MAX_LEVELS], *gQv[OB_MAX_LEVELS];
    for (int n = 0; n < NL; ++n) {
        size_t px = (size_t)lv[n].w * lv[n].h;
        gLv[n] = (double *)calloc(px, sizeof(double));
        gRv[n] = (double *)calloc(px, sizeof(double));
        gQv[n] = (double *)calloc(px, sizeof(double));
    }
    double *M = (double *)malloc(sizeof(double) * N);
    if (p->use_sgmm) ob_sgmm_table(P, p->sigma_s, M);
    else for (int i = 0; i < N; ++i) M[i] = 1.0;
    double delta[5];
    ob_window_offsets(p->window_step, delta);
    const double inv = 1.0 / ((double)w * h);

    /* 1. loss -> D and the direct image terms (level 0), or the given dloss/dD */
    double *gD = (double *)calloc((size_t)w * h, sizeof(double));
    {
        const ob_mlevel *v = &lv[0];
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                size_t i = (size_t)y * w + x;
                if (!st->valid[i]) continue;
                if (gD_in) {
                    gD[i] = gD_in[i];
                    continue;
                }
                double X = x - v->D[i];
                double r = sample_row(v->R, w, y, X) - v->L[i];
                double s = sgn(r) * inv;
                gD[i] += -s * slope_row(v->R, w, y, X);
                int a0, a1;
                double t;
                taps_row(w, X, &a0, &a1, &t);
                gRv[0][(size_t)y * w + a0] += s * (1.0 - t);
                gRv[0][(size_t)y * w + a1] += s * t;
                gLv[0][i] += -s;
                if (x + 1 < w && st->valid[i + 1]) {
                    double q = lambda * inv * sgn_tie(v->D[i] - v->D[i + 1], v->D[i], v->D[i + 1]);
                    gD[i] += q;
                    gD[i + 1] -= q;
                }
                if (y + 1 < h && st->valid[i + w]) {
                    double q = lambda * inv * sgn_tie(v->D[i] - v->D[i + w], v->D[i], v->D[i + w]);
                    gD[i] += q;
                    gD[i + w] -= q;
                }
            }
    }

    double *T = (double *)malloc(sizeof(double) * N), *gt = (double *)malloc(sizeof(double) * N);
    double *a = (double *)malloc(sizeof(double) * N);
    for (int n = 0; n < NL; ++n) {
        ob_mlevel *v = &lv[n];
        const int lw = v->w, lh = v->h, npx = v->npx, npy = v->npy, np = npx * npy;
        const uint8_t *kept = st->kept[n];
        double *gd = (double *)calloc((size_t)np, sizeof(double));
        double *grho = (double *)calloc((size_t)np, sizeof(double));
        double *gG = (double *)calloc((size_t)lw * lh, sizeof(double));
        /* 2. fusion adjoint: D (level 0, Eq. 12) and Q (levels >= 1) */
        for (int k = 0; k < np; ++k) {
            if (!kept[k]) continue;
            const int x0 = v->ox[k % npx], y0 = v->oy[k / npx];
            const ob_dpatch *q = &v->dp[k];
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    size_t i = (size_t)(y0 + r) * lw + x0 + c;
                    if (v->W[i] <= 0.0) continue;
                    double m = M[r * P + c];
                    if (n == 0 && st->valid[i]) {
                        gd[k] += gD[i] * q->rho * m / v->W[i];
                        grho[k] += gD[i] * m * (q->d - v->D[i]) / v->W[i];
                    }
                    /* Q = sum rho^2 M / sum rho M: dQ/drho_k = M (2 rho_k - Q) / W */
                    if (n > 0) grho[k] += gQv[n][i] * m * (2.0 * q->rho - v->Q[i]) / v->W[i];
                }
        }
        /* 3. rho = Gamma_n pi + Q^(n+1)(centre): pi, and the coarser Q map */
        const double gw = ob_gamma_weight(n, NL);
        double *gpi = (double *)calloc((size_t)np, sizeof(double));
        for (int k = 0; k < np; ++k) {
            if (!kept[k]) continue;
            gpi[k] = p->use_c2f ? gw * grho[k] : grho[k];
            if (p->use_c2f && n + 1 < NL && grho[k] != 0.0) {
                const double cx = v->ox[k % npx] + (P - 1) / 2.0, cy = v->oy[k / npx] + (P - 1) / 2.0;
                int ix[4], iy[4];
                double wt[4];
                coarse_taps(lv[n + 1].w, lv[n + 1].h, cx, cy, ix, iy, wt);
                for (int j = 0; j < 4; ++j)
                    gQv[n + 1][(size_t)iy[j] * lv[n + 1].w + ix[j]] += grho[k] * wt[j];
            }
        }
        /* 4. posterior (Eq. 5-6) -> window energies and sigma_r */
        const double sr = v->sr, S2 = 2.0 * sr * sr * 25.0;
        int nk = 0;
        double gsr = 0.0;
        double *gE = (double *)calloc((size_t)np * 5, sizeof(double));
        for (int k = 0; k < np; ++k) {
            if (!kept[k]) continue;
            ++nk;
            const ob_dpatch *q = &v->dp[k];
            for (int i = 1; i < 5; ++i) {
                double g = gpi[k] * q->pi * q->pik[i] / S2;
                gE[k * 5 + i] += g;
                gE[k * 5 + 0] -= g;
                gsr += gpi[k] * (-q->pi * q->pik[i]) * (-2.0 * q->e[i] / sr);
            }
        }
        const int sr_free = !(st->sr_const[n] || p->sigma_r_mode == OB_SIGMA_R_FIXED) && nk > 0;
        if (sr_free)
            for (int k = 0; k < np; ++k)
                if (kept[k]) gE[k * 5 + 0] += gsr / (2.0 * sr * (double)nk * P * P);
        /* 5. window energies and the patch solve -> this level's images */
        for (int k = 0; k < np; ++k) {
            if (!kept[k]) continue;
            const int x0 = v->ox[k % npx], y0 = v->oy[k / npx];
            const double d = v->dp[k].d;
            double gbar = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    T[r * P + c] = v->L[(size_t)(y0 + r) * lw + x0 + c];
                    gt[r * P + c] = v->G[(size_t)(y0 + r) * lw + x0 + c];
                    gbar += gt[r * P + c];
                }
            gbar /= N;
            for (int i = 0; i < N; ++i) gt[i] -= gbar;
            double gdt = gd[k];
            for (int i = 0; i < 5; ++i) {
                const double ge = gE[k * 5 + i];
                double mean = 0.0;
                for (int r = 0; r < P; ++r)
                    for (int c = 0; c < P; ++c) {
                        a[r * P + c] = sample_row(v->R, lw, y0 + r, (double)(x0 + c) - d - delta[i]) -
                                       T[r * P + c];
                        mean += a[r * P + c];
                    }
                mean /= N;
                for (int r = 0; r < P; ++r)
                    for (int c = 0; c < P; ++c) {
                        double X = (double)(x0 + c) - d - delta[i];
                        double dE_da = 2.0 * (a[r * P + c] - mean);
                        gdt += ge * dE_da * (-slope_row(v->R, lw, y0 + r, X));
                        int a0, a1;
                        double t;
                        taps_row(lw, X, &a0, &a1, &t);
                        gRv[n][(size_t)(y0 + r) * lw + a0] += ge * dE_da * (1.0 - t);
                        gRv[n][(size_t)(y0 + r) * lw + a1] += ge * dE_da * t;
                        gLv[n][(size_t)(y0 + r) * lw + x0 + c] += -ge * dE_da;
                    }
            }
            if (n == 0 && gdk_out) gdk_out[k] = gdt;
            const double vF = -gdt / v->dp[k].Fd;
            double mres = 0.0;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c)
                    mres += sample_row(v->R, lw, y0 + r, (double)(x0 + c) - d) - T[r * P + c];
            mres /= N;
            for (int r = 0; r < P; ++r)
                for (int c = 0; c < P; ++c) {
                    double X = (double)(x0 + c) - d;
                    int a0, a1;
                    double t;
                    taps_row(lw, X, &a0, &a1, &t);
                    gRv[n][(size_t)(y0 + r) * lw + a0] += vF * gt[r * P + c] * (1.0 - t);
                    gRv[n][(size_t)(y0 + r) * lw + a1] += vF * gt[r * P + c] * t;
                    gLv[n][(size_t)(y0 + r) * lw + x0 + c] += -vF * gt[r * P + c];
                    double res = sample_row(v->R, lw, y0 + r, X) - T[r * P + c];
                    gG[(size_t)(y0 + r) * lw + x0 + c] += vF * (res - mres);
                }
        }
        if (n == 0 && gdk_out)
            for (int k = 0; k < np; ++k)
                if (!kept[k]) gdk_out[k] = 0.0;
        /* 6. Sobel-x/8 transpose -> this level's left image */
        static const double wr[3] = {1.0, 2.0, 1.0};
        for (int y = 0; y < lh; ++y)
            for (int x = 0; x < lw; ++x) {
                double g = gG[(size_t)y * lw + x];
                if (g == 0.0) continue;
                for (int j = -1; j <= 1; ++j) {
                    int yy = reflect101(y + j, lh);
                    gLv[n][(size_t)yy * lw + reflect101(x + 1, lw)] += g * wr[j + 1] / 8.0;
                    gLv[n][(size_t)yy * lw + reflect101(x - 1, lw)] -= g * wr[j + 1] / 8.0;
                }
            }
        free(gd);
        free(grho);
        free(gpi);
        free(gE);
        free(gG);
    }
    /* 7. pyramid transpose, coarsest first: the blur-and-decimate of level
     * n - 1 gives level n, so its gradient flows back to level n - 1 */
    static const double k5[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    for (int n = NL - 1; n >= 1; --n) {
        const int w1 = lv[n].w, h1 = lv[n].h, w0 = lv[n - 1].w, h0 = lv[n - 1].h;
        for (int Y = 0; Y < h1; ++Y)
            for (int X = 0; X < w1; ++X) {
                const double gl = gLv[n][(size_t)Y * w1 + X], gr = gRv[n][(size_t)Y * w1 + X];
                if (gl == 0.0 && gr == 0.0) continue;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        size_t o = (size_t)reflect101(2 * Y + j, h0) * w0 + reflect101(2 * X + i, w0);
                        gLv[n - 1][o] += k5[j + 2] * k5[i + 2] * gl;
                        gRv[n - 1][o] += k5[j + 2] * k5[i + 2] * gr;
                    }
            }
    }
    memcpy(gL_out, gLv[0], sizeof(double) * w * h);
    memcpy(gR_out, gRv[0], sizeof(double) * w * h);
    for (int n = 0; n < NL; ++n) {
        free(gLv[n]);
        free(gRv[n]);
        free(gQv[n]);
    }
    free(gD);
    free(M);
    free(T);
    free(gt);
    free(a);
    mlevels_free(lv, NL);
    return loss;
}

double ob_mdiff_grad(const ob_params *p, const double *L, const double *R, int w, int h,
                     const ob_mstate *st, double lambda, double *gL_out, double *gR_out,
                     double *gdk_out)
{
    return mdiff_grad_impl(p, L, R, w, h, st, lambda, NULL, gL_out, gR_out, gdk_out);
}

/* The adjoint through every level alone, for a given level-0 dloss/dD. */
void ob_mdiff_adjoint(const ob_params *p, const double *L, const double *R, int w, int h,
                      const ob_mstate *st, const double *gD_in, double *gL_out, double *gR_out,
                      double *gdk_out)
{
    mdiff_grad_impl(p, L, R, w, h, st, 0.0, gD_in, gL_out, gR_out, gdk_out);
}
