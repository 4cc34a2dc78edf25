/*
 * bdis.h -- C ABI of the GB300 (sm_103a) BDIS library (libbdis.so).
 *
 * BDIS (Bayesian Dense Inverse Search, arXiv 2205.03133) estimates a dense
 * disparity map, and optionally a per-pixel disparity variance, for a
 * rectified stereo pair.  Per pyramid level, coarsest first (Fig. 1):
 *   - image pyramid and left x-gradient (Sec. III-A: the inverse-
 *     compositional Jacobian is computed once);
 *   - per-patch 1D inverse-compositional Gauss-Newton search (Eq. 1);
 *   - window energies, rejection of saddle / unconverged patches, dynamic
 *     sigma_r and the window posterior (Sec. III-B, Eq. 4-6);
 *   - coarse-to-fine probability propagation (Sec. III-D, Eq. 10-11);
 *   - sGMM-weighted dense fusion (Sec. III-C, Eq. 8-9, Eq. 12);
 *   - optional per-patch PDF fit and pixel variance (Sec. III-E, Eq. 14-17).
 *
 * Conventions shared by every entry point
 *   - Disparity d >= 0 with I_r(x - d, y) ~= I_l(x, y) (the paper's u = -d).
 *   - Images are 8-bit grayscale, row-major, `pitch` bytes between rows
 *     (pitch >= w).  Outputs are dense row-major float/uint8 arrays of w*h.
 *   - Device pointers are caller-owned CUDA device memory on the current
 *     device; the library never frees them.  `stream` is a cudaStream_t
 *     (NULL = legacy default stream).  Device calls are asynchronous on that
 *     stream: outputs are ready when the stream reaches that point.
 *   - Errors are returned as bdis_status; nothing crosses the ABI as an
 *     exception.  Arguments are validated before any launch; on an error no
 *     output is written.  bdis_last_error() gives a one-line reason.
 *   - Pixels with no valid estimate get disp = NaN, var = NaN, valid = 0.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef BDIS_H
#define BDIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BDIS_OK = 0,
    BDIS_EINVAL = 1,        /* bad argument (null pointer, size, parameter) */
    BDIS_ENOMEM = 2,        /* device or pinned host allocation failed       */
    BDIS_ECUDA = 3,         /* a CUDA runtime call or a launch failed        */
    BDIS_EUNSUPPORTED = 4   /* valid request outside what this build handles */
} bdis_status;

/* Storage type of the pyramid levels 1..L-1 and of the x-gradient images.
 * Level 0 is the caller's 8-bit image.  Arithmetic is FP32 in every case.
 * U8: the pyramid levels as 8-bit integers (the FP32 blur rounded to the
 * nearest integer, ties to even, within 0..255) and the gradients as FP16
 * (Sobel-x/8 of 8-bit values is a multiple of 1/8 within +-127.5, which
 * FP16 holds exactly).  Not available to the persistent and cooperative
 * forms, to the adjoint through every level and to bdis_match_noalloc. */
typedef enum { BDIS_STORE_F32 = 0, BDIS_STORE_F16 = 1, BDIS_STORE_U8 = 2 } bdis_storage;

/* Reading of the dynamic scale sigma_r^(n) (text after Eq. 6):
 * POOLED  sqrt(sum_valid E_k(0) / (N_valid P^2)) -- the default;
 * LITERAL population std over valid patches of E_k(0);
 * FIXED   sigma_r_fixed (the ablation of Table VII uses 8). */
typedef enum {
    BDIS_SIGMA_R_POOLED = 0,
    BDIS_SIGMA_R_LITERAL = 1,
    BDIS_SIGMA_R_FIXED = 2
} bdis_sigma_r_mode;

/* Fusion weights of the densification.
 * BDIS: omega_k(x) = rho_k m[x - ox_k] m[y - oy_k], the sGMM kernel times the
 *       propagated probability (Eq. 8, Eq. 12) -- the default;
 * DIS:  omega_k(x) = 1 / max(1, r_k(x)^2), the inverse photometric residual
 *       of Eq. 2, with r_k(x) = I_r(x - d_k) - I_l(x) - mu_k the residual of
 *       patch k at pixel x after its mean offset mu_k (mean normalisation as
 *       in the search).  Q and V use the same normalised weights. */
typedef enum { BDIS_WEIGHT_BDIS = 0, BDIS_WEIGHT_DIS = 1 } bdis_weight_mode;

typedef struct {
    int patch;            /* P: patch side (px), 4..16                       */
    int stride;           /* S: patch stride (px), 1..P                      */
    int levels;           /* L: pyramid levels incl. full resolution, 1..8   */
    int iters;            /* Gauss-Newton iterations per patch (fixed), >= 0 */
    float sigma_s;        /* sGMM spatial sigma (Eq. 8), paper: 4            */
    float window_step;    /* window offsets {0, +-h, +-2h} (Sec. IV-A: 0.5)  */
    float conv_eps;       /* max |last GN update| of a kept patch, 0.05      */
    float valid_gamma;    /* min in-image sample ratio of a kept patch, 0.75 */
    float pix_thresh;     /* min fused probability of a valid pixel, 0.15    */
    float search_radius;  /* tau: max |d - d_init| (px at the level); <= 0: P */
    int sigma_r_mode;     /* bdis_sigma_r_mode                               */
    float sigma_r_floor;  /* lower bound of sigma_r (DN), default 0.5        */
    float sigma_r_fixed;  /* value for BDIS_SIGMA_R_FIXED, default 8         */
    int variance;         /* 1: per-patch PDF fit + pixel variance (Eq. 14-17) */
    int pdf_iters;        /* GN iterations of the PDF fit (Sec. III-E: 10)   */
    float pdf_resid;      /* max RMS log residual of the fit (Sec. III-E: 0.1) */
    int storage;          /* bdis_storage                                    */
    float hess_eps;       /* patch rejected as flat if H < hess_eps * P^2    */
    int use_sgmm;         /* 0: equal pixel weights (ablation, Table VII)    */
    int use_c2f;          /* 0: no coarse-to-fine probability (ablation)     */
    int weight_mode;      /* bdis_weight_mode of the fusion                  */
    int finest_level;     /* finest processed level f, 0..L-1 (default 0).
                             f > 0: levels < f are only pyramid steps; the
                             level-f result is upsampled to full resolution:
                             disp = 2^f bilinear(D_f), var = 4^f bilinear(V_f)
                             at level-f coordinate (x + 0.5) / 2^f - 0.5,
                             valid iff every level-f pixel with a non-zero
                             bilinear weight is valid (Sec. IV-A: 2^1)      */
    int fast_exp;         /* 1: Schraudolph's exponential in the window
                             posterior (Sec. IV, technical details)         */
} bdis_params;

typedef struct bdis_handle bdis_handle;

/* One stereo pair of a batch; all pointers are device memory. */
typedef struct {
    const uint8_t *left, *right;  /* w x h, `pitch` bytes per row           */
    int w, h, pitch;
    float *disp;                  /* w*h out                                 */
    float *var;                   /* w*h out, may be NULL (or variance off)  */
    uint8_t *valid;               /* w*h out                                 */
} bdis_pair;

/* Per-call counters of the last completed call on a handle. */
typedef struct {
    int levels, pairs;
    int patches[8];          /* patches searched per level (all pairs)       */
    int valid_patches[8];    /* patches kept per level (all pairs)           */
    float sigma_r[8];        /* sigma_r per level of the first pair           */
    long long valid_pixels;  /* valid output pixels (all pairs)              */
    int persistent;          /* 1 if the call ran in the persistent form, 2 if
                                its coarse levels ran in one cooperative launch */
    int barrier_timeouts;    /* persistent form: a grid-barrier wait ran out  */
} bdis_stats;

/* Fills `p` with the defaults (8x8 patches, stride 4, 3 levels, 8 iterations,
 * paper values from Sec. IV-A / III-E for the rest, FP32 pyramids). */
void bdis_default_params(bdis_params *p);

/* Validates `p` and creates a handle.  The handle owns a device scratch
 * arena (pyramids, patch records, coarse maps) that grows on demand and is
 * freed by bdis_destroy.  No CUDA call is made here. */
bdis_status bdis_create(const bdis_params *p, bdis_handle **out);
void bdis_destroy(bdis_handle *h);
const char *bdis_strerror(bdis_status s);
/* One-line description of the last error on this handle (never NULL). */
const char *bdis_last_error(const bdis_handle *h);
/* Copies the handle's parameters (with search_radius resolved). */
bdis_status bdis_get_params(const bdis_handle *h, bdis_params *out);

/* Dense BDIS on one pair of device images (the whole pipeline, Fig. 1).
 * w, h must leave the coarsest level at least `patch` pixels per axis:
 * ceil(w / 2^(L-1)) >= P and ceil(h / 2^(L-1)) >= P.  `var` may be NULL;
 * it is written only when params.variance is 1.  Asynchronous on `stream`. */
bdis_status bdis_match(bdis_handle *h, const uint8_t *left, const uint8_t *right, int w,
                       int hgt, int pitch, float *disp, float *var, uint8_t *valid,
                       void *stream);

/* Same computation with HOST buffers, on `stream`; the call returns after
 * the stream has finished (host outputs are ready).  Page-locked buffers the
 * device can address are read and written in place by the kernels
 * (BDIS_OPT_HOST_MAPPED); other host memory goes through staging copies
 * (inputs copied to the device, outputs copied back). */
bdis_status bdis_match_host(bdis_handle *h, const uint8_t *left, const uint8_t *right, int w,
                            int hgt, int pitch, float *disp, float *var, uint8_t *valid,
                            void *stream);

/* Many pairs of possibly different sizes in one pass: every stage runs as
 * one launch per pyramid level over all pairs (work decomposed through a
 * per-level descriptor table).  All pairs share the handle's parameters.
 * Results are identical to calling bdis_match on each pair. */
bdis_status bdis_match_batched(bdis_handle *h, int n, const bdis_pair *pairs, void *stream);

/* Allocation-free variant of bdis_match (the paper has no counterpart: it
 * exists for callers that cannot allocate device memory).  Callers such as a
 * video pipeline whose memory pool owns the whole device, a process with a
 * fixed device-memory budget, or a latency-critical loop that cannot take
 * the device-wide synchronisation of cudaMalloc/cudaFree, get the same
 * result as bdis_match without any allocation: no handle, no cudaMalloc,
 * cudaFree or pinned staging.  The scratch (pyramids, patch records, coarse
 * maps, descriptor table) lives in one static device array of 32 MiB that
 * every GPU loading the library holds until the process exits; the caller
 * passes inputs and outputs as for bdis_match (device pointers).
 *   - Returns BDIS_EUNSUPPORTED, before any launch, when the pair needs more
 *     than that 32 MiB (e.g. 1920x1080 with FP32 pyramids); a 640x480 pair
 *     fits with any settings, a 1280x720 pair with 8x8 patches, stride 4,
 *     3 levels.  BDIS_EINVAL for invalid parameters or sizes.
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (other streams or host threads) race and
 *     must be serialised by the caller.
 *   - Asynchronous on `stream`; no bdis_last_error text (no handle). */
bdis_status bdis_match_noalloc(const bdis_params *p, const uint8_t *left, const uint8_t *right,
                               int w, int hgt, int pitch, float *disp, float *var,
                               uint8_t *valid, void *stream);

/* Counters of the last call (synchronises `stream` to read them).  The
 * counters are filled in every case; the status is BDIS_ECUDA when a
 * persistent-form call whose grid-barrier wait ran out has not been reported
 * yet (barrier_timeouts = 1 if it was the last call). */
bdis_status bdis_get_stats(bdis_handle *h, bdis_stats *out, void *stream);

/* Waits until `stream` has finished the handle's calls and returns their
 * device-side status: BDIS_ECUDA (reason in bdis_last_error) when a
 * grid-barrier wait of a persistent-form call ran out, else BDIS_OK. */
bdis_status bdis_wait(bdis_handle *h, void *stream);

/* ---- differentiable form (finest level) ----
 * A forward on float images followed by a loss and its adjoint.  The
 * function differentiated is the finest level with the forward's discrete
 * state frozen (kept patches, their initial estimates and inherited coarse
 * probabilities, valid pixels, sigma_r at its floor or not):
 *   d_k  root of F_k(d) = sum_i gt_i (I_r(x_i - d) - T_i) (Eq. 1), reached by
 *        the forward's Gauss-Newton iterations;
 *   E_k, pi_k, rho_k (Eq. 5-6, 10-11), D = sum omega_k d_k / sum omega_k (Eq. 12).
 * The patch adjoint is the implicit-function rule
 *   dd_k/dtheta = -(dF_k/dd)^-1 dF_k/dtheta,
 * exact where the iteration has converged.  The coarser levels are frozen.
 * The paper has no loss or gradient: they are the extension that makes BDIS
 * usable inside a learned pipeline. */

typedef struct {
    const float *left, *right;    /* w x h float images, `pitch` ELEMENTS per row */
    int w, h, pitch;
    float *disp, *var;            /* w*h out (var may be NULL)                    */
    uint8_t *valid;               /* w*h out                                      */
} bdis_pair_f32;

/* Forward on float images (same pipeline as bdis_match; the level-0 images
 * are read as float).  Required before bdis_loss / bdis_backward.  Its state
 * (pyramids, gradients, patch and fusion records, weight sums, sigma_r) stays
 * in the handle until the handle's next call. */
bdis_status bdis_match_f32(bdis_handle *h, const float *left, const float *right, int w, int hgt,
                           int pitch, float *disp, float *var, uint8_t *valid, void *stream);
bdis_status bdis_match_batched_f32(bdis_handle *h, int n, const bdis_pair_f32 *pairs,
                                   void *stream);

/* Caller-owned state of one differentiable forward (the saved tensors of an
 * autograd graph).  A forward run into a bdis_saved keeps its state -- the
 * pyramids, x-gradients, patch and fusion records, fusion-weight sums and
 * sigma_r of every level (Sec. III-A..III-C), plus the caller's level-0
 * image and output pointers -- in the object's own device memory, so any
 * number of forwards on one handle can be differentiated later, each through
 * its own state, in any order.
 *   - bdis_saved_create ties the object to `h` (no CUDA call; the device
 *     memory is allocated by the first forward into it, grows, never
 *     shrinks) and bdis_saved_destroy frees it (synchronising the device).
 *     A saved object outlives its handle only to be destroyed.
 *   - bdis_match_batched_f32_saved is bdis_match_batched_f32 with the state
 *     kept in `s`; running it again into the same `s` replaces the state.
 *   - The caller keeps that forward's images and outputs (left, right, disp,
 *     valid) unchanged until the last bdis_loss / bdis_backward on `s`.
 *   - BDIS_EINVAL for an `s` created on another handle or holding no forward. */
typedef struct bdis_saved bdis_saved;
bdis_status bdis_saved_create(bdis_handle *h, bdis_saved **out);
void bdis_saved_destroy(bdis_saved *s);
bdis_status bdis_match_batched_f32_saved(bdis_handle *h, int n, const bdis_pair_f32 *pairs,
                                         bdis_saved *s, void *stream);

/* Per-pair gradient buffers (device, dense w*h unless stated). */
typedef struct {
    float *loss;          /* 1 float: the pair's loss (bdis_loss)                   */
    float *g_disp;        /* dloss/dD (written by bdis_loss, read by bdis_backward) */
    float *g_left;        /* dloss/dI_l                                            */
    float *g_right;       /* dloss/dI_r                                            */
    float *g_patch_disp;  /* npx*npy level-0 patches: dloss/dd_k with the images
                             held fixed (bdis_backward), 0 for a rejected
                             patch; may be NULL                                */
} bdis_grad;

/* Loss of a float forward -- the one kept in `s`, or with s == NULL the
 * handle's last call (bdis_match_f32 / _batched_f32) -- for every pair:
 *   loss = ( sum_{valid x} |I_r(x - D(x)) - I_l(x)|
 *          + lambda sum_{valid 4-neighbour pairs} |D(p) - D(q)| ) / (w h)
 * (I_r sampled by clamped linear interpolation along x).  Writes loss,
 * g_disp, and the direct image terms: g_left is overwritten, g_right is
 * zeroed and then accumulated.  `g` has one entry per pair of that forward. */
bdis_status bdis_loss(bdis_handle *h, const bdis_saved *s, float lambda, const bdis_grad *g,
                      void *stream);

/* Adjoint of a float forward (the one kept in `s`, or with s == NULL the
 * handle's last call): reads g_disp (from bdis_loss or from the caller's own
 * loss), ADDS dloss/dI_l and dloss/dI_r to g_left / g_right (zero them first
 * when g_disp comes from another loss) and writes g_patch_disp.  Needs the
 * pooled or fixed sigma_r (BDIS_EUNSUPPORTED for LITERAL).  Image gradients
 * are accumulated with float atomics, so their last bits may differ from
 * run to run.  The handle's backward scratch is shared by all its saved
 * states: backward calls of one handle on different streams must not overlap. */
bdis_status bdis_backward(bdis_handle *h, const bdis_saved *s, const bdis_grad *g, void *stream);

/* ---- execution options ---- */

typedef enum {
    /* 1 (default): when a call repeats the previous call's geometry and
     * pointers on a non-default stream, replay the captured CUDA graph of its
     * launch sequence instead of launching each kernel; 0: plain launches. */
    BDIS_OPT_GRAPH = 1,
    /* 1: bracket every kernel launch with CUDA events on the call's stream
     * and accumulate per-kernel device time (graph replay is off while on). */
    BDIS_OPT_PROFILE = 2,
    /* 1 (default): on the first call of a geometry (pair count and sizes),
     * time the candidate launch configurations (search patches per block,
     * fusion tile size) level by level, each five times, and keep the fastest; the
     * call waits for the timing runs.  All configurations compute identical results.
     * 0: the default configuration.  Never tunes while the stream is being
     * captured. */
    BDIS_OPT_AUTOTUNE = 3,
    /* Execution form: 0 (default) as chosen by the autotuner, 1 one launch per
     * stage (the BDIS_OPT_COARSE_LEVELS coarsest levels excepted), 2
     * persistent (every stage in one cooperative launch with grid barriers;
     * 8-bit inputs, patch sizes 6, 8, 10, 12, 16).  The autotuner times the
     * launch sequence, each number of coarse levels in one cooperative
     * launch and the persistent form.  Same results in every form.
     * Every grid-barrier wait of the persistent form is bounded
     * (BDIS_OPT_BARRIER_LIMIT); a wait that runs out lets the kernel finish
     * with outputs that are not valid and is reported as BDIS_ECUDA by the
     * next call on the handle, by bdis_get_stats and by bdis_wait. */
    BDIS_OPT_FORM = 4,
    /* 1 (default): launch each kernel of the launch sequence with
     * programmatic stream serialisation, so that it is scheduled while its
     * predecessor drains and starts reading once the predecessor has
     * completed (hides the launch gap between dependent kernels); each block
     * of a kernel releases the next one at its end.  2: the same, but a
     * kernel whose grid fits in one wave of resident blocks releases the next
     * one at its start, and every kernel after a call's first prefetches its
     * descriptor while it waits.  0: plain stream order.  Same results. */
    BDIS_OPT_PDL = 5,
    /* Pyramid launches: 0 (default) two steps per launch (level l -> l+1 ->
     * l+2 with the gradients of l and l+1, recomputing a 2-pixel halo of level
     * l+1; a launch whose l+1 is the coarsest level ends with its gradient)
     * when the call has at most 2^21 level-0 pixels, else one step per launch;
     * 1 always one step; 2 always two steps while a coarser level remains.
     * Same results. */
    BDIS_OPT_PYRAMID_STEPS = 6,
    /* Extent of bdis_backward: 0 (default) the finest level, with the coarser
     * levels' state frozen (their propagated probability enters as a
     * constant); 1 through every level: the coarse levels reach the loss
     * through rho = Gamma_n pi + Q^(n+1)(centre) (Eq. 10), so their window
     * posteriors, sigma_r, patch solves, gradients and the pyramid are
     * differentiated too (FP32 pyramids only).  The coarse disparity maps
     * only initialise the finer searches and carry no gradient. */
    BDIS_OPT_ADJOINT_LEVELS = 7,
    /* bdis_match_host: 1 (default) when every buffer is page-locked host
     * memory the device can address (cudaMallocHost, cudaHostRegister), the
     * kernels read the inputs and write the outputs in place over the
     * host-device link; 0, or any other buffer: staging copies through device
     * memory.  Same results. */
    BDIS_OPT_HOST_MAPPED = 8,
    /* Polls of one grid-barrier wait of the persistent form, and of one wait
     * for bulk copies (BDIS_OPT_BULK_COPY), before it gives up (a poll is one
     * read and a short sleep): >= 1, default 2^22. */
    BDIS_OPT_BARRIER_LIMIT = 9,
    /* 1: test the timeout paths -- no arrival completes a grid barrier of the
     * persistent form, and every wait for bulk copies expects 16 bytes that
     * no copy delivers, so each wait runs out after BDIS_OPT_BARRIER_LIMIT
     * polls and the call is reported as failed (see BDIS_OPT_FORM).  0
     * (default): normal waits.  Only for tests of the error reporting. */
    BDIS_OPT_BARRIER_TEST = 10,
    /* With BDIS_OPT_FORM 1: the number k of coarsest searched levels whose
     * stages (their pyramid steps, searches and fusions) run as one
     * cooperative launch with grid barriers between the stages, the finer
     * levels as separate launches; 0 (default) none, at most
     * levels - finest_level - 1; patch sizes 6, 8, 10, 12, 16.  The coarse
     * levels' grids are small, so one launch replaces several short
     * dependent ones.  Same results. */
    BDIS_OPT_COARSE_LEVELS = 11,
    /* Bit flags, 0 (default, faster on GB300): every stage stages its
     * shared-memory tiles by the block's own loads.
     * Bit 1: the one-step pyramid launches (calls of more than 2^21 level-0
     * pixels, or BDIS_OPT_PYRAMID_STEPS 1) stage each interior tile by bulk
     * asynchronous copies (cp.async.bulk, one per row, completing on an
     * mbarrier), the next tile's copies in flight while the current one is
     * computed.
     * Bit 2: the search launches (patch sizes 8 and 12; others ignore the
     * bit) copy the right-image band of each block whose band window lies
     * inside the image by one cp.async.bulk per patch row, issued before
     * the left-image and gradient bands are loaded, then widen it to FP32
     * in shared memory.
     * Same results in every case.  The wait for a block's copies is
     * bounded; one that runs out is reported like a grid-barrier timeout
     * (BDIS_OPT_FORM).  Values outside 0..3: BDIS_EINVAL. */
    BDIS_OPT_BULK_COPY = 12,
    /* Search chunk of every level: 0 (default) as tuned (or the default
     * configuration with BDIS_OPT_AUTOTUNE 0); 1..4 that many passes of the
     * block's lane groups per chunk (32 patches per pass for patch sizes up
     * to 8, 16 above).  Same results: the sigma_r sums are exact integers, so
     * the chunking does not change them.  Other values: BDIS_EINVAL. */
    BDIS_OPT_SEARCH_PASSES = 13,
    /* Fusion tile of every level: 0 (default) as tuned (or the default
     * configuration with BDIS_OPT_AUTOTUNE 0); 1 32x16, 2 64x32, 3 64x64
     * pixels.  Same results: each pixel's sums run over its covering
     * patches in the same order whatever the tile.  Other values:
     * BDIS_EINVAL. */
    BDIS_OPT_FUSE_TILE = 14
} bdis_option;

bdis_status bdis_set_option(bdis_handle *h, int option, int value);

/* kernels: pyramid + gradient; patch search; fused sigma_r + posterior + densify;
 * the persistent form (all stages in one launch); full-resolution upsampling
 * of the finest processed level (finest_level > 0) */
enum { BDIS_K_PYRAMID = 0, BDIS_K_SEARCH = 1, BDIS_K_FUSE = 2, BDIS_K_PERSISTENT = 3,
       BDIS_K_UPSAMPLE = 4, BDIS_K_COUNT = 5 };

typedef struct {
    int launches[BDIS_K_COUNT];   /* launches per kernel since the last reset */
    double ms[BDIS_K_COUNT];      /* summed CUDA-event time per kernel (ms)   */
    int launches_level[BDIS_K_COUNT][8];  /* the same per pyramid level of the  */
    double ms_level[BDIS_K_COUNT][8];     /* launch (a pyramid launch counts at
                                             the level it reads; a persistent
                                             launch at its first stage's level) */
} bdis_profile;

/* Per-kernel launch counts and event times accumulated while
 * BDIS_OPT_PROFILE is on (waits for the recorded events); reset != 0 clears. */
bdis_status bdis_get_profile(bdis_handle *h, bdis_profile *out, int reset);

/* ---- inspection of the last call's intermediate buffers (diagnostics; the parity tests read every level through it) ---- */

/* Per-patch record, as written by the search and posterior stages. */
typedef struct {
    float d, dinit, dlast, H;      /* estimate, initial value, last GN step, Hessian */
    float E[5];                    /* E[0] = E(0); E[k] = E(delta_k) - E(0) for the
                                      window offsets delta = {-h, +h, -2h, +2h}        */
    float cT;                      /* sum of centred gradient x template             */
    uint32_t flags;                /* rejection bits (0 = kept), see BDIS_F_*         */
    uint16_t nout;                 /* samples outside the image at the estimate      */
    uint16_t pdf_flags;            /* PDF-fit exception bits, see BDIS_PDF_*          */
    float pi, rho, sig2;           /* window posterior, propagated probability, var  */
    float mu;                      /* patch mean of I_r(x - d) - I_l(x) at the
                                      estimate (the mean offset the normalised
                                      residual removes)                          */
} bdis_patch_record;

enum {
    BDIS_F_FLAT = 1u << 0, BDIS_F_UNCONVERGED = 1u << 1, BDIS_F_MOVED = 1u << 2,
    BDIS_F_OUTSIDE = 1u << 3, BDIS_F_SADDLE = 1u << 4, BDIS_F_NONFINITE = 1u << 5
};
enum { BDIS_PDF_NOT_PEAK = 1u << 0, BDIS_PDF_FAILED = 1u << 1, BDIS_PDF_RESIDUAL = 1u << 2 };

typedef struct {
    int w, h;                 /* level size                                    */
    int npx, npy;             /* patch grid                                    */
    int image_pitch;          /* elements per row of left/right                */
    int grad_pitch;           /* elements per row of grad                      */
    int storage;              /* element type of left/right/grad (level 0: u8) */
    const void *left, *right, *grad;   /* device pointers (level 0: caller's)  */
    const bdis_patch_record *records;  /* npx*npy records, row-major           */
    const float *D, *Q;       /* fused maps (w*h), NULL at level 0; at the
                                 finest processed level f > 0, D is NaN where
                                 the level-f pixel is invalid                 */
    const float *sigma_r;     /* one float                                     */
} bdis_level_view;

/* Device pointers into the handle's arena for (pair, level) of the last call.
 * Valid until the next call on the handle. */
bdis_status bdis_level_view_get(const bdis_handle *h, int pair, int level,
                                bdis_level_view *out);

/* Companion of bdis_level_view_get for callers without a CUDA runtime of
 * their own (the Python binding): copies `bytes` between any two addresses
 * the device can reach (host, page-locked or device; e.g. a level view's
 * device pointers into a host buffer the caller owns) with
 * cudaMemcpyAsync(..., cudaMemcpyDefault) on `stream` (NULL: the legacy
 * default stream) and waits for it.  Nothing is allocated or kept.
 * BDIS_EINVAL for a null pointer with bytes > 0; BDIS_ECUDA if the copy
 * fails (bad address, or an error of an earlier asynchronous call). */
bdis_status bdis_copy(void *dst, const void *src, size_t bytes, void *stream);

/* ---- depth (Eq. 13) and depth variance (Eq. 17) ---- */

/* Elementwise on n pixels of device buffers, asynchronous on `stream`:
 *   depth = fb / disp,   depth_var = fb^2 / disp^4 * var,
 * fb = focal length (px) x baseline (any length unit; depth comes out in
 * that unit).  A pixel whose disp is not a positive finite number (NaN,
 * <= 0 or infinite) gets NaN in both.  `var`
 * and `depth_var` may be NULL (then no variance is written); n == 0 is a
 * no-op.  BDIS_EINVAL for a null disp / depth with n > 0, n < 0, or a
 * non-finite or non-positive fb. */
bdis_status bdis_depth(const float *disp, const float *var, long long n, float fb, float *depth,
                       float *depth_var, void *stream);

/* ---- measurement ----
 * L2 read-bandwidth probe (the paper has no counterpart: it gives the
 * denominator of the L2 roofline fractions the benchmark reports).  Reads
 * the device buffer `buf` (16-byte aligned, `bytes` >= 16; make it small
 * enough to stay in L2, e.g. 48 MiB of the 129 MB) `reps` times in one
 * launch with 16-byte loads that bypass L1, writing nothing; asynchronous on
 * `stream` (time it with events: bytes x reps / elapsed).  BDIS_EINVAL for a
 * null or unaligned buffer, bytes < 16 or reps < 1. */
bdis_status bdis_probe_l2_read(const void *buf, size_t bytes, int reps, void *stream);


#ifdef __cplusplus
}
#endif
#endif /* BDIS_H */
