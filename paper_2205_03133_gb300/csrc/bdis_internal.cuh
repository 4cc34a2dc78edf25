// bdis_internal.cuh -- device-side descriptors shared by the kernels and the
// host library of libbdis.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "bdis.h"

namespace bdis {

constexpr int kMaxLevels = 8;
constexpr int kMinPatch = 4;
constexpr int kMaxPatch = 16;
constexpr int kWindow = 5;  // samples of the small window P' (Sec. III-B, s = 5)

// Work spaces of the per-level kernels.  Each (pair, level) owns the
// half-open unit range [work_begin[k], work_begin[k] + units) of kernel k.
enum WorkKind { W_PYR = 0, W_SEARCH = 1, W_FUSE = 2, W_UP = 3, W_COUNT = 4 };
// Pixels per unit of the full-resolution upsampling (256 threads x 4).
constexpr int kUpUnitPixels = 1024;

// Largest pixel tile of the fused posterior / densify kernel.
constexpr int kFuseTileWMax = 64;
constexpr int kFuseTileHMax = 64;

// Launch configuration of one level (chosen by the autotuner): search passes
// per block (a block's chunk is passes x groups patches) and fuse tile size.
struct LevelCfg {
    int passes;
    int tile_w, tile_h;
};
// Extra columns of the search's right band for the spread of the initial
// estimates inside one chunk (wider spreads read the image directly).
constexpr int kBandSpread = 64;
// Fixed-point scale of the sigma_r sum of E(0) (E(0) <= 255^2 * 256 per patch).
constexpr float kSigmaFix1 = 65536.f;

// Element types of the level images.
enum ElemType { E_U8 = 0, E_F32 = 1, E_F16 = 2 };

// Element type of the stored pyramid levels 1..L-1 and of the gradients.
inline int image_type_of(int storage) {
    return storage == BDIS_STORE_F16 ? E_F16 : storage == BDIS_STORE_U8 ? E_U8 : E_F32;
}
inline int grad_type_of(int storage) { return storage == BDIS_STORE_F32 ? E_F32 : E_F16; }
inline size_t elem_size(int type) { return type == E_U8 ? 1 : type == E_F16 ? 2 : 4; }

// One (pair, level).  All pointers are device pointers.
struct alignas(16) LevelDesc {
    const void *L, *R;        // level images (level 0: caller's 8-bit images)
    void *G;                  // x-gradient of L at this level (storage type)
    void *Ln, *Rn;            // next coarser level to build (nullptr at the coarsest)
    float *D, *Q;             // fused disparity / probability maps (levels >= 1)
    const float *Dc, *Qc;     // coarser fused maps (nullptr at the coarsest level)
    float *disp, *var;        // level-0 outputs (var may be nullptr); at the finest
                              // processed level f > 0, var is its V map
    uint8_t *valid;
    const float *Df, *Vf;     // level 0 with f > 0: the level-f maps to upsample
    int wf, hf;               // their size
    float *wsum;              // float-image forward: sum of the fusion weights per
                              // pixel of every level (read by the adjoint), else nullptr
    bdis_patch_record *rec;   // npx * npy records of this pair at this level
    float4 *fuse;             // (d, rho, sig2, mu) per patch for the fusion gather (rho = 0: rejected)
    float *sigma_r;           // one float
    unsigned long long *acc;  // sigma_r sums of kept patches: E(0) * 2^16, count, E(0)^2
    int w, h, pitch;          // level size, row pitch (elements) of L and R
    int gpitch;               // row pitch (elements) of G
    int wn, hn, pitchn;       // next coarser level size and pitch
    int wc, hc;               // coarser map size (levels < L-1)
    int npx, npy, kxreg, kyreg;
    int nchunks;              // search chunks per patch row
    int tiles_x;              // fuse tiles per row
    int work_begin[W_COUNT];
};

// Per-launch arguments (passed by value).
struct LaunchArgs {
    const LevelDesc *descs;   // the npairs descriptors of this level
    const LevelDesc *descs2;  // two-step pyramid stage: the descriptors of the next level
    int npairs;
    int total;                // total work units of this launch
    int level, levels;
    int P, S, iters;
    float window_step, conv_eps, valid_gamma, pix_thresh;
    float tau;                // search radius at this level (px)
    float tau0;               // search radius at level 0 (PDF exception value)
    float hess_eps;
    float gamma_w;            // Gamma weight of this level (Eq. 11)
    int sigma_r_mode;
    float sigma_r_floor, sigma_r_fixed;
    int variance, pdf_iters;
    float pdf_resid;
    int use_c2f, use_sgmm;
    int chunk;                // patches per search chunk
    int tile_w, tile_h;       // fuse tile
    int band_pitch;           // floats per row of the staged right band
    int band_cap;             // usable columns of the right band
    int chunk_pitch;          // floats per row of the staged left / gradient band
    float m[kMaxPatch];       // 1D sGMM factors m[a] (Eq. 8 is separable)
    unsigned long long *acc_zero;  // finest pyramid launch: accumulators to clear
    int acc_count;
    int kind;                 // stage of the persistent form: 0 pyramid, 1 search, 2 fuse,
                              // 3 upsample, 4 two-step pyramid
    int finest;               // finest processed level f
    int weight_mode;          // bdis_weight_mode
    int fast_exp;             // Schraudolph exponential in the posterior
    int img_type;             // ElemType of this level's L, R (read by the DIS fusion)
    int pdl;                  // programmatic stream serialisation: 0 off, 1 the next kernel
                              // released at block end, 2 released at kernel start when
                              // the grid fits in one wave of resident blocks
    int early;                // set by the launcher: release the next kernel at the start
    int prefetch;             // the descriptor table is complete before this kernel starts
                              // (every stage after a call's first): prefetched while waiting
    int bulk;                 // bit 1: one-step pyramid tiles, bit 2: search bands, by bulk async copies
    int *err_host;            // mapped status word of the handle (a device wait ran out), or nullptr
    unsigned copy_limit;      // polls of a bulk-copy wait before it gives up (0: the default)
    int copy_test;            // test switch: each bulk-copy wait expects 16 bytes that no copy
                              // delivers, so it runs out (BDIS_OPT_BARRIER_TEST)
};

// Persistent form: every stage of a call in one cooperative launch, with a
// grid barrier between dependent stages.
struct MegaArgs {
    const LaunchArgs *stages;  // device array of nstages stage arguments
    int nstages;
    unsigned *bar;             // [0] arrivals, [1] generation (cleared before each launch)
    int *err;                  // set to 1 when a barrier wait runs out (cleared before each launch)
    int *err_host;             // mapped page-locked word of the handle: also set to 1 (sticky)
    unsigned spin_limit;       // polls of one barrier wait before it gives up
    int unreachable;           // test: no arrival completes a barrier, so every wait runs out
};

// Default poll limit of one grid-barrier wait (a poll is one L2 read and a
// 64 ns sleep); a wait that runs out sets MegaArgs::err and lets the block
// continue, so the kernel always ends.
constexpr unsigned kBarrierSpinLimit = 1u << 22;

// ---- differentiable finest level (bdis_grad.cu)

// G_PIX: 256 pixels per unit; G_GROUP: one lane group per patch, 256 / group
// patches per unit (the fusion and patch adjoints)
enum GradWork { G_PIX = 0, G_GROUP = 1, G_COUNT = 2 };

// One (pair, level) of the backward pass.  Images are the float images of the
// forward at that level; gradients are dense w*h arrays of the level.
struct alignas(16) GradDesc {
    const float *L, *R;            // level-0 images, `pitch` elements per row
    const void *G;                 // level-0 x-gradient (storage type)
    const float *disp;             // forward disparity (valid pixels)
    const float *wsum;             // forward fusion-weight sums per pixel
    const uint8_t *valid;
    const bdis_patch_record *rec;  // level-0 records
    const float4 *fuse;            // level-0 fusion records
    const float *sigma_r;
    float *gDisp, *gL, *gR, *gPatch, *loss;        // caller buffers
    float *gDw, *gG, *gd, *gpi, *sig_part, *coefE0, *loss_part;  // scratch
    float *cpatch;                 // per patch: P x P template and gradient-image terms
    // levels >= 1 (the adjoint through every level)
    const float *Q;                // the level's fused probability map (forward)
    float *gQ;                     // dL/dQ of this level (zeroed, accumulated by level - 1)
    float *gQn;                    // dL/dQ of the next coarser level, or nullptr
    const float *gLc, *gRc;        // image gradients of the next coarser level, or nullptr
    int wn, hn;                    // next coarser level size
    int w, h, pitch, gpitch, gtype;
    int npx, npy, kxreg, kyreg;
    int work_begin[G_COUNT];
};

struct GradArgs {
    const GradDesc *descs;         // the npairs descriptors of this level
    int npairs, total;
    int level;
    int P, S;
    float window_step, lambda, gamma_w;
    int sigma_r_mode;
    float sigma_r_floor;
    int use_sgmm, use_c2f;
    float m[kMaxPatch];
};

// Argument checks shared by every entry point (bdis_api.cu): an empty string
// when valid, else the reason.
std::string check_params(const bdis_params &p);
std::string check_pair(const bdis_params &p, const bdis_pair &q);

cudaError_t launch_loss(const GradArgs &a, cudaStream_t s);        // zeroes dL/dI_r; + per-pair reduce
cudaError_t launch_bwd_pix(const GradArgs &a, cudaStream_t s);
cudaError_t launch_bwd_dens(const GradArgs &a, cudaStream_t s);    // + sigma_r adjoint
cudaError_t launch_bwd_patch(const GradArgs &a, cudaStream_t s);
cudaError_t launch_bwd_gather(const GradArgs &a, cudaStream_t s);
cudaError_t launch_bwd_sobel(const GradArgs &a, cudaStream_t s);
cudaError_t launch_bwd_pyr(const GradArgs &a, cudaStream_t s);   // pyramid transpose into this level

// Kernel launchers (bdis_kernels.cu).  Each returns cudaGetLastError().
// in_type: the images the launch reads; img_type: the next levels it
// writes; g_type: the gradients it writes.
cudaError_t launch_pyramid(const LaunchArgs &a, int in_type, int img_type, int g_type, cudaStream_t s);
// Two pyramid steps (level l -> l+1 -> l+2, with both gradients) per launch.
cudaError_t launch_pyramid2(const LaunchArgs &a, int in_type, int img_type, int g_type, cudaStream_t s);
cudaError_t launch_search(const LaunchArgs &a, int in_type, int g_type, size_t smem, int grid,
                          cudaStream_t s);
cudaError_t launch_fuse(const LaunchArgs &a, size_t smem, cudaStream_t s);
cudaError_t launch_upsample(const LaunchArgs &a, cudaStream_t s);
cudaError_t launch_depth(const float *disp, const float *var, long long n, float fb, float *depth,
                         float *depth_var, cudaStream_t s);
// Shared-memory layout of the search (band pitch and capacity, chunk pitch, bytes).
// bulk: with the raw area of the right band's bulk staging (BDIS_OPT_BULK_COPY bit 2)
void search_layout(int P, int S, float tau, float window_step, int passes, int &band_pitch,
                   int &band_cap, int &chunk_pitch, size_t &bytes, bool bulk = false);
size_t fuse_smem(int P, int S, int tile_w, int tile_h);
cudaError_t prepare_fuse(size_t smem_bytes);
// Persistent form: available for the patch sizes with an instance; grid =
// co-resident blocks (0 if unavailable).
bool mega_supported(int P);
int mega_grid(int P, int st_type, size_t smem);
// pdl: also allow programmatic stream serialisation (the kernel waits in
// pdl_wait() before touching memory)
cudaError_t launch_mega(const MegaArgs &m, int P, int st_type, int grid, size_t smem, bool pdl,
                        cudaStream_t s);
constexpr size_t kPyrSmemBytes = sizeof(float) * (2 * 36 * 76 + 2 * 36 * 36);
constexpr size_t kPyr2SmemBytes = sizeof(float) * (2 * 44 * 76 + 2 * 20 * 36 + 2 * 44 * 36);
// Raise (never lower) the dynamic shared-memory limit of every search instance.
cudaError_t prepare_search(int P, size_t smem_bytes);
// Number of resident search blocks per SM for (P, image type, gradient type, smem).
int search_occupancy(int P, int in_type, int g_type, size_t smem_bytes, bool bulk = false);
bool search_supported(int P);
int search_group(int P);      // lanes per patch
int search_chunk(int P, int passes);  // patches per chunk

}  // namespace bdis
