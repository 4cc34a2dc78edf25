// bdis_noalloc.cu -- bdis_match_noalloc: the full single-pair pipeline for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a video pipeline that hands all
// device memory to its own pool at start-up, a process that runs under a
// fixed device-memory budget, or a latency-critical loop that cannot afford
// the device-wide synchronisation cudaMalloc / cudaFree imply.  bdis_match
// allocates its scratch arena (and pinned staging) on first use; this entry
// point allocates nothing.  Its scratch -- pyramids, gradients, patch
// records, coarse maps and the descriptor table -- lives in one file-scope
// device array of kNoAllocScratchBytes, which every GPU that loads the
// library holds until the process exits.  The caller still provides the
// input and output buffers.
//
// The array name is a host-side stand-in in host code, not a device address:
// handing it to a kernel would fault or, where the GPU can reach host memory,
// silently use the wrong memory.  The device address is therefore resolved
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.  The first call on each device does this set-up.
//
// Every call shares the one array and it keeps the previous call's contents.
// Only the sigma_r accumulators must start at zero; each call's first kernel
// clears them.  Every other element is written before it is read.  Calls that overlap on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "bdis_internal.cuh"

namespace bdis {
namespace {

// Largest scratch this entry point can use: enough for one 1280x720 pair
// with 8x8 patches, stride 4, 3 levels and FP32 pyramids (about 15 MiB), or
// one 640x480 pair with any supported settings.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DescTable {
    LevelDesc d[kMaxLevels];
    int n;
};

// Writes the descriptor table into the scratch array (the table travels as a
// kernel parameter, so no host-to-device copy is needed).
__global__ void k_noalloc_write_descs(DescTable t, LevelDesc *dst) {
    const int i = threadIdx.x;
    if (i < t.n) dst[i] = t.d[i];
}

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

int na_level_dim(int n, int l) {
    for (int i = 0; i < l; ++i) n = (n + 1) / 2;
    return n;
}

size_t na_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Resolves (once per device) the device address of the scratch array.
bdis_status na_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BDIS_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) return BDIS_ECUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return BDIS_OK;
}

}  // namespace
}  // namespace bdis

using namespace bdis;

extern "C" bdis_status bdis_match_noalloc(const bdis_params *pp, const uint8_t *left,
                                          const uint8_t *right, int w, int hgt, int pitch,
                                          float *disp, float *var, uint8_t *valid,
                                          void *stream) {
    if (!pp || !left || !right || !disp || !valid) return BDIS_EINVAL;
    const bdis_params p = *pp;
    // the same parameter and size checks as every other entry point
    if (!check_params(p).empty()) return BDIS_EINVAL;
    const bdis_pair q{left, right, w, hgt, pitch, disp, var, valid};
    if (!check_pair(p, q).empty()) return BDIS_EINVAL;
    const int NL = p.levels, P = p.patch, S = p.stride;
    // full resolution and FP32 / FP16 pyramids only (the upsampled form and
    // 8-bit pyramids need bdis_match)
    if (p.finest_level != 0 || p.storage == BDIS_STORE_U8) return BDIS_EUNSUPPORTED;

    // ---- layout inside the scratch array (no heap use)
    DescTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = NL;
    const size_t esz = p.storage == BDIS_STORE_F16 ? 2 : 4;
    const LevelCfg cfg{2, 32, 16};  // default launch configuration (no tuning here)
    const int chunk = search_chunk(P, cfg.passes);
    size_t off = na_align(sizeof(LevelDesc) * kMaxLevels, 256);
    const size_t off_acc = off;  // sigma_r accumulators: 3 per level, cleared by the pyramid
    off += sizeof(unsigned long long) * 3 * kMaxLevels;
    size_t oG[kMaxLevels], oL[kMaxLevels], oR[kMaxLevels], oD[kMaxLevels], oQ[kMaxLevels];
    size_t oRec[kMaxLevels], oFuse[kMaxLevels], oSr[kMaxLevels];
    int units[kMaxLevels][W_COUNT];
    auto take = [&](size_t n) {
        off = na_align(off, 256);
        const size_t r = off;
        off += n;
        return r;
    };
    for (int l = 0; l < NL; ++l) {
        LevelDesc &d = tab.d[l];
        d.w = na_level_dim(w, l);
        d.h = na_level_dim(hgt, l);
        d.kxreg = (d.w - P) / S + 1;
        d.kyreg = (d.h - P) / S + 1;
        d.npx = d.kxreg + ((d.w - P) % S != 0 ? 1 : 0);
        d.npy = d.kyreg + ((d.h - P) % S != 0 ? 1 : 0);
        d.nchunks = (d.npx + chunk - 1) / chunk;
        d.tiles_x = (d.w + cfg.tile_w - 1) / cfg.tile_w;
        units[l][W_PYR] = ((d.w + 63) / 64) * ((d.h + 31) / 32);
        units[l][W_SEARCH] = d.npy * d.nchunks;
        units[l][W_FUSE] = d.tiles_x * ((d.h + cfg.tile_h - 1) / cfg.tile_h);
        const size_t gp = na_align((size_t)d.w * esz, 128) / esz;
        d.gpitch = (int)gp;
        d.pitch = l == 0 ? pitch : (int)gp;
        oG[l] = take(gp * esz * d.h);
        if (l > 0) {
            oL[l] = take(gp * esz * d.h);
            oR[l] = take(gp * esz * d.h);
            oD[l] = take(sizeof(float) * (size_t)d.w * d.h);
            oQ[l] = take(sizeof(float) * (size_t)d.w * d.h);
        }
        const size_t np = (size_t)d.npx * d.npy;
        oRec[l] = take(sizeof(bdis_patch_record) * np);
        oFuse[l] = take(sizeof(float4) * np);
        oSr[l] = take(sizeof(float));
    }
    if (off > kNoAllocScratchBytes) return BDIS_EUNSUPPORTED;  // needs more than the static maximum

    // shared memory of the search and fuse blocks
    const float tau = p.search_radius > 0.f ? p.search_radius : (float)P;
    int band_pitch, band_cap, chunk_pitch;
    size_t smem;
    search_layout(P, S, tau, p.window_step, cfg.passes, band_pitch, band_cap, chunk_pitch, smem);
    const size_t fsmem = fuse_smem(P, S, cfg.tile_w, cfg.tile_h);
    int optin = 0, dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BDIS_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return BDIS_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    // the search band and the fuse tile must fit the device's per-block limit
    if (smem > (size_t)optin || fsmem > (size_t)optin) return BDIS_EUNSUPPORTED;

    void *scratch = nullptr;
    const bdis_status ss = na_scratch(&scratch);
    if (ss != BDIS_OK) return ss;
    char *base = (char *)scratch;
    LevelDesc *d_descs = (LevelDesc *)base;

    for (int l = 0; l < NL; ++l) {
        LevelDesc &d = tab.d[l];
        d.G = base + oG[l];
        if (l == 0) {
            d.L = left;
            d.R = right;
            d.disp = disp;
            d.var = var;
            d.valid = valid;
        } else {
            d.L = base + oL[l];
            d.R = base + oR[l];
            d.D = (float *)(base + oD[l]);
            d.Q = (float *)(base + oQ[l]);
        }
        d.rec = (bdis_patch_record *)(base + oRec[l]);
        d.fuse = (float4 *)(base + oFuse[l]);
        d.sigma_r = (float *)(base + oSr[l]);
        d.acc = (unsigned long long *)(base + off_acc) + 3 * l;
    }
    for (int l = 0; l + 1 < NL; ++l) {
        LevelDesc &d = tab.d[l];
        const LevelDesc &c = tab.d[l + 1];
        d.Ln = (void *)c.L;
        d.Rn = (void *)c.R;
        d.wn = d.wc = c.w;
        d.hn = d.hc = c.h;
        d.pitchn = c.pitch;
        d.Dc = c.D;
        d.Qc = c.Q;
    }

    // ---- launches (the same kernels as bdis_match)
    cudaStream_t st = (cudaStream_t)stream;
    // the kernels' shared-memory limits are only ever raised, never lowered
    if (prepare_search(P, smem) != cudaSuccess) return BDIS_ECUDA;
    if (prepare_fuse(fsmem) != cudaSuccess) return BDIS_ECUDA;
    k_noalloc_write_descs<<<1, 32, 0, st>>>(tab, d_descs);
    if (cudaGetLastError() != cudaSuccess) return BDIS_ECUDA;

    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.npairs = 1;
    a.levels = NL;
    a.P = P;
    a.S = S;
    a.iters = p.iters;
    a.window_step = p.window_step;
    a.conv_eps = p.conv_eps;
    a.valid_gamma = p.valid_gamma;
    a.pix_thresh = p.pix_thresh;
    a.tau = a.tau0 = p.search_radius > 0.f ? p.search_radius : (float)P;
    a.hess_eps = p.hess_eps;
    a.sigma_r_mode = p.sigma_r_mode;
    a.sigma_r_floor = p.sigma_r_floor;
    a.sigma_r_fixed = p.sigma_r_fixed;
    a.variance = p.variance;
    a.pdf_iters = p.pdf_iters;
    a.pdf_resid = p.pdf_resid;
    a.use_c2f = p.use_c2f;
    a.use_sgmm = p.use_sgmm;
    a.weight_mode = p.weight_mode;
    a.fast_exp = p.fast_exp;
    a.finest = 0;
    a.pdl = 1;  // each launch may start while its predecessor drains
    a.chunk = chunk;
    a.tile_w = cfg.tile_w;
    a.tile_h = cfg.tile_h;
    for (int i = 0; i < kMaxPatch; ++i) {  // 1D sGMM factor of Eq. 8
        double s = 0.0;
        if (i < P)
            for (int j = 0; j < P; ++j)
                s += std::exp(-(double)(i - j) * (i - j) / (2.0 * p.sigma_s * p.sigma_s));
        a.m[i] = (float)s;
    }
    double gsum = 0.0;
    for (int l = 0; l < NL; ++l) gsum += std::ldexp(1.0, l);
    const int st_type = p.storage == BDIS_STORE_F16 ? E_F16 : E_F32;
    for (int l = 0; l < NL; ++l) {
        a.descs = d_descs + l;
        a.level = l;
        a.total = units[l][W_PYR];
        a.acc_zero = l == 0 ? (unsigned long long *)(base + off_acc) : nullptr;
        a.acc_count = l == 0 ? 3 * kMaxLevels : 0;
        if (launch_pyramid(a, l == 0 ? E_U8 : st_type, st_type, st_type, st) != cudaSuccess)
            return BDIS_ECUDA;
    }
    for (int l = NL - 1; l >= 0; --l) {
        a.descs = d_descs + l;
        a.level = l;
        a.gamma_w = (float)(std::ldexp(1.0, l) / gsum);
        a.band_pitch = band_pitch;
        a.band_cap = band_cap;
        a.chunk_pitch = chunk_pitch;
        a.total = units[l][W_SEARCH];
        const int itype = l == 0 ? E_U8 : st_type;
        a.img_type = itype;
        int occ = search_occupancy(P, itype, st_type, smem);
        if (occ < 1) occ = 1;
        const int grid = a.total < sms * occ ? a.total : sms * occ;
        if (launch_search(a, itype, st_type, smem, grid > 0 ? grid : 1, st) != cudaSuccess)
            return BDIS_ECUDA;
        a.total = units[l][W_FUSE];
        if (launch_fuse(a, fsmem, st) != cudaSuccess) return BDIS_ECUDA;
    }
    return BDIS_OK;
}
