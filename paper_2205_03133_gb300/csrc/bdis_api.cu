// bdis_api.cu -- host side of libbdis: argument checks, the per-call plan
// (level geometry, arena layout, per-level descriptor tables), the device
// scratch arena and the coarse-to-fine launch sequence (Fig. 1 of
// arXiv 2205.03133: coarsest level first; each level's fused map seeds the
// next finer level).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "bdis_internal.cuh"

using namespace bdis;

// State of one differentiable forward kept by the caller (bdis_saved_create):
// the forward ran with this object's device arena in place of the handle's,
// so the pyramids, gradients, patch and fusion records, weight sums and
// sigma_r it produced stay here until the object is reused or destroyed.
struct bdis_saved {
    bdis_handle *owner = nullptr;
    char *arena = nullptr;
    size_t arena_cap = 0;
    std::vector<LevelDesc> descs;  // [level][pair] of that forward
    int npairs = 0, levels = 0, in_type = -1;
};

struct bdis_handle {
    bdis_params p{};
    std::string err = "no error";
    // device scratch arena (grows, never shrinks)
    char *arena = nullptr;
    size_t arena_cap = 0;
    // pinned staging for the descriptor upload
    char *pinned = nullptr;
    size_t pinned_cap = 0;
    cudaEvent_t upload_done = nullptr;
    std::vector<char> last_upload;
    // the last call's layout (for views and stats)
    std::vector<LevelDesc> descs;  // [level][pair]
    int npairs = 0;
    int levels = 0;
    int in_type = E_U8;
    LevelDesc *d_descs = nullptr;
    size_t smem_prepared = 0;
    int prepared_P = 0;
    // CUDA graph of the last launch sequence and the descriptors it bakes in
    bool use_graph = true;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<char> graph_descs;
    // scratch of the backward pass (grows, never shrinks)
    char *garena = nullptr;
    size_t garena_cap = 0;
    // the gradient-descriptor table the backward scratch holds (its bytes,
    // uploaded at the start of garena); a call whose table is these bytes or
    // a prefix of them skips the upload and the wait for the staging buffer
    std::vector<char> last_grad_upload;
    // autotuner: per-level launch configuration cached per geometry key
    bool autotune = true;
    // execution form of a call: kFormLaunches, kFormPersistent, or k > 0:
    // the k coarsest searched levels (with their pyramid steps) in one
    // cooperative launch, the finer levels as separate launches
    struct Tuned {
        std::vector<LevelCfg> cfg;
        int form;
    };
    std::map<std::string, Tuned> tuned;
    int *err_flag = nullptr;  // timeout flag of the last cooperative launch (device)
    int last_persistent = 0;  // bdis_stats::persistent of the last call
    int coarse_levels = 0;    // BDIS_OPT_COARSE_LEVELS
    int bulk_copy = 0;        // BDIS_OPT_BULK_COPY (bit 1 pyramid, bit 2 search band)
    unsigned barrier_limit = kBarrierSpinLimit;  // BDIS_OPT_BARRIER_LIMIT
    bool barrier_unreachable = false;            // BDIS_OPT_BARRIER_TEST
    // sticky timeout word in mapped page-locked host memory: a persistent
    // launch whose barrier wait ran out stores 1 there; the next call on the
    // handle takes it (atomic exchange with 0) and fails
    int *status_host = nullptr;
    int *status_dev = nullptr;  // the device's address of the same word
    // caller-owned forward states created on this handle, and the one whose
    // arena the last call's descriptors point into (nullptr: the handle's own)
    std::vector<bdis_saved *> saved;
    bdis_saved *last_saved = nullptr;
    int form = 0;             // BDIS_OPT_FORM
    int use_pdl = 1;          // BDIS_OPT_PDL: 0, 1 or 2
    int pyr_steps = 0;        // BDIS_OPT_PYRAMID_STEPS
    int search_passes = 0;    // BDIS_OPT_SEARCH_PASSES (0: tuned)
    int fuse_tile = 0;        // BDIS_OPT_FUSE_TILE (0: tuned)
    bool adjoint_levels = false;  // BDIS_OPT_ADJOINT_LEVELS
    bool host_mapped = true;      // BDIS_OPT_HOST_MAPPED
    // repeat of the previous call: same pairs, stream, options and arena ->
    // the captured graph is replayed without rebuilding the plan
    struct Repeat {
        std::vector<bdis_pair> pairs;
        int in_type = -1;
        cudaStream_t st = nullptr;
        char *arena = nullptr;
        size_t arena_cap = 0;
        int opts = -1;
    } repeat;
    bool repeat_ok = false;
    // per-kernel event timing
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_marks;  // (kernel id + 16 level, index of start event)
    int prof_launches[BDIS_K_COUNT] = {0};
    double prof_ms[BDIS_K_COUNT] = {0};
    int prof_launches_level[BDIS_K_COUNT][kMaxLevels] = {{0}};
    double prof_ms_level[BDIS_K_COUNT][kMaxLevels] = {{0}};
};

namespace {

const char *kStatusText[] = {"ok", "invalid argument", "out of memory", "CUDA error",
                             "unsupported"};

bdis_status fail(bdis_handle *h, bdis_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

bdis_status cuda_fail(bdis_handle *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, BDIS_ECUDA, m);
}

int level_dim(int n, int l) {
    for (int i = 0; i < l; ++i) n = (n + 1) / 2;
    return n;
}

int num_origins(int n, int P, int S, int *kreg) {
    const int r = (n - P) / S + 1;
    if (kreg) *kreg = r;
    return r + ((n - P) % S != 0 ? 1 : 0);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool finite_nonneg(float v) { return std::isfinite(v) && v >= 0.f; }

}  // namespace

namespace bdis {

std::string check_params(const bdis_params &p) {
    if (p.patch < kMinPatch || p.patch > kMaxPatch) return "patch must be in [4, 16]";
    if (p.stride < 1 || p.stride > p.patch) return "stride must be in [1, patch]";
    if (p.levels < 1 || p.levels > kMaxLevels) return "levels must be in [1, 8]";
    if (p.iters < 0 || p.iters > 1000) return "iters must be in [0, 1000]";
    if (!(std::isfinite(p.sigma_s) && p.sigma_s > 0.f)) return "sigma_s must be > 0";
    if (!(std::isfinite(p.window_step) && p.window_step > 0.f)) return "window_step must be > 0";
    if (!finite_nonneg(p.conv_eps)) return "conv_eps must be >= 0";
    if (!(finite_nonneg(p.valid_gamma) && p.valid_gamma <= 1.f)) return "valid_gamma must be in [0, 1]";
    if (!finite_nonneg(p.pix_thresh)) return "pix_thresh must be >= 0";
    if (!std::isfinite(p.search_radius)) return "search_radius must be finite";
    if (p.sigma_r_mode < 0 || p.sigma_r_mode > 2) return "bad sigma_r_mode";
    if (!finite_nonneg(p.sigma_r_floor)) return "sigma_r_floor must be >= 0";
    if (!(std::isfinite(p.sigma_r_fixed) && p.sigma_r_fixed > 0.f)) return "sigma_r_fixed must be > 0";
    if (p.sigma_r_mode != BDIS_SIGMA_R_FIXED && !(p.sigma_r_floor > 0.f))
        return "sigma_r_floor must be > 0 for the dynamic modes";
    if (p.variance != 0 && p.variance != 1) return "variance must be 0 or 1";
    if (p.pdf_iters < 0 || p.pdf_iters > 100) return "pdf_iters must be in [0, 100]";
    if (!finite_nonneg(p.pdf_resid)) return "pdf_resid must be >= 0";
    if (p.storage != BDIS_STORE_F32 && p.storage != BDIS_STORE_F16 && p.storage != BDIS_STORE_U8)
        return "bad storage";
    if (!finite_nonneg(p.hess_eps)) return "hess_eps must be >= 0";
    if (p.use_sgmm != 0 && p.use_sgmm != 1) return "use_sgmm must be 0 or 1";
    if (p.use_c2f != 0 && p.use_c2f != 1) return "use_c2f must be 0 or 1";
    if (p.weight_mode != BDIS_WEIGHT_BDIS && p.weight_mode != BDIS_WEIGHT_DIS) return "bad weight_mode";
    if (p.finest_level < 0 || p.finest_level >= p.levels) return "finest_level must be in [0, levels-1]";
    if (p.fast_exp != 0 && p.fast_exp != 1) return "fast_exp must be 0 or 1";
    return "";
}

std::string check_pair(const bdis_params &p, const bdis_pair &q) {
    if (!q.left || !q.right || !q.disp || !q.valid) return "null image or output pointer";
    if (q.w < 1 || q.h < 1 || q.w > 32768 || q.h > 32768) return "w, h must be in [1, 32768]";
    if (q.pitch < q.w) return "pitch must be >= w";
    const int wl = level_dim(q.w, p.levels - 1), hl = level_dim(q.h, p.levels - 1);
    if (wl < p.patch || hl < p.patch)
        return "image too small: the coarsest level must be at least patch pixels per axis";
    return "";
}

}  // namespace bdis

namespace {

void fill_sgmm(const bdis_params &p, float *m) {
    // 1D factor of Eq. 8: m[a] = sum_{j<P} exp(-(a - j)^2 / (2 sigma_s^2)),
    // the 2D kernel being m[a] m[b]
    for (int a = 0; a < kMaxPatch; ++a) {
        double s = 0.0;
        if (a < p.patch)
            for (int j = 0; j < p.patch; ++j)
                s += std::exp(-(double)(a - j) * (a - j) / (2.0 * p.sigma_s * p.sigma_s));
        m[a] = (float)s;
    }
}

float tau_at(const bdis_params &p) { return p.search_radius > 0.f ? p.search_radius : (float)p.patch; }

LaunchArgs base_args(const bdis_params &p, int level, const LevelDesc *descs, int npairs) {
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.descs = descs;
    a.npairs = npairs;
    a.level = level;
    a.levels = p.levels;
    a.P = p.patch;
    a.S = p.stride;
    a.iters = p.iters;
    a.window_step = p.window_step;
    a.conv_eps = p.conv_eps;
    a.valid_gamma = p.valid_gamma;
    a.pix_thresh = p.pix_thresh;
    a.tau = tau_at(p);
    a.tau0 = tau_at(p);
    a.hess_eps = p.hess_eps;
    // Gamma weight over the processed levels finest .. L-1 (Eq. 11)
    double s = 0.0;
    for (int m = p.finest_level; m < p.levels; ++m) s += std::ldexp(1.0, m);
    a.gamma_w = (float)(std::ldexp(1.0, level) / s);
    a.finest = p.finest_level;
    a.weight_mode = p.weight_mode;
    a.fast_exp = p.fast_exp;
    a.sigma_r_mode = p.sigma_r_mode;
    a.sigma_r_floor = p.sigma_r_floor;
    a.sigma_r_fixed = p.sigma_r_fixed;
    a.variance = p.variance;
    a.pdf_iters = p.pdf_iters;
    a.pdf_resid = p.pdf_resid;
    a.use_c2f = p.use_c2f;
    a.use_sgmm = p.use_sgmm;
    fill_sgmm(p, a.m);
    return a;
}

// Arena layout and descriptor tables of one call.
struct Plan {
    size_t bytes = 0;
    size_t off_desc = 0;
    size_t off_acc = 0, acc_count = 0;  // sigma_r accumulators, contiguous
    size_t off_stages = 0;              // stage arguments of the persistent form (3 per level)
    size_t off_bar = 0;                 // barrier arrivals, generation, timeout flag
    std::vector<LevelDesc> descs;  // [level][pair]
    int wmax[kMaxLevels] = {0};
    int units[kMaxLevels][W_COUNT] = {{0}};
    // arena offsets, index level * n + pair
    std::vector<size_t> oG, oL, oR, oD, oQ, oV, oW, oRec, oFuse, oSr;
};

struct Bump {
    size_t off = 0;
    size_t take(size_t n) {
        off = align_up(off, 256);
        size_t r = off;
        off += n;
        return r;
    }
};

// Phase 1: geometry, work ranges and arena offsets.
void plan_layout(const bdis_params &p, int n, const bdis_pair *pairs, const LevelCfg *cfg,
                 Plan &pl, bool wsum) {
    const int NL = p.levels, P = p.patch, S = p.stride;
    const size_t esz = elem_size(image_type_of(p.storage));  // pyramid images
    const size_t gsz = elem_size(grad_type_of(p.storage));   // gradients
    const size_t cnt = (size_t)NL * n;
    pl.descs.assign(cnt, LevelDesc{});
    // every byte defined (padding included): the table keys the upload skip
    // and the graph replay bytewise
    std::memset(pl.descs.data(), 0, sizeof(LevelDesc) * cnt);
    for (auto *v : {&pl.oG, &pl.oL, &pl.oR, &pl.oD, &pl.oQ, &pl.oV, &pl.oW, &pl.oRec, &pl.oFuse, &pl.oSr})
        v->assign(cnt, 0);
    const int F = p.finest_level;
    Bump b;
    // the persistent form's barrier words sit at the start of the arena,
    // whatever the pair count (they are cleared before every cooperative launch)
    pl.off_bar = b.take(4 * sizeof(unsigned));
    pl.off_desc = b.take(sizeof(LevelDesc) * cnt);
    pl.off_stages = b.take(sizeof(LaunchArgs) * 3 * NL);
    pl.acc_count = 3 * cnt;
    pl.off_acc = b.take(sizeof(unsigned long long) * pl.acc_count);
    for (int l = 0; l < NL; ++l) {
        const int chunk = search_chunk(P, cfg[l].passes);
        int begin[W_COUNT] = {0, 0, 0, 0};
        pl.wmax[l] = 0;
        for (int i = 0; i < n; ++i) {
            const size_t k = (size_t)l * n + i;
            LevelDesc &d = pl.descs[k];
            d.w = level_dim(pairs[i].w, l);
            d.h = level_dim(pairs[i].h, l);
            pl.wmax[l] = std::max(pl.wmax[l], d.w);
            d.npx = num_origins(d.w, P, S, &d.kxreg);
            d.npy = num_origins(d.h, P, S, &d.kyreg);
            d.nchunks = (d.npx + chunk - 1) / chunk;
            d.tiles_x = (d.w + cfg[l].tile_w - 1) / cfg[l].tile_w;
            const bool searched = l >= F;
            const int units[W_COUNT] = {
                ((d.w + 63) / 64) * ((d.h + 31) / 32),             // pyramid: 64 x 32 tiles
                searched ? d.npy * d.nchunks : 0,                 // search: chunks of a patch row
                searched ? d.tiles_x * ((d.h + cfg[l].tile_h - 1) / cfg[l].tile_h) : 0,  // fuse tiles
                (l == 0 && F > 0)
                    ? (int)(((size_t)d.w * d.h + kUpUnitPixels - 1) / kUpUnitPixels) : 0,  // upsample
            };
            for (int q = 0; q < W_COUNT; ++q) {
                d.work_begin[q] = begin[q];
                begin[q] += units[q];
            }
            const size_t gp = align_up((size_t)d.w * esz, 128) / esz;   // image pitch
            const size_t ggp = align_up((size_t)d.w * gsz, 128) / gsz;  // gradient pitch
            d.gpitch = (int)ggp;
            if (searched) pl.oG[k] = b.take(ggp * gsz * d.h);
            if (l == F && F > 0 && p.variance) pl.oV[k] = b.take(sizeof(float) * (size_t)d.w * d.h);
            if (l == 0) {
                d.pitch = pairs[i].pitch;

            } else {
                d.pitch = (int)gp;
                pl.oL[k] = b.take(gp * esz * d.h);
                pl.oR[k] = b.take(gp * esz * d.h);
                pl.oD[k] = b.take(sizeof(float) * (size_t)d.w * d.h);
                pl.oQ[k] = b.take(sizeof(float) * (size_t)d.w * d.h);
            }
            if (wsum && F == 0) pl.oW[k] = b.take(sizeof(float) * (size_t)d.w * d.h);
            const size_t np = searched ? (size_t)d.npx * d.npy : 0;
            if (searched) {
                pl.oRec[k] = b.take(sizeof(bdis_patch_record) * np);
                pl.oFuse[k] = b.take(sizeof(float4) * np);
            }
            pl.oSr[k] = b.take(sizeof(float));
        }
        for (int q = 0; q < W_COUNT; ++q) pl.units[l][q] = begin[q];
    }
    pl.bytes = align_up(b.off, 256);
}

// Phase 2: pointers, once the arena base is known.
void plan_pointers(const bdis_params &p, int n, const bdis_pair *pairs, char *base, Plan &pl,
                   bool wsum) {
    const int NL = p.levels, F = p.finest_level;
    for (int l = 0; l < NL; ++l)
        for (int i = 0; i < n; ++i) {
            const size_t k = (size_t)l * n + i;
            LevelDesc &d = pl.descs[k];
            const bool searched = l >= F;
            d.G = searched ? base + pl.oG[k] : nullptr;
            if (l == 0) {
                d.L = pairs[i].left;
                d.R = pairs[i].right;
                d.D = d.Q = nullptr;
                d.disp = pairs[i].disp;
                d.var = pairs[i].var;
                d.valid = pairs[i].valid;
            } else {
                d.L = base + pl.oL[k];
                d.R = base + pl.oR[k];
                d.D = (float *)(base + pl.oD[k]);
                d.Q = (float *)(base + pl.oQ[k]);
                d.disp = d.var = nullptr;
                d.valid = nullptr;
            }
            if (l == F && F > 0) d.var = p.variance ? (float *)(base + pl.oV[k]) : nullptr;
            d.rec = searched ? (bdis_patch_record *)(base + pl.oRec[k]) : nullptr;
            d.fuse = searched ? (float4 *)(base + pl.oFuse[k]) : nullptr;
            d.sigma_r = (float *)(base + pl.oSr[k]);
            d.acc = (unsigned long long *)(base + pl.off_acc) + 3 * k;
            d.Df = d.Vf = nullptr;
            d.wf = d.hf = 0;
            d.wsum = (wsum && F == 0) ? (float *)(base + pl.oW[k]) : nullptr;
        }
    if (F > 0)
        for (int i = 0; i < n; ++i) {
            LevelDesc &d0 = pl.descs[(size_t)i];
            const LevelDesc &df = pl.descs[(size_t)F * n + i];
            d0.Df = df.D;
            d0.Vf = df.var;
            d0.wf = df.w;
            d0.hf = df.h;
        }
    for (int l = 0; l < NL; ++l)
        for (int i = 0; i < n; ++i) {
            LevelDesc &d = pl.descs[(size_t)l * n + i];
            if (l + 1 < NL) {
                const LevelDesc &c = pl.descs[(size_t)(l + 1) * n + i];
                d.Ln = (void *)c.L;
                d.Rn = (void *)c.R;
                d.wn = d.wc = c.w;
                d.hn = d.hc = c.h;
                d.pitchn = c.pitch;
                d.Dc = c.D;
                d.Qc = c.Q;
            } else {
                d.Ln = d.Rn = nullptr;
                d.Dc = d.Qc = nullptr;
                d.wn = d.hn = d.pitchn = d.wc = d.hc = 0;
            }
        }
}

bdis_status ensure_arena(bdis_handle *h, size_t bytes) {
    if (bytes <= h->arena_cap) return BDIS_OK;
    cudaError_t e;
    if (h->arena) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
        cudaFree(h->arena);
        h->arena = nullptr;
        h->arena_cap = 0;
    }
    const size_t cap = align_up(bytes + bytes / 4, 1 << 20);
    e = cudaMalloc((void **)&h->arena, cap);
    if (e != cudaSuccess) {
        h->arena = nullptr;
        cudaGetLastError();
        return fail(h, BDIS_ENOMEM, "cudaMalloc of the scratch arena failed");
    }
    // zeroed once (every element is written before it is read; the barrier
    // words are also cleared before each persistent launch)
    e = cudaMemset(h->arena, 0, cap);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset");
    h->arena_cap = cap;
    h->last_upload.clear();
    return BDIS_OK;
}

bdis_status ensure_pinned(bdis_handle *h, size_t bytes) {
    if (!h->upload_done) {
        cudaError_t e = cudaEventCreateWithFlags(&h->upload_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    }
    if (bytes <= h->pinned_cap) return BDIS_OK;
    cudaError_t e = cudaEventSynchronize(h->upload_done);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    h->pinned_cap = 0;
    const size_t cap = align_up(bytes, 1 << 16);
    e = cudaMallocHost((void **)&h->pinned, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, BDIS_ENOMEM, "cudaMallocHost of the descriptor staging failed");
    }
    h->pinned_cap = cap;
    return BDIS_OK;
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

const LevelCfg kDefaultCfg{2, 32, 16};
constexpr int kFormLaunches = 0;
constexpr int kFormPersistent = -1;

// The mapped page-locked status word that cooperative launches set when a
// grid-barrier wait runs out (allocated on first use).
bdis_status ensure_status_word(bdis_handle *h) {
    if (h->status_host) return BDIS_OK;
    cudaError_t e = cudaHostAlloc((void **)&h->status_host, sizeof(int),
                                  cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        __atomic_store_n(h->status_host, 0, __ATOMIC_SEQ_CST);
        e = cudaHostGetDevicePointer((void **)&h->status_dev, h->status_host, 0);
    }
    if (e != cudaSuccess) {
        if (h->status_host) cudaFreeHost(h->status_host);
        h->status_host = h->status_dev = nullptr;
        cudaGetLastError();
        return fail(h, BDIS_ENOMEM, "mapped page-locked status word unavailable");
    }
    return BDIS_OK;
}
const LevelCfg kSearchCands[4] = {{1, 32, 16}, {2, 64, 32}, {4, 64, 64}, {3, 64, 32}};

// The whole coarse-to-fine pipeline for n pairs with per-level launch
// configuration cfg.  graph: replay / capture allowed; prof: bracket each
// launch with events (kernel id and level recorded in h->ev_marks).
bdis_status run_cfg(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st,
                    const LevelCfg *cfg, bool graph, bool prof, int mform = kFormLaunches) {
    const bool mega = mform == kFormPersistent;
    const bdis_params &p = h->p;
    const int NL = p.levels;
    Plan pl;
    const bool wsum = in_type == E_F32;  // the differentiable form keeps the weight sums
    plan_layout(p, n, pairs, cfg, pl, wsum);
    int bpitch[kMaxLevels], bcap[kMaxLevels], cpitch[kMaxLevels];
    size_t ssm[kMaxLevels], fsm[kMaxLevels], smax = 0, fmax = 0;
    for (int l = 0; l < NL; ++l) {
        search_layout(p.patch, p.stride, tau_at(p), p.window_step, cfg[l].passes, bpitch[l], bcap[l],
                      cpitch[l], ssm[l], (h->bulk_copy & 2) != 0);
        fsm[l] = fuse_smem(p.patch, p.stride, cfg[l].tile_w, cfg[l].tile_h);
        smax = std::max(smax, ssm[l]);
        fmax = std::max(fmax, fsm[l]);
    }
    if (smax > 227 * 1024 || fmax > 227 * 1024)
        return fail(h, BDIS_EUNSUPPORTED, "search radius too large for the shared-memory band");
    bdis_status s = ensure_arena(h, pl.bytes);
    if (s != BDIS_OK) return s;
    plan_pointers(p, n, pairs, h->arena, pl, wsum);
    {
        // limits are only raised, so other handles' settings stay valid
        cudaError_t e = prepare_search(p.patch, smax);
        if (e == cudaSuccess) e = prepare_fuse(fmax);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
    }
    const int st_type = image_type_of(p.storage);  // pyramid levels 1..L-1
    const int g_type = grad_type_of(p.storage);    // gradients
    LevelDesc *d_descs = (LevelDesc *)(h->arena + pl.off_desc);
    // stage list: the pyramid levels, then (search, fuse) per level coarse to fine
    std::vector<LaunchArgs> stages;
    std::vector<int> stage_itype;
    // pyramid stages: two steps per launch (level l -> l+1 -> l+2, with the
    // gradients of l and l+1; when l+1 is the coarsest level the launch ends
    // with its gradient) while a coarser level remains, then a single step
    // (the coarsest alone builds only its gradient).  Two steps save launches
    // but recompute a halo: worth it while the launch latency dominates, i.e.
    // for calls of up to 2^21 level-0 pixels.
    size_t px0 = 0;
    for (int i = 0; i < n; ++i) px0 += (size_t)pairs[i].w * pairs[i].h;
    const bool two_steps = h->pyr_steps == 2 || (h->pyr_steps == 0 && px0 <= ((size_t)1 << 21));
    for (int l = 0; l < NL;) {
        LaunchArgs a = base_args(p, l, d_descs + (size_t)l * n, n);
        const bool two = two_steps && l + 1 <= NL - 1;
        a.kind = two ? 4 : 0;
        a.descs2 = two ? d_descs + (size_t)(l + 1) * n : nullptr;
        a.total = pl.units[l][W_PYR];
        if (l == 0) {
            a.acc_zero = (unsigned long long *)(h->arena + pl.off_acc);
            a.acc_count = (int)pl.acc_count;
        }
        stages.push_back(a);
        stage_itype.push_back(l == 0 ? in_type : st_type);
        l += two ? 2 : 1;
    }
    const int F = p.finest_level;
    for (int l = NL - 1; l >= F; --l) {
        LaunchArgs a = base_args(p, l, d_descs + (size_t)l * n, n);
        a.img_type = l == 0 ? in_type : st_type;
        a.chunk = search_chunk(p.patch, cfg[l].passes);
        a.tile_w = cfg[l].tile_w;
        a.tile_h = cfg[l].tile_h;
        a.band_pitch = bpitch[l];
        a.band_cap = bcap[l];
        a.chunk_pitch = cpitch[l];
        a.kind = 1;
        a.total = pl.units[l][W_SEARCH];
        stages.push_back(a);
        stage_itype.push_back(l == 0 ? in_type : st_type);
        a.kind = 2;
        a.total = pl.units[l][W_FUSE];
        stages.push_back(a);
        stage_itype.push_back(l == 0 ? in_type : st_type);
    }
    if (F > 0) {
        LaunchArgs a = base_args(p, 0, d_descs, n);
        a.kind = 3;
        a.total = pl.units[0][W_UP];
        stages.push_back(a);
        stage_itype.push_back(in_type);
    }
    s = ensure_status_word(h);
    if (s != BDIS_OK) return s;
    for (auto &a : stages) {
        a.pdl = h->use_pdl;
        a.prefetch = &a == &stages.front() ? 0 : 1;  // the table is uploaded before the first stage
        a.bulk = h->bulk_copy;
        a.err_host = h->status_dev;
        a.copy_limit = h->barrier_limit;
        a.copy_test = h->barrier_unreachable ? 1 : 0;
    }
    // upload descriptors (and the stage list) unless identical to the last upload
    const size_t dbytes = sizeof(LevelDesc) * pl.descs.size();
    const size_t sbytes = sizeof(LaunchArgs) * stages.size();
    const size_t blob = pl.off_stages - pl.off_desc + sbytes;
    std::vector<char> host((size_t)blob, 0);
    std::memcpy(host.data(), pl.descs.data(), dbytes);
    std::memcpy(host.data() + (pl.off_stages - pl.off_desc), stages.data(), sbytes);
    // graph key: descriptors, stage arguments and the execution form with its
    // barrier settings (launch parameters are baked into a captured graph)
    std::vector<char> key = host;
    {
        const unsigned extra[3] = {(unsigned)mform, h->barrier_limit, h->barrier_unreachable ? 1u : 0u};
        key.insert(key.end(), (const char *)extra, (const char *)extra + sizeof(extra));
    }
    const bool same = h->last_upload.size() == host.size() &&
                      std::memcmp(h->last_upload.data(), host.data(), host.size()) == 0;
    if (!same) {
        s = ensure_pinned(h, host.size());
        if (s != BDIS_OK) return s;
        cudaError_t e = cudaEventSynchronize(h->upload_done);  // staging free again
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
        std::memcpy(h->pinned, host.data(), host.size());
        e = cudaMemcpyAsync(d_descs, h->pinned, host.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "descriptor upload");
        e = cudaEventRecord(h->upload_done, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
        h->last_upload.swap(host);
    }

    // one kernel launch, optionally bracketed by profiling events
    auto timed = [&](int kid, auto &&fn) -> cudaError_t {
        size_t i0 = 0;
        if (prof) {
            i0 = h->ev_marks.empty() ? 0 : h->ev_marks.back().second + 2;
            while (h->ev_pool.size() < i0 + 2) {
                cudaEvent_t ev;
                cudaError_t e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return e;
                h->ev_pool.push_back(ev);
            }
            cudaError_t e = cudaEventRecord(h->ev_pool[i0], st);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = fn();
        if (e != cudaSuccess) return e;
        if (prof) {
            e = cudaEventRecord(h->ev_pool[i0 + 1], st);
            if (e != cudaSuccess) return e;
            h->ev_marks.emplace_back(kid, i0);
        }
        return cudaSuccess;
    };

    if (mega && p.storage == BDIS_STORE_U8)
        return fail(h, BDIS_EUNSUPPORTED, "no persistent form with 8-bit pyramids");
    if (mega) {
        // persistent form: one cooperative launch runs every stage
        const size_t msm = std::max(kPyr2SmemBytes, std::max(smax, fmax));
        const int grid = mega_grid(p.patch, st_type, msm);
        if (grid < 1) return fail(h, BDIS_EUNSUPPORTED, "persistent form unavailable");
        MegaArgs m;
        m.stages = (const LaunchArgs *)(h->arena + pl.off_stages);
        m.nstages = (int)stages.size();
        m.bar = (unsigned *)(h->arena + pl.off_bar);
        m.err = (int *)(m.bar + 2);
        m.spin_limit = h->barrier_limit;
        m.unreachable = h->barrier_unreachable ? 1 : 0;
        s = ensure_status_word(h);
        if (s != BDIS_OK) return s;
        m.err_host = h->status_dev;
        // arrival counter, generation and timeout flag start at zero in every launch
        cudaError_t e = cudaMemsetAsync(m.bar, 0, 4 * sizeof(unsigned), st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
        e = timed(BDIS_K_PERSISTENT,
                  [&] { return launch_mega(m, p.patch, st_type, grid, msm, false, st); });
        if (e != cudaSuccess) return cuda_fail(h, e, "persistent launch");
        h->descs = pl.descs;
        h->npairs = n;
        h->levels = NL;
        h->in_type = in_type;
        h->d_descs = d_descs;
        h->err_flag = m.err;
        h->last_persistent = 1;
        h->repeat_ok = false;
        return BDIS_OK;
    }

    // Coarse levels in one cooperative launch (mform = k > 0): the pyramid
    // stages that start at level >= NL - k and the search and fuse stages of
    // levels >= NL - k, which are consecutive in the stage list.  Their grids
    // are small, so one launch with grid barriers between the stages replaces
    // several short dependent launches.
    size_t cm_first = stages.size(), cm_count = 0;
    int cm_grid = 0;
    size_t cm_smem = 0;
    MegaArgs cm{};
    if (mform > 0 && mega_supported(p.patch) && p.storage != BDIS_STORE_U8) {
        const int lmin = NL - mform;
        for (size_t k = 0; k < stages.size(); ++k) {
            const LaunchArgs &a = stages[k];
            const bool in = a.kind != 3 && a.level >= lmin && lmin > F;
            if (in && cm_count == 0) cm_first = k;
            if (in) ++cm_count;
        }
        int umax = 0;
        for (size_t k = cm_first; k < cm_first + cm_count; ++k) umax = std::max(umax, stages[k].total);
        cm_smem = std::max(kPyr2SmemBytes, std::max(smax, fmax));
        cm_grid = std::min(mega_grid(p.patch, st_type, cm_smem), std::max(1, umax));
        if (cm_count < 2 || cm_grid < 1) {
            cm_first = stages.size();
            cm_count = 0;
        } else {
            s = ensure_status_word(h);
            if (s != BDIS_OK) return s;
            cm.stages = (const LaunchArgs *)(h->arena + pl.off_stages) + cm_first;
            cm.nstages = (int)cm_count;
            cm.bar = (unsigned *)(h->arena + pl.off_bar);
            cm.err = (int *)(cm.bar + 2);
            cm.spin_limit = h->barrier_limit;
            cm.unreachable = h->barrier_unreachable ? 1 : 0;
            cm.err_host = h->status_dev;
        }
    }

    auto launch_all = [&]() -> bdis_status {
        cudaError_t e;
        for (size_t k = 0; k < stages.size(); ++k) {
            const LaunchArgs &a = stages[k];
            const int itype = stage_itype[k];
            if (k == cm_first) {
                e = cudaMemsetAsync(cm.bar, 0, 4 * sizeof(unsigned), st);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
                // with programmatic serialisation where the runtime accepts it
                // on a cooperative launch (remembered per process)
                static int pdl_ok = -1;
                const bool try_pdl = h->use_pdl && pdl_ok != 0;
                e = timed(BDIS_K_PERSISTENT + 16 * stages[cm_first].level, [&] {
                    cudaError_t r = launch_mega(cm, p.patch, st_type, cm_grid, cm_smem, try_pdl, st);
                    if (r != cudaSuccess && try_pdl) {
                        cudaGetLastError();
                        r = launch_mega(cm, p.patch, st_type, cm_grid, cm_smem, false, st);
                        if (r == cudaSuccess) pdl_ok = 0;
                    } else if (r == cudaSuccess && try_pdl) {
                        pdl_ok = 1;
                    }
                    return r;
                });
                if (e != cudaSuccess) return cuda_fail(h, e, "coarse-level cooperative launch");
                k += cm_count - 1;
                continue;
            }
            if (a.kind == 0 || a.kind == 4) {
                e = timed(BDIS_K_PYRAMID + 16 * a.level, [&] {
                    return a.kind == 4 ? launch_pyramid2(a, itype, st_type, g_type, st)
                                       : launch_pyramid(a, itype, st_type, g_type, st);
                });
                if (e != cudaSuccess) return cuda_fail(h, e, "pyramid launch");
            } else if (a.kind == 1) {
                const size_t sm = ssm[a.level];
                const int occ = search_occupancy(p.patch, itype, g_type, sm, (a.bulk & 2) != 0);
                const int grid = std::max(1, std::min(a.total, sm_count() * occ));
                e = timed(BDIS_K_SEARCH + 16 * a.level,
                          [&] { return launch_search(a, itype, g_type, sm, grid, st); });
                if (e != cudaSuccess) return cuda_fail(h, e, "search launch");
            } else if (a.kind == 2) {
                e = timed(BDIS_K_FUSE + 16 * a.level, [&] { return launch_fuse(a, fsm[a.level], st); });
                if (e != cudaSuccess) return cuda_fail(h, e, "fuse launch");
            } else {
                e = timed(BDIS_K_UPSAMPLE + 16 * a.level, [&] { return launch_upsample(a, st); });
                if (e != cudaSuccess) return cuda_fail(h, e, "upsample launch");
            }
        }
        return BDIS_OK;
    };

    // Graph replay: only on a non-default stream that is not already being
    // captured by the caller, and only for the exact descriptors captured.
    bool can_graph = graph && h->use_graph && !prof && st != nullptr;
    if (can_graph) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            can_graph = false;
        cudaGetLastError();
    }
    const bool graph_hit = can_graph && h->graph_exec != nullptr && h->graph_descs == key;
    h->repeat_ok = false;
    if (graph_hit) {
        cudaError_t e = cudaGraphLaunch(h->graph_exec, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
        h->repeat_ok = true;
    } else if (can_graph) {
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
            h->graph_descs.clear();
        }
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = launch_all();
            if (s != BDIS_OK) return s;
        } else {
            s = launch_all();
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (s == BDIS_OK && e2 == cudaSuccess) {
                e2 = cudaGraphInstantiate(&h->graph_exec, g, 0);
                if (e2 != cudaSuccess) h->graph_exec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
            if (s == BDIS_OK && e2 == cudaSuccess) {
                h->graph_descs = key;
                e2 = cudaGraphLaunch(h->graph_exec, st);
                if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaGraphLaunch");
                h->repeat_ok = true;
            } else {
                // a launch that cannot be captured or instantiated (nothing
                // has run yet): issue the same launches directly
                cudaGetLastError();
                s = launch_all();
                if (s != BDIS_OK) return s;
            }
        }
    } else {
        s = launch_all();
        if (s != BDIS_OK) return s;
    }
    h->descs = pl.descs;
    h->npairs = n;
    h->levels = NL;
    h->in_type = in_type;
    h->d_descs = d_descs;
    h->last_persistent = cm_count > 0 ? 2 : 0;
    if (cm_count > 0) h->err_flag = cm.err;
    return BDIS_OK;
}

std::string geometry_key(const bdis_handle *h, int n, const bdis_pair *pairs, int in_type) {
    std::string k = std::to_string(in_type) + ":" + std::to_string(n);
    for (int i = 0; i < n; ++i) k += ":" + std::to_string(pairs[i].w) + "x" + std::to_string(pairs[i].h);
    (void)h;
    return k;
}

// Autotuner: times the candidate configurations with per-launch events on
// this geometry and keeps, per level, the fastest search passes and the
// fastest fuse tile.  Every configuration computes identical results.
bdis_status autotune(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st,
                     std::vector<LevelCfg> &best) {
    const int NL = h->p.levels;
    std::vector<LevelCfg> cfg((size_t)NL, kDefaultCfg);
    bdis_status s = run_cfg(h, n, pairs, in_type, st, cfg.data(), false, false);  // warm-up
    if (s != BDIS_OK) return s;
    // every candidate is timed five times (interleaved) and keeps its fastest
    // run, so that noisy timings of short launches do not decide a level's
    // configuration
    double tsearch[4][kMaxLevels], tfuse[4][kMaxLevels];
    for (int c = 0; c < 4; ++c)
        for (int l = 0; l < kMaxLevels; ++l) tsearch[c][l] = tfuse[c][l] = 1e30;
    for (int it = 0; it < 20; ++it) {
        const int c = it % 4;
        for (int l = 0; l < NL; ++l) cfg[l] = kSearchCands[c];
        const size_t m0 = h->ev_marks.size();
        s = run_cfg(h, n, pairs, in_type, st, cfg.data(), false, true);
        if (s != BDIS_OK) return s;
        // search and fuse marks come coarsest level first
        int ns = 0, nf = 0;
        for (size_t m = m0; m < h->ev_marks.size(); ++m) {
            float ms = 0.f;
            const size_t ev = h->ev_marks[m].second;
            cudaError_t e = cudaEventSynchronize(h->ev_pool[ev + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev_pool[ev], h->ev_pool[ev + 1]);
            if (e != cudaSuccess) return cuda_fail(h, e, "autotune events");
            const int kid = h->ev_marks[m].first & 15;
            if (kid == BDIS_K_SEARCH) {
                double &t = tsearch[c][NL - 1 - ns++];
                t = std::min(t, (double)ms);
            } else if (kid == BDIS_K_FUSE) {
                double &t = tfuse[c][NL - 1 - nf++];
                t = std::min(t, (double)ms);
            }
        }
        h->ev_marks.resize(m0);
    }
    best.assign((size_t)NL, kDefaultCfg);
    for (int l = h->p.finest_level; l < NL; ++l) {
        int bs = 0, bf = 0;
        for (int c = 1; c < 4; ++c) {
            if (tsearch[c][l] < tsearch[bs][l]) bs = c;
            if (tfuse[c][l] < tfuse[bf][l]) bf = c;
        }
        best[l].passes = kSearchCands[bs].passes;
        best[l].tile_w = kSearchCands[bf].tile_w;
        best[l].tile_h = kSearchCands[bf].tile_h;
    }
    return BDIS_OK;
}

// Mean device time of `reps` back-to-back calls of one form (events).
bdis_status time_form(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st,
                      const LevelCfg *cfg, int mform, int reps, float &ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(h, cudaGetLastError(), "cudaEventCreate");
    }
    bdis_status s = run_cfg(h, n, pairs, in_type, st, cfg, true, false, mform);  // warm / capture
    if (s == BDIS_OK) {
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == BDIS_OK; ++r)
            s = run_cfg(h, n, pairs, in_type, st, cfg, true, false, mform);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (s == BDIS_OK && e != cudaSuccess) s = cuda_fail(h, e, "autotune events");
        ms /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

// Runs the whole pipeline for n pairs with the tuned configuration of this
// geometry (tuned on first use unless the stream is being captured).
bdis_status run_tuned(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st);

int option_bits(const bdis_handle *h) {
    return (h->use_graph ? 1 : 0) | (h->profile ? 2 : 0) | (h->use_pdl << 14) | (h->autotune ? 8 : 0) |
           (h->form << 4) | (h->pyr_steps << 6) | (h->search_passes << 18) | (h->fuse_tile << 21) | (h->coarse_levels << 8) |
           (h->barrier_unreachable ? 1 << 12 : 0) | ((h->bulk_copy & 1) << 13) | ((h->bulk_copy & 2) << 15);
}

// A persistent launch whose grid-barrier wait ran out has stored 1 in the
// handle's mapped status word: the next call that looks at it (any call on
// the handle; bdis_get_stats and bdis_wait after synchronising) takes the
// word and fails.  That launch's outputs are not valid.
bdis_status take_status(bdis_handle *h) {
    if (!h->status_host) return BDIS_OK;
    if (__atomic_exchange_n(h->status_host, 0, __ATOMIC_SEQ_CST) != 0)
        return fail(h, BDIS_ECUDA,
                    "a bounded device wait (a grid-barrier wait of a cooperative launch, or the "
                    "wait for a bulk copy) ran out in an earlier call: that call's outputs are "
                    "not valid");
    return BDIS_OK;
}

bdis_status run(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st) {
    {
        const bdis_status ps = take_status(h);
        if (ps != BDIS_OK) return ps;
    }
    h->last_saved = nullptr;
    // the same call as the last one, which replayed or captured a graph: replay it
    bdis_handle::Repeat &r = h->repeat;
    auto same_pair = [](const bdis_pair &x, const bdis_pair &y) {  // field by field (no padding)
        return x.left == y.left && x.right == y.right && x.w == y.w && x.h == y.h && x.pitch == y.pitch &&
               x.disp == y.disp && x.var == y.var && x.valid == y.valid;
    };
    bool same = h->repeat_ok && h->graph_exec != nullptr && r.in_type == in_type && r.st == st &&
                r.arena == h->arena && r.arena_cap == h->arena_cap && r.opts == option_bits(h) &&
                (int)r.pairs.size() == n;
    for (int i = 0; i < n && same; ++i) same = same_pair(r.pairs[i], pairs[i]);
    if (same) {
        cudaError_t e = cudaGraphLaunch(h->graph_exec, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
        return BDIS_OK;
    }
    bdis_status rs = run_tuned(h, n, pairs, in_type, st);
    if (rs == BDIS_OK) {
        r.pairs.assign(pairs, pairs + n);
        r.in_type = in_type;
        r.st = st;
        r.arena = h->arena;
        r.arena_cap = h->arena_cap;
        r.opts = option_bits(h);
    } else {
        h->repeat_ok = false;
    }
    return rs;
}

bdis_status run_tuned(bdis_handle *h, int n, const bdis_pair *pairs, int in_type, cudaStream_t st) {
    const std::string key = geometry_key(h, n, pairs, in_type);
    auto it = h->tuned.find(key);
    bdis_handle::Tuned t;
    if (it != h->tuned.end()) {
        t = it->second;
    } else {
        bool capturing = false;
        if (st != nullptr) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
                capturing = true;
            cudaGetLastError();
        }
        if (h->autotune && !capturing) {
            bdis_status s = autotune(h, n, pairs, in_type, st, t.cfg);
            if (s != BDIS_OK) return s;
            // the execution forms against each other: the launch sequence, the
            // k coarsest levels in one cooperative launch (k = 1 .. while a
            // finer searched level remains), and, for 8-bit inputs, every
            // stage in one persistent launch
            t.form = kFormLaunches;
            if (mega_supported(h->p.patch) && h->p.storage != BDIS_STORE_U8 && st != nullptr) {
                float best = 0.f;
                s = time_form(h, n, pairs, in_type, st, t.cfg.data(), kFormLaunches, 5, best);
                if (s != BDIS_OK) return s;
                std::vector<int> cands;
                for (int k = 1; h->p.levels - k > h->p.finest_level; ++k) cands.push_back(k);
                if (in_type == E_U8) cands.push_back(kFormPersistent);
                for (int f : cands) {
                    float tf = 0.f;
                    s = time_form(h, n, pairs, in_type, st, t.cfg.data(), f, 5, tf);
                    if (s != BDIS_OK) {  // a form that cannot run here is skipped
                        cudaGetLastError();
                        continue;
                    }
                    if (tf < best) {
                        best = tf;
                        t.form = f;
                    }
                }
            }
            h->tuned[key] = t;
        } else {
            t.cfg.assign((size_t)h->p.levels, kDefaultCfg);
            t.form = kFormLaunches;
        }
    }
    if (h->search_passes > 0)
        for (auto &c : t.cfg) c.passes = h->search_passes;
    if (h->fuse_tile > 0) {
        const int tw[3] = {32, 64, 64}, th[3] = {16, 32, 64};
        for (auto &c : t.cfg) {
            c.tile_w = tw[h->fuse_tile - 1];
            c.tile_h = th[h->fuse_tile - 1];
        }
    }
    int form = t.form;
    if (h->form == 1) form = h->coarse_levels;
    if (h->form == 2) form = (in_type == E_U8 && mega_supported(h->p.patch) &&
                              h->p.storage != BDIS_STORE_U8) ? kFormPersistent
                                                                              : kFormLaunches;
    return run_cfg(h, n, pairs, in_type, st, t.cfg.data(), true, h->profile, form);
}

}  // namespace

extern "C" {

void bdis_default_params(bdis_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->patch = 8;
    p->stride = 4;
    p->levels = 3;
    p->iters = 8;
    p->sigma_s = 4.0f;       // Sec. IV-A
    p->window_step = 0.5f;   // Sec. IV-A: disturbances 0.5 and 1 px
    p->conv_eps = 0.05f;     // Sec. IV-A: early-stopping 0.05
    p->valid_gamma = 0.75f;  // Sec. IV-A
    p->pix_thresh = 0.15f;   // Sec. IV-A
    p->search_radius = 0.f;  // = patch
    p->sigma_r_mode = BDIS_SIGMA_R_POOLED;
    p->sigma_r_floor = 0.5f;
    p->sigma_r_fixed = 8.0f;  // Table VII ablation value
    p->variance = 0;
    p->pdf_iters = 10;        // Sec. III-E
    p->pdf_resid = 0.1f;      // Sec. III-E
    p->storage = BDIS_STORE_F32;
    p->hess_eps = 1e-4f;
    p->use_sgmm = 1;
    p->use_c2f = 1;
    p->weight_mode = BDIS_WEIGHT_BDIS;
    p->finest_level = 0;
    p->fast_exp = 0;
}

bdis_status bdis_create(const bdis_params *p, bdis_handle **out) {
    if (!out) return BDIS_EINVAL;
    *out = nullptr;
    bdis_params q;
    if (p) q = *p; else bdis_default_params(&q);
    if (!check_params(q).empty()) return BDIS_EINVAL;
    bdis_handle *h = new (std::nothrow) bdis_handle();
    if (!h) return BDIS_ENOMEM;
    h->p = q;
    *out = h;
    return BDIS_OK;
}

void bdis_destroy(bdis_handle *h) {
    if (!h) return;
    for (bdis_saved *sv : h->saved) sv->owner = nullptr;  // they stay valid objects to destroy
    if (h->upload_done) {
        cudaEventSynchronize(h->upload_done);
        cudaEventDestroy(h->upload_done);
    }
    if (h->arena) {
        cudaDeviceSynchronize();
        cudaFree(h->arena);
    }
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->garena) cudaFree(h->garena);
    if (h->status_host) {
        cudaDeviceSynchronize();  // no launch may still write the word
        cudaFreeHost(h->status_host);
    }
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    delete h;
}

bdis_status bdis_set_option(bdis_handle *h, int option, int value) {
    if (!h) return BDIS_EINVAL;
    if (option == BDIS_OPT_GRAPH) {
        h->use_graph = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_PROFILE) {
        h->profile = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_AUTOTUNE) {
        h->autotune = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_FORM) {
        if (value < 0 || value > 2) return fail(h, BDIS_EINVAL, "form must be 0, 1 or 2");
        h->form = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_PDL) {
        if (value < 0 || value > 2) return fail(h, BDIS_EINVAL, "pdl must be 0, 1 or 2");
        h->use_pdl = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_HOST_MAPPED) {
        h->host_mapped = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_BARRIER_LIMIT) {
        if (value < 1) return fail(h, BDIS_EINVAL, "barrier limit must be >= 1 poll");
        h->barrier_limit = (unsigned)value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_BARRIER_TEST) {
        h->barrier_unreachable = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_BULK_COPY) {
        if (value < 0 || value > 3) return fail(h, BDIS_EINVAL, "bulk copy option must be 0..3");
        h->bulk_copy = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_COARSE_LEVELS) {
        if (value < 0 || value >= h->p.levels - h->p.finest_level)
            return fail(h, BDIS_EINVAL, "coarse levels must be in [0, levels - finest_level - 1]");
        h->coarse_levels = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_ADJOINT_LEVELS) {
        h->adjoint_levels = value != 0;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_PYRAMID_STEPS) {
        if (value < 0 || value > 2) return fail(h, BDIS_EINVAL, "pyramid steps must be 0, 1 or 2");
        h->pyr_steps = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_FUSE_TILE) {
        if (value < 0 || value > 3) return fail(h, BDIS_EINVAL, "fuse tile must be 0..3");
        h->fuse_tile = value;
        return BDIS_OK;
    }
    if (option == BDIS_OPT_SEARCH_PASSES) {
        if (value < 0 || value > 4) return fail(h, BDIS_EINVAL, "search passes must be 0..4");
        h->search_passes = value;
        return BDIS_OK;
    }
    return fail(h, BDIS_EINVAL, "unknown option");
}

bdis_status bdis_get_profile(bdis_handle *h, bdis_profile *out, int reset) {
    if (!h || !out) return BDIS_EINVAL;
    for (const auto &mk : h->ev_marks) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(h->ev_pool[mk.second + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev_pool[mk.second], h->ev_pool[mk.second + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "profile events");
        const int kid = mk.first & 15, lvl = mk.first >> 4;
        h->prof_launches[kid] += 1;
        h->prof_ms[kid] += ms;
        h->prof_launches_level[kid][lvl] += 1;
        h->prof_ms_level[kid][lvl] += ms;
    }
    h->ev_marks.clear();
    for (int k = 0; k < BDIS_K_COUNT; ++k) {
        out->launches[k] = h->prof_launches[k];
        out->ms[k] = h->prof_ms[k];
        for (int l = 0; l < kMaxLevels; ++l) {
            out->launches_level[k][l] = h->prof_launches_level[k][l];
            out->ms_level[k][l] = h->prof_ms_level[k][l];
        }
        if (reset) {
            h->prof_launches[k] = 0;
            h->prof_ms[k] = 0.0;
            for (int l = 0; l < kMaxLevels; ++l) {
                h->prof_launches_level[k][l] = 0;
                h->prof_ms_level[k][l] = 0.0;
            }
        }
    }
    return BDIS_OK;
}

const char *bdis_strerror(bdis_status s) {
    if ((int)s < 0 || (int)s > 4) return "unknown status";
    return kStatusText[(int)s];
}

const char *bdis_last_error(const bdis_handle *h) { return h ? h->err.c_str() : "null handle"; }

bdis_status bdis_get_params(const bdis_handle *h, bdis_params *out) {
    if (!h || !out) return BDIS_EINVAL;
    *out = h->p;
    out->search_radius = tau_at(h->p);
    return BDIS_OK;
}

bdis_status bdis_match_batched(bdis_handle *h, int n, const bdis_pair *pairs, void *stream) {
    if (!h) return BDIS_EINVAL;
    if (n < 1 || !pairs) return fail(h, BDIS_EINVAL, "need at least one pair");
    for (int i = 0; i < n; ++i) {
        std::string m = check_pair(h->p, pairs[i]);
        if (!m.empty()) return fail(h, BDIS_EINVAL, "pair " + std::to_string(i) + ": " + m);
    }
    return run(h, n, pairs, E_U8, (cudaStream_t)stream);
}

bdis_status bdis_match(bdis_handle *h, const uint8_t *left, const uint8_t *right, int w,
                       int hgt, int pitch, float *disp, float *var, uint8_t *valid,
                       void *stream) {
    bdis_pair q{left, right, w, hgt, pitch, disp, var, valid};
    return bdis_match_batched(h, 1, &q, stream);
}

bdis_status bdis_match_host(bdis_handle *h, const uint8_t *left, const uint8_t *right, int w,
                            int hgt, int pitch, float *disp, float *var, uint8_t *valid,
                            void *stream) {
    if (!h) return BDIS_EINVAL;
    bdis_pair q{left, right, w, hgt, pitch, disp, var, valid};
    std::string m = check_pair(h->p, q);
    if (!m.empty()) return fail(h, BDIS_EINVAL, m);
    cudaStream_t st = (cudaStream_t)stream;
    // Page-locked host buffers that the device can address (cudaMallocHost,
    // cudaHostRegister): the kernels read the inputs and write the outputs in
    // place over the host link, so no staging copies are made.
    if (h->host_mapped) {
        const bool want_var = var && h->p.variance;
        const void *hp[5] = {left, right, disp, want_var ? var : nullptr, valid};
        void *dp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        bool mapped = true;
        for (int i = 0; i < 5 && mapped; ++i) {
            if (hp[i] == nullptr) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, hp[i]) != cudaSuccess || at.type != cudaMemoryTypeHost ||
                at.devicePointer == nullptr) {
                cudaGetLastError();
                mapped = false;
            } else {
                dp[i] = (char *)at.devicePointer + ((const char *)hp[i] - (const char *)at.hostPointer);
            }
        }
        if (mapped) {
            bdis_pair dq{(const uint8_t *)dp[0], (const uint8_t *)dp[1], w, hgt, pitch, (float *)dp[2],
                         (float *)dp[3], (uint8_t *)dp[4]};
            bdis_status s = run(h, 1, &dq, E_U8, st);
            if (s != BDIS_OK) return s;
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
            return BDIS_OK;
        }
    }
    // device staging for the inputs and outputs, after the pipeline's arena
    Plan pl;
    std::vector<LevelCfg> dcfg((size_t)h->p.levels, LevelCfg{2, 32, 16});
    plan_layout(h->p, 1, &q, dcfg.data(), pl, false);
    const size_t img = align_up((size_t)w * hgt, 256);
    const size_t fo = align_up(sizeof(float) * (size_t)w * hgt, 256);
    const size_t extra = 2 * img + 2 * fo + img;
    const size_t base = align_up(pl.bytes, 256);
    bdis_status s = ensure_arena(h, base + extra);
    if (s != BDIS_OK) return s;
    char *dl = h->arena + base;
    char *dr = dl + img;
    float *dd = (float *)(dr + img);
    float *dv = (float *)((char *)dd + fo);
    uint8_t *dm = (uint8_t *)((char *)dv + fo);
    cudaError_t e = cudaMemcpy2DAsync(dl, w, left, pitch, w, hgt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dr, w, right, pitch, w, hgt, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "input copy");
    bdis_pair dq{(const uint8_t *)dl, (const uint8_t *)dr, w, hgt, w, dd,
                 (var && h->p.variance) ? dv : nullptr, dm};
    s = run(h, 1, &dq, E_U8, st);
    if (s != BDIS_OK) return s;
    const size_t npx = (size_t)w * hgt;
    e = cudaMemcpyAsync(disp, dd, sizeof(float) * npx, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && var && h->p.variance)
        e = cudaMemcpyAsync(var, dv, sizeof(float) * npx, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(valid, dm, npx, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "output copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return BDIS_OK;
}

bdis_status bdis_level_view_get(const bdis_handle *h, int pair, int level, bdis_level_view *out) {
    if (!h || !out) return BDIS_EINVAL;
    if (pair < 0 || pair >= h->npairs || level < 0 || level >= h->levels) return BDIS_EINVAL;
    const LevelDesc &d = h->descs[(size_t)level * h->npairs + pair];
    out->w = d.w;
    out->h = d.h;
    out->npx = d.npx;
    out->npy = d.npy;
    out->image_pitch = d.pitch;
    out->grad_pitch = d.gpitch;
    out->storage = level == 0 ? -1 : h->p.storage;
    out->left = d.L;
    out->right = d.R;
    out->grad = d.G;
    out->records = d.rec;
    out->D = d.D;
    out->Q = d.Q;
    out->sigma_r = d.sigma_r;
    return BDIS_OK;
}

bdis_status bdis_get_stats(bdis_handle *h, bdis_stats *out, void *stream) {
    if (!h || !out) return BDIS_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (h->npairs == 0) return fail(h, BDIS_EINVAL, "no call yet");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    out->levels = h->levels;
    out->pairs = h->npairs;
    std::vector<bdis_patch_record> recs;
    for (int l = 0; l < h->levels; ++l) {
        for (int i = 0; i < h->npairs; ++i) {
            const LevelDesc &d = h->descs[(size_t)l * h->npairs + i];
            if (d.rec == nullptr) continue;  // below the finest processed level
            const size_t np = (size_t)d.npx * d.npy;
            recs.resize(np);
            e = cudaMemcpy(recs.data(), d.rec, sizeof(bdis_patch_record) * np, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "stats copy");
            out->patches[l] += (int)np;
            for (const auto &r : recs) out->valid_patches[l] += r.flags == 0u ? 1 : 0;
            if (i == 0) {
                e = cudaMemcpy(&out->sigma_r[l], d.sigma_r, sizeof(float), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_fail(h, e, "stats copy");
            }
        }
    }
    out->persistent = h->last_persistent;
    if (h->last_persistent && h->err_flag) {
        e = cudaMemcpy(&out->barrier_timeouts, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "stats copy");
    }
    std::vector<uint8_t> v;
    for (int i = 0; i < h->npairs; ++i) {
        const LevelDesc &d = h->descs[(size_t)i];
        v.resize((size_t)d.w * d.h);
        e = cudaMemcpy(v.data(), d.valid, v.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "stats copy");
        for (uint8_t b : v) out->valid_pixels += b;
    }
    // the counters are filled either way; a timed-out barrier wait is an error
    return take_status(h);
}

bdis_status bdis_wait(bdis_handle *h, void *stream) {
    if (!h) return BDIS_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return take_status(h);
}

bdis_status bdis_copy(void *dst, const void *src, size_t bytes, void *stream) {
    if (bytes == 0) return BDIS_OK;
    if (!dst || !src) return BDIS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st) != cudaSuccess) return BDIS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BDIS_ECUDA;
    return BDIS_OK;
}

bdis_status bdis_depth(const float *disp, const float *var, long long n, float fb, float *depth,
                       float *depth_var, void *stream) {
    if (n < 0 || !(std::isfinite(fb) && fb > 0.f)) return BDIS_EINVAL;
    if (n == 0) return BDIS_OK;
    if (!disp || !depth) return BDIS_EINVAL;
    if ((var == nullptr) != (depth_var == nullptr)) return BDIS_EINVAL;
    return launch_depth(disp, var, n, fb, depth, depth_var, (cudaStream_t)stream) == cudaSuccess
               ? BDIS_OK : BDIS_ECUDA;
}

bdis_status bdis_match_batched_f32(bdis_handle *h, int n, const bdis_pair_f32 *pairs,
                                   void *stream) {
    if (!h) return BDIS_EINVAL;
    if (n < 1 || !pairs) return fail(h, BDIS_EINVAL, "need at least one pair");
    std::vector<bdis_pair> q((size_t)n);
    for (int i = 0; i < n; ++i) {
        const bdis_pair_f32 &f = pairs[i];
        // level 0 is indexed in elements; check_pair only needs pitch >= w
        q[i] = bdis_pair{(const uint8_t *)f.left, (const uint8_t *)f.right, f.w, f.h, f.pitch,
                         f.disp, f.var, f.valid};
        std::string m = check_pair(h->p, q[i]);
        if (!m.empty()) return fail(h, BDIS_EINVAL, "pair " + std::to_string(i) + ": " + m);
    }
    return run(h, n, q.data(), E_F32, (cudaStream_t)stream);
}

bdis_status bdis_match_f32(bdis_handle *h, const float *left, const float *right, int w, int hgt,
                           int pitch, float *disp, float *var, uint8_t *valid, void *stream) {
    bdis_pair_f32 q{left, right, w, hgt, pitch, disp, var, valid};
    return bdis_match_batched_f32(h, 1, &q, stream);
}

bdis_status bdis_saved_create(bdis_handle *h, bdis_saved **out) {
    if (!out) return BDIS_EINVAL;
    *out = nullptr;
    if (!h) return BDIS_EINVAL;
    bdis_saved *sv = new (std::nothrow) bdis_saved();
    if (!sv) return fail(h, BDIS_ENOMEM, "out of host memory");
    sv->owner = h;
    h->saved.push_back(sv);
    *out = sv;
    return BDIS_OK;
}

void bdis_saved_destroy(bdis_saved *sv) {
    if (!sv) return;
    if (bdis_handle *h = sv->owner) {
        h->saved.erase(std::remove(h->saved.begin(), h->saved.end(), sv), h->saved.end());
        if (h->last_saved == sv) {  // the handle's last-call views pointed into this arena
            h->last_saved = nullptr;
            h->descs.clear();
            h->npairs = 0;
        }
        h->repeat_ok = false;  // a replay must not reuse this arena's address
    }
    if (sv->arena) cudaFree(sv->arena);  // synchronises with work still using it
    delete sv;
}

bdis_status bdis_match_batched_f32_saved(bdis_handle *h, int n, const bdis_pair_f32 *pairs,
                                         bdis_saved *sv, void *stream) {
    if (!h) return BDIS_EINVAL;
    if (!sv) return fail(h, BDIS_EINVAL, "null saved state");
    if (sv->owner != h) return fail(h, BDIS_EINVAL, "saved state created on another handle");
    if (n < 1 || !pairs) return fail(h, BDIS_EINVAL, "need at least one pair");
    std::vector<bdis_pair> q((size_t)n);
    for (int i = 0; i < n; ++i) {
        const bdis_pair_f32 &f = pairs[i];
        q[i] = bdis_pair{(const uint8_t *)f.left, (const uint8_t *)f.right, f.w, f.h, f.pitch,
                         f.disp, f.var, f.valid};
        std::string m = check_pair(h->p, q[i]);
        if (!m.empty()) return fail(h, BDIS_EINVAL, "pair " + std::to_string(i) + ": " + m);
    }
    // the forward runs with the saved state's arena in place of the handle's
    std::swap(h->arena, sv->arena);
    std::swap(h->arena_cap, sv->arena_cap);
    const bdis_status st = run(h, n, q.data(), E_F32, (cudaStream_t)stream);
    std::swap(h->arena, sv->arena);
    std::swap(h->arena_cap, sv->arena_cap);
    if (st != BDIS_OK) {
        sv->npairs = 0;
        sv->descs.clear();
        return st;
    }
    sv->descs = h->descs;
    sv->npairs = h->npairs;
    sv->levels = h->levels;
    sv->in_type = h->in_type;
    h->last_saved = sv;
    return BDIS_OK;
}

namespace {

// Backward plan: per-level launch arguments and work totals.
struct GradPlan {
    int nlev = 1;
    GradArgs a[kMaxLevels];
    int tot[kMaxLevels][G_COUNT];
    size_t zero_off = 0, zero_bytes = 0;  // gradient buffers of levels >= 1 (zeroed per call)
};

// The forward a loss or an adjoint differentiates: a caller-owned saved
// state, or (sv == nullptr) the handle's last call.
struct FwdView {
    const std::vector<LevelDesc> *descs;
    int npairs, levels, in_type;
};

bdis_status fwd_view(bdis_handle *h, const bdis_saved *sv, FwdView &v) {
    if (sv != nullptr) {
        if (sv->owner != h) return fail(h, BDIS_EINVAL, "saved state created on another handle");
        v = FwdView{&sv->descs, sv->npairs, sv->levels, sv->in_type};
    } else {
        v = FwdView{&h->descs, h->npairs, h->levels, h->in_type};
    }
    if (v.npairs < 1 || v.in_type != E_F32)
        return fail(h, BDIS_EINVAL, "no float-image forward to differentiate (call bdis_match_f32)");
    return BDIS_OK;
}

// Builds and uploads the (level, pair) descriptors of the backward pass for
// levels 0 .. nlev-1.
bdis_status grad_setup(bdis_handle *h, const FwdView &fv, const bdis_grad *g, bool need_loss,
                       cudaStream_t st, int nlev, GradPlan &gp) {
    if (!g) return fail(h, BDIS_EINVAL, "null gradient table");
    const bdis_params &p = h->p;
    if (p.finest_level != 0 || p.weight_mode != BDIS_WEIGHT_BDIS || p.fast_exp != 0)
        return fail(h, BDIS_EUNSUPPORTED,
                    "the adjoint covers the default fusion at full resolution "
                    "(finest_level 0, BDIS weights, exact exponential)");
    if (nlev > 1 && p.storage != BDIS_STORE_F32)
        return fail(h, BDIS_EUNSUPPORTED, "the adjoint through every level needs FP32 pyramids");
    const int n = fv.npairs;
    for (int i = 0; i < n; ++i) {
        if (!g[i].g_disp || !g[i].g_left || !g[i].g_right)
            return fail(h, BDIS_EINVAL, "null gradient buffer");
        if (need_loss && !g[i].loss) return fail(h, BDIS_EINVAL, "null loss pointer");
    }
    gp.nlev = nlev;
    const size_t cnt = (size_t)nlev * n;
    std::vector<GradDesc> gd(cnt);
    // every byte defined (padding included): the table is compared bytewise
    // with the last upload
    std::memset(gd.data(), 0, sizeof(GradDesc) * cnt);
    Bump b;
    const size_t off_desc = b.take(sizeof(GradDesc) * cnt);
    std::vector<size_t> oDw(cnt), oG(cnt), od(cnt), opi(cnt), osp(cnt), oce(cnt), olp(cnt), ocp(cnt);
    std::vector<size_t> oL(cnt), oR(cnt), oQ(cnt);
    const int ngrp = 256 / search_group(p.patch);
    for (int l = 0; l < nlev; ++l) {
        int begin[G_COUNT] = {0, 0};
        for (int i = 0; i < n; ++i) {
            const size_t k = (size_t)l * n + i;
            const LevelDesc &d = (*fv.descs)[k];
            GradDesc &q = gd[k];
            q.w = d.w;
            q.h = d.h;
            q.pitch = d.pitch;
            q.gpitch = d.gpitch;
            q.gtype = grad_type_of(p.storage);
            q.npx = d.npx;
            q.npy = d.npy;
            q.kxreg = d.kxreg;
            q.kyreg = d.kyreg;
            const size_t px = (size_t)d.w * d.h, np = (size_t)d.npx * d.npy;
            const int units[G_COUNT] = {(int)((px + 255) / 256), (int)((np + ngrp - 1) / ngrp)};
            for (int u = 0; u < G_COUNT; ++u) {
                q.work_begin[u] = begin[u];
                begin[u] += units[u];
            }
            oDw[k] = b.take(sizeof(float) * px);
            od[k] = b.take(sizeof(float) * np);
            opi[k] = b.take(sizeof(float) * np);
            osp[k] = b.take(sizeof(float) * 2 * ((np + ngrp - 1) / ngrp));
            oce[k] = b.take(sizeof(float));
            olp[k] = b.take(sizeof(float) * ((px + 255) / 256));
            ocp[k] = b.take(sizeof(float) * np * 2 * p.patch * p.patch);
            oG[k] = b.take(sizeof(float) * px);
        }
        for (int u = 0; u < G_COUNT; ++u) gp.tot[l][u] = begin[u];
    }
    // image and probability gradients of the coarser levels: one zeroed block
    gp.zero_off = b.take(0);
    for (int l = 1; l < nlev; ++l)
        for (int i = 0; i < n; ++i) {
            const size_t k = (size_t)l * n + i;
            const size_t px = (size_t)gd[k].w * gd[k].h;
            oL[k] = b.take(sizeof(float) * px);
            oR[k] = b.take(sizeof(float) * px);
            oQ[k] = b.take(sizeof(float) * px);
        }
    gp.zero_bytes = b.off - gp.zero_off;
    const size_t bytes = align_up(b.off, 256);
    if (bytes > h->garena_cap) {
        if (h->garena) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
            cudaFree(h->garena);
            h->garena = nullptr;
            h->garena_cap = 0;
            h->last_grad_upload.clear();
        }
        const size_t cap = align_up(bytes + bytes / 4, 1 << 20);
        if (cudaMalloc((void **)&h->garena, cap) != cudaSuccess) {
            cudaGetLastError();
            h->garena = nullptr;
            return fail(h, BDIS_ENOMEM, "cudaMalloc of the backward scratch failed");
        }
        h->garena_cap = cap;
    }
    char *base = h->garena;
    for (int l = 0; l < nlev; ++l)
        for (int i = 0; i < n; ++i) {
            const size_t k = (size_t)l * n + i;
            const LevelDesc &d = (*fv.descs)[k];
            GradDesc &q = gd[k];
            q.L = (const float *)d.L;
            q.R = (const float *)d.R;
            q.G = d.G;
            q.disp = d.disp;
            q.wsum = d.wsum;
            q.valid = d.valid;
            q.rec = d.rec;
            q.fuse = d.fuse;
            q.sigma_r = d.sigma_r;
            q.Q = l > 0 ? d.Q : nullptr;
            if (l == 0) {
                q.gDisp = g[i].g_disp;
                q.gL = g[i].g_left;
                q.gR = g[i].g_right;
                q.gPatch = g[i].g_patch_disp;
                q.loss = g[i].loss;
                q.gQ = nullptr;
            } else {
                q.gDisp = nullptr;
                q.gL = (float *)(base + oL[k]);
                q.gR = (float *)(base + oR[k]);
                q.gPatch = nullptr;
                q.loss = nullptr;
                q.gQ = (float *)(base + oQ[k]);
            }
            q.gDw = (float *)(base + oDw[k]);
            q.gG = (float *)(base + oG[k]);
            q.gd = (float *)(base + od[k]);
            q.gpi = (float *)(base + opi[k]);
            q.sig_part = (float *)(base + osp[k]);
            q.coefE0 = (float *)(base + oce[k]);
            q.loss_part = (float *)(base + olp[k]);
            q.cpatch = (float *)(base + ocp[k]);
            if (l + 1 < nlev) {
                const size_t kc = (size_t)(l + 1) * n + i;
                q.gQn = (float *)(base + oQ[kc]);
                q.gLc = (const float *)(base + oL[kc]);
                q.gRc = (const float *)(base + oR[kc]);
                q.wn = gd[kc].w;
                q.hn = gd[kc].h;
            } else {
                q.gQn = nullptr;
                q.gLc = q.gRc = nullptr;
                q.wn = q.hn = 0;
            }
            if (q.wsum == nullptr) return fail(h, BDIS_EINVAL, "forward kept no fusion weights");
        }
    const size_t tbytes = sizeof(GradDesc) * cnt;
    GradDesc *d_desc = (GradDesc *)(base + off_desc);
    const bool same = h->last_grad_upload.size() >= tbytes &&
                      std::memcmp(h->last_grad_upload.data(), gd.data(), tbytes) == 0;
    if (!same) {
        bdis_status s = ensure_pinned(h, std::max(tbytes, h->last_upload.size()));
        if (s != BDIS_OK) return s;
        cudaError_t e = cudaEventSynchronize(h->upload_done);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
        std::memcpy(h->pinned, gd.data(), tbytes);
        e = cudaMemcpyAsync(d_desc, h->pinned, tbytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "gradient descriptor upload");
        e = cudaEventRecord(h->upload_done, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
        const char *tb = (const char *)gd.data();
        h->last_grad_upload.assign(tb, tb + tbytes);
    }
    double gsum = 0.0;
    for (int m = 0; m < p.levels; ++m) gsum += std::ldexp(1.0, m);
    for (int l = 0; l < nlev; ++l) {
        GradArgs &a = gp.a[l];
        std::memset(&a, 0, sizeof(a));
        a.descs = d_desc + (size_t)l * n;
        a.npairs = n;
        a.level = l;
        a.P = p.patch;
        a.S = p.stride;
        a.window_step = p.window_step;
        a.gamma_w = (float)(std::ldexp(1.0, l) / gsum);
        a.sigma_r_mode = p.sigma_r_mode;
        a.sigma_r_floor = p.sigma_r_floor;
        a.use_sgmm = p.use_sgmm;
        a.use_c2f = p.use_c2f;
        fill_sgmm(p, a.m);
    }
    return BDIS_OK;
}

}  // namespace

bdis_status bdis_loss(bdis_handle *h, const bdis_saved *sv, float lambda, const bdis_grad *g,
                      void *stream) {
    if (!h) return BDIS_EINVAL;
    if (!std::isfinite(lambda) || lambda < 0.f) return fail(h, BDIS_EINVAL, "lambda must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    FwdView fv;
    bdis_status s = fwd_view(h, sv, fv);
    if (s != BDIS_OK) return s;
    GradPlan gp;
    s = grad_setup(h, fv, g, true, st, 1, gp);
    if (s != BDIS_OK) return s;
    GradArgs a = gp.a[0];
    a.lambda = lambda;
    a.total = gp.tot[0][G_PIX];
    cudaError_t e = launch_loss(a, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "loss launch");
    return BDIS_OK;
}

bdis_status bdis_backward(bdis_handle *h, const bdis_saved *sv, const bdis_grad *g, void *stream) {
    if (!h) return BDIS_EINVAL;
    if (h->p.sigma_r_mode == BDIS_SIGMA_R_LITERAL)
        return fail(h, BDIS_EUNSUPPORTED, "no adjoint for the LITERAL sigma_r reading");
    cudaStream_t st = (cudaStream_t)stream;
    FwdView fv;
    bdis_status s = fwd_view(h, sv, fv);
    if (s != BDIS_OK) return s;
    const int nlev = h->adjoint_levels ? fv.levels : 1;
    GradPlan gp;
    s = grad_setup(h, fv, g, false, st, nlev, gp);
    if (s != BDIS_OK) return s;
    cudaError_t e;
    if (gp.zero_bytes > 0) {
        e = cudaMemsetAsync(h->garena + gp.zero_off, 0, gp.zero_bytes, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    }
    // finest level first: each level's fusion adjoint feeds the next level's dL/dQ
    for (int l = 0; l < nlev; ++l) {
        GradArgs a = gp.a[l];
        a.total = gp.tot[l][G_PIX];
        if ((e = launch_bwd_pix(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
        a.total = gp.tot[l][G_GROUP];
        if ((e = launch_bwd_dens(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
        if ((e = launch_bwd_patch(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
        a.total = gp.tot[l][G_PIX];
        if ((e = launch_bwd_gather(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
        if ((e = launch_bwd_sobel(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
    }
    // pyramid transpose, coarsest first
    for (int l = nlev - 2; l >= 0; --l) {
        GradArgs a = gp.a[l];
        a.total = gp.tot[l][G_PIX];
        if ((e = launch_bwd_pyr(a, st)) != cudaSuccess) return cuda_fail(h, e, "backward launch");
    }
    return BDIS_OK;
}

}  // extern "C"
