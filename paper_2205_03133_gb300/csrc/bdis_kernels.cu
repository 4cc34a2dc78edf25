// bdis_kernels.cu -- sm_103a kernels of the BDIS forward pipeline.
//
// Every kernel processes one pyramid level of a whole batch of pairs: work
// units are flattened over the pairs through LevelDesc::work_begin, and each
// block strides over the units (grid sized to the SM count), so the plain
// single-pair call and the batched call run the same code.
//   k_pyramid   one pyramid step (64x32 tiles staged in shared memory): the
//               [1 4 6 4 1]/16 blur and decimation of L and R and Sobel-x/8 of
//               the left image (Sec. III-A)
//   k_pyramid2  two steps per launch (level l -> l+1 -> l+2 with the gradients
//               of l and l+1), the level-(l+1) halo recomputed in the block
//   k_search    inverse-compositional GN per patch (Eq. 1), window energies,
//               rejection flags (Sec. III-B, Sec. IV technical details), and the
//               sums of the dynamic sigma_r (text after Eq. 6), accumulated in
//               exact 64-bit fixed point
//   k_fuse      per 32x16, 64x32 or 64x64 pixel tile: window posterior (Eq. 5-6),
//               coarse-to-fine rho (Eq. 10-11) and PDF fit (Eq. 14-16) of the
//               patches overlapping the tile, then the sGMM fusion gather
//               (Eq. 8-9, Eq. 12) and pixel variance (Eq. 17)
//   k_upsample  full-resolution output from a finest processed level f > 0
//   k_depth     depth and its variance (Eq. 13, Eq. 17)
//   k_mega      every stage of a call in one cooperative launch, with a
//               bounded grid barrier between dependent stages
#include <algorithm>
#include <climits>
#include <cfloat>
#include <cstring>
#include <cmath>

#include "bdis_device.cuh"

namespace bdis {
namespace {

// Entry and exit of a stage kernel launched with programmatic stream
// serialisation.  With `early` the next kernel may be scheduled at once (it
// still waits in pdl_wait() for this one to complete); otherwise each block
// releases it at its end.  A stage whose descriptor table is complete before
// it starts (every stage after a call's first) prefetches its single
// descriptor into L1 while it waits for its predecessor.
__device__ __forceinline__ void pdl_enter(const LaunchArgs &a) {
    if (a.early) pdl_release();
    if (a.prefetch && a.npairs == 1 && threadIdx.x * 128 < sizeof(LevelDesc))
        asm volatile("prefetch.L1 [%0];" ::"l"((const char *)a.descs + 128 * threadIdx.x));
    pdl_wait();
}
__device__ __forceinline__ void pdl_leave(const LaunchArgs &a) {
    if (!a.early) pdl_release();
}

// ---------------------------------------------------------------- pyramid

// A block owns a 64 x 32 pixel tile of level l and the 32 x 16 tile of
// level l+1 under it.  It stages the 72 x 36 region of L (and R when a
// coarser level is built) that starts 4 columns and 2 rows before the tile,
// with reflect-101 indices applied once, then writes Sobel-x/8 of L for the
// 64 x 32 pixels and the [1 4 6 4 1]/16 blur of L and R at the even pixels
// (2X, 2Y).  A region inside the image with rows aligned to four elements is
// staged with four-element loads; a thread computes eight Sobel outputs of a
// row, four horizontally blurred columns and two blurred pixels from 16-byte
// shared-memory reads, and stores them as vectors where the row allows.
constexpr int kPyrTW = 64, kPyrTH = 32;
constexpr int kPyrSW = kPyrTW + 8, kPyrSH = kPyrTH + 4;
constexpr int kPyrOX = 4;  // staged column of the tile's first pixel
// Row pitches (floats) of the staged region and of the horizontal blur:
// 76 = 12 and 36 = 4 modulo 32 banks, so eight consecutive rows at the same
// column fall in distinct 4-bank groups (16-byte reads and writes by a
// quarter warp without conflicts).
constexpr int kPyrSP = kPyrSW + 4, kPyrHP = kPyrTW / 2 + 4;
static_assert(kPyrSmemBytes == sizeof(float) * (2 * kPyrSH * kPyrSP + 2 * kPyrSH * kPyrHP),
              "one-step pyramid shared memory");

// Staging of a one-step tile's region (72 x 36 pixels from 4 columns and 2
// rows before the tile) by the block's own loads: four-element vector loads
// for a region inside the image with rows aligned to four elements, else
// element loads with reflect-101 indices.
template <typename TI>
__device__ __forceinline__ void pyramid_stage_loads(const LevelDesc &D, int tx, int ty,
                                                    float (*Ls)[kPyrSP], float (*Rs)[kPyrSP]) {
    const int xs = tx * kPyrTW - kPyrOX, y0 = ty * kPyrTH - 2;  // region origin
    const int w = D.w, h = D.h, pitch = D.pitch;
    const TI *L = (const TI *)D.L;
    const TI *R = (const TI *)D.R;
    const bool next = D.Ln != nullptr;
    const int tid = threadIdx.x;
    const bool vec_in = xs >= 0 && xs + kPyrSW <= w && y0 >= 0 && y0 + kPyrSH <= h && pitch % 4 == 0 &&
                        ((uintptr_t)L | (next ? (uintptr_t)R : (uintptr_t)0)) % (4 * sizeof(TI)) == 0;
    // all of a thread's loads are issued before its stores (memory-level parallelism);
    // every launch of the pyramid stage uses 256 threads
    if (vec_in) {
        constexpr int NV = kPyrSH * (kPyrSW / 4);
        constexpr int PER = (NV + 255) / 256;
        float4 vl[PER], vr[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * 256;
            if (i < NV) {
                const int r = i / (kPyrSW / 4), c = 4 * (i - r * (kPyrSW / 4));
                const size_t o = (size_t)(y0 + r) * pitch + xs + c;
                vl[k] = ld4f(L + o);
                vr[k] = next ? ld4f(R + o) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * 256;
            if (i < NV) {
                const int r = i / (kPyrSW / 4), c = 4 * (i - r * (kPyrSW / 4));
                *(float4 *)&Ls[r][c] = vl[k];
                if (next) *(float4 *)&Rs[r][c] = vr[k];
            }
        }
    } else {
        // image borders or unaligned rows: element loads with reflected
        // indices, in two batches of loads in flight
        constexpr int NEL = kPyrSH * kPyrSW;
        constexpr int PER = (NEL + 511) / 512;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float vl[PER], vr[PER];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int i = tid + (half * PER + k) * 256;
                if (i < NEL) {
                    const int r = i / kPyrSW, c = i - r * kPyrSW;
                    // only indices within 2 of the image are ever used by a stencil
                    const int gy = refl(min(max(y0 + r, -2), h + 1), h);
                    const int gx = refl(min(max(xs + c, -2), w + 1), w);
                    vl[k] = ldf(L + (size_t)gy * pitch + gx);
                    vr[k] = next ? ldf(R + (size_t)gy * pitch + gx) : 0.f;
                }
            }
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int i = tid + (half * PER + k) * 256;
                if (i < NEL) {
                    const int r = i / kPyrSW, c = i - r * kPyrSW;
                    Ls[r][c] = vl[k];
                    if (next) Rs[r][c] = vr[k];
                }
            }
        }
    }
}

// Sobel-x/8 of L over the 64 x 32 tile and the blurred, decimated 32 x 16
// tile of the next level of L and R, from the staged region.
template <typename TN, typename TG>
__device__ __forceinline__ void pyramid_compute(const LevelDesc &D, int tx, int ty,
                                                float (*Ls)[kPyrSP], float (*Rs)[kPyrSP],
                                                float (*Lh)[kPyrHP], float (*Rh)[kPyrHP]) {
    const int w = D.w, h = D.h;
    const bool next = D.Ln != nullptr;
    const int tid = threadIdx.x;
    TG *G = (TG *)D.G;  // nullptr below the finest processed level
    if (G != nullptr) {
        // pixels lx0 .. lx0 + 7 of row ly: staged columns lx0 + 3 .. lx0 + 12
        // of rows ly + 1 .. ly + 3.  A quarter warp takes eight rows of one
        // segment (conflict-free shared reads); a warp, eight rows of four
        // segments (whole 32-byte sectors of G)
        const int lane = tid & 31, wp = tid >> 5;
        const int ly = (wp & 3) * 8 + (lane & 7), lx0 = ((wp >> 2) * 4 + (lane >> 3)) * 8;
        const int x = tx * kPyrTW + lx0, y = ty * kPyrTH + ly;
        if (x < w && y < h) {
            float u[3][10];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float *row = Ls[ly + 1 + q] + lx0;
                const float4 c0 = *(const float4 *)row, c1 = *(const float4 *)(row + 4);
                const float4 c2 = *(const float4 *)(row + 8);
                u[q][0] = c0.w;
                u[q][1] = c1.x; u[q][2] = c1.y; u[q][3] = c1.z; u[q][4] = c1.w;
                u[q][5] = c2.x; u[q][6] = c2.y; u[q][7] = c2.z; u[q][8] = c2.w;
                u[q][9] = row[12];
            }
            float g[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float acc = (u[0][j + 2] - u[0][j]) + 2.f * (u[1][j + 2] - u[1][j]) +
                                  (u[2][j + 2] - u[2][j]);
                g[j] = acc * 0.125f;
            }
            TG *gp = G + (size_t)y * D.gpitch + x;
            if (x + 8 <= w && (((uintptr_t)gp) & 15u) == 0) {
                st8(gp, g);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (x + j < w) stf(gp + j, g[j]);
            }
        }
    }
    if (next) {
        // separable blur: horizontal at the even columns of every staged row
        // (outputs q .. q + 3 read staged columns 2q .. 2q + 15), then
        // vertical at the even rows (the multiply-add order of the 2D sum)
        const float k[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
        auto hblur = [&](const float *src, float *dst) {
            float v[16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 a4 = *(const float4 *)(src + 4 * c);
                v[4 * c] = a4.x;
                v[4 * c + 1] = a4.y;
                v[4 * c + 2] = a4.z;
                v[4 * c + 3] = a4.w;
            }
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                o[j] = 0.f;
#pragma unroll
                for (int t = 0; t < 5; ++t) o[j] += k[t] * v[2 * j + 2 + t];
            }
            *(float4 *)dst = make_float4(o[0], o[1], o[2], o[3]);
        };
        // consecutive threads take consecutive rows of one column quad
        for (int i = tid; i < kPyrSH * (kPyrTW / 8); i += blockDim.x) {
            const int qd = i / kPyrSH, r = i - qd * kPyrSH, q = 4 * qd;
            hblur(&Ls[r][2 * q], &Lh[r][q]);
            hblur(&Rs[r][2 * q], &Rh[r][q]);
        }
        __syncthreads();
        {
            const int oy = tid >> 4, ox = (tid & 15) * 2;
            const int X = tx * (kPyrTW / 2) + ox, Y = ty * (kPyrTH / 2) + oy;
            if (X < D.wn && Y < D.hn) {
                const int cy = 2 * oy + 2;
                float aL0 = 0.f, aL1 = 0.f, aR0 = 0.f, aR1 = 0.f;
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const float2 l2 = *(const float2 *)&Lh[cy + j - 2][ox];
                    const float2 r2 = *(const float2 *)&Rh[cy + j - 2][ox];
                    aL0 += k[j] * l2.x;
                    aL1 += k[j] * l2.y;
                    aR0 += k[j] * r2.x;
                    aR1 += k[j] * r2.y;
                }
                TN *lp = (TN *)D.Ln + (size_t)Y * D.pitchn + X;
                TN *rp = (TN *)D.Rn + (size_t)Y * D.pitchn + X;
                const float s = 1.f / 256.f;
                if (X + 1 < D.wn && ((((uintptr_t)lp) | ((uintptr_t)rp)) & (2 * sizeof(TN) - 1)) == 0) {
                    st2(lp, aL0 * s, aL1 * s);
                    st2(rp, aR0 * s, aR1 * s);
                } else {
                    stf(lp, aL0 * s);
                    stf(rp, aR0 * s);
                    if (X + 1 < D.wn) {
                        stf(lp + 1, aL1 * s);
                        stf(rp + 1, aR1 * s);
                    }
                }
            }
        }
    }
}

template <typename TI, typename TN, typename TG>
__device__ __forceinline__ void pyramid_unit(const LaunchArgs &a, int unit, float (*Ls)[kPyrSP],
                                             float (*Rs)[kPyrSP], float (*Lh)[kPyrHP],
                                             float (*Rh)[kPyrHP]) {
    static_assert(kPyrTW * kPyrTH == 8 * 256 && (kPyrTW / 2) * (kPyrTH / 2) == 2 * 256,
                  "one Sobel segment and one blurred pair per thread");
    const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_PYR)];
    const int tile = unit - D.work_begin[W_PYR];
    const int ntx = (D.w + kPyrTW - 1) / kPyrTW;
    const int ty = udiv_small(tile, recip(ntx)), tx = tile - ty * ntx;
    __syncthreads();  // the previous unit's readers are done with the staged region
    pyramid_stage_loads<TI>(D, tx, ty, Ls, Rs);
    __syncthreads();
    pyramid_compute<TN, TG>(D, tx, ty, Ls, Rs, Lh, Rh);
}

// Two pyramid steps in one unit: a 64x32 tile of level l gives its Sobel-x,
// the 32x16 tile of level l+1 with its Sobel-x, and the 16x8 tile of level
// l+2.  The level-(l+1) values the second step reads (the tile plus a
// 2-pixel halo) are computed here from a 76x44 level-l region and rounded to
// the storage type exactly as when they are read back from memory; a halo
// pixel outside level l+1 takes the value of its reflect-101 image pixel.
constexpr int kPyr2SW = kPyrTW + 12, kPyr2SH = kPyrTH + 12;    // level l: +-6
constexpr int kPyr2MW = kPyrTW / 2 + 4, kPyr2MH = kPyrTH / 2 + 4;  // level l+1: +-2
// level l region (L, R), level l+1 region (L, R), horizontal blur rows (L, R)
constexpr size_t kPyr2SmemFloats = 2 * (size_t)kPyr2SW * kPyr2SH + 2 * (size_t)kPyr2MW * kPyr2MH +
                                   2 * (size_t)kPyr2SH * kPyr2MW;
static_assert(kPyr2SmemFloats * sizeof(float) == kPyr2SmemBytes, "two-step pyramid shared memory");

template <typename TO>
__device__ __forceinline__ float round_to(float v) {
    if constexpr (sizeof(TO) == 2) return __half2float(__float2half_rn(v));
    if constexpr (sizeof(TO) == 1) return (float)__float2uint_rn(fminf(fmaxf(v, 0.f), 255.f));
    return v;
}

template <typename TI, typename TN, typename TG>
__device__ __forceinline__ void pyramid2_unit(const LaunchArgs &a, int unit, float *sm) {
    float(*Ls)[kPyr2SW] = (float(*)[kPyr2SW])sm;
    float(*Rs)[kPyr2SW] = Ls + kPyr2SH;
    float(*Lm)[kPyr2MW] = (float(*)[kPyr2MW])(sm + 2 * kPyr2SW * kPyr2SH);
    float(*Rm)[kPyr2MW] = Lm + kPyr2MH;
    float(*Lh)[kPyr2MW] = Rm + kPyr2MH;   // horizontal blur of every level-l row
    float(*Rh)[kPyr2MW] = Lh + kPyr2SH;
    const int pi = find_pair(a.descs, a.npairs, unit, W_PYR);
    const LevelDesc &D = a.descs[pi];     // level l
    const LevelDesc &E = a.descs2[pi];    // level l+1 (its Ln, Rn: level l+2)
    const int tile = unit - D.work_begin[W_PYR];
    const int ntx = (D.w + kPyrTW - 1) / kPyrTW;
    const int ty = udiv_small(tile, recip(ntx)), tx = tile - ty * ntx;
    const int x0 = tx * kPyrTW - 6, y0 = ty * kPyrTH - 6;  // level-l region origin
    const int X0 = tx * (kPyrTW / 2) - 2, Y0 = ty * (kPyrTH / 2) - 2;  // level-(l+1) region origin
    const int w = D.w, h = D.h, pitch = D.pitch;
    const int w1 = E.w, h1 = E.h;
    const TI *L = (const TI *)D.L;
    const TI *R = (const TI *)D.R;
    __syncthreads();
    constexpr int NEL = kPyr2SH * kPyr2SW;
    constexpr int PER = (NEL + 255) / 256;
    float vl[PER], vr[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x + k * 256;
        if (i < NEL) {
            const int r = i / kPyr2SW, c = i - r * kPyr2SW;
            const int gy = refl(min(max(y0 + r, -2), h + 1), h);
            const int gx = refl(min(max(x0 + c, -2), w + 1), w);
            vl[k] = ldf(L + (size_t)gy * pitch + gx);
            vr[k] = ldf(R + (size_t)gy * pitch + gx);
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x + k * 256;
        if (i < NEL) {
            const int r = i / kPyr2SW, c = i - r * kPyr2SW;
            Ls[r][c] = vl[k];
            Rs[r][c] = vr[k];
        }
    }
    __syncthreads();
    // Sobel-x/8 of level l over the 64x32 tile
    TG *G = (TG *)D.G;
    for (int i = threadIdx.x; G != nullptr && i < kPyrTW * kPyrTH; i += blockDim.x) {
        const int ly = i / kPyrTW, lx = i - ly * kPyrTW;
        const int x = x0 + 6 + lx, y = y0 + 6 + ly;
        if (x >= w || y >= h) continue;
        const int cx = lx + 6, cy = ly + 6;
        const float acc = (Ls[cy - 1][cx + 1] - Ls[cy - 1][cx - 1]) +
                          2.f * (Ls[cy][cx + 1] - Ls[cy][cx - 1]) +
                          (Ls[cy + 1][cx + 1] - Ls[cy + 1][cx - 1]);
        stf(G + (size_t)y * D.gpitch + x, acc * 0.125f);
    }
    // level l+1 over the tile and its 2-pixel halo (halo pixels take their
    // reflect-101 image pixel): horizontal pass at the needed even columns,
    // then vertical pass; the same multiply-add order as the one-step kernel
    const float k5[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
    for (int i = threadIdx.x; i < kPyr2SH * kPyr2MW; i += blockDim.x) {
        const int r = i / kPyr2MW, mx = i - r * kPyr2MW;
        const int Xr = refl(min(max(X0 + mx, -2), w1 + 1), w1);
        const int cx = 2 * Xr - x0;
        float sl = 0.f, sr = 0.f;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            sl += k5[q] * Ls[r][cx + q - 2];
            sr += k5[q] * Rs[r][cx + q - 2];
        }
        Lh[r][mx] = sl;
        Rh[r][mx] = sr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPyr2MW * kPyr2MH; i += blockDim.x) {
        const int my = i / kPyr2MW, mx = i - my * kPyr2MW;
        const int X = X0 + mx, Y = Y0 + my;
        const int Yr = refl(min(max(Y, -2), h1 + 1), h1);
        const int cy = 2 * Yr - y0;
        float accL = 0.f, accR = 0.f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            accL += k5[j] * Lh[cy + j - 2][mx];
            accR += k5[j] * Rh[cy + j - 2][mx];
        }
        const float vL = accL * (1.f / 256.f), vR = accR * (1.f / 256.f);
        Lm[my][mx] = round_to<TN>(vL);
        Rm[my][mx] = round_to<TN>(vR);
        const bool own = mx >= 2 && mx < 2 + kPyrTW / 2 && my >= 2 && my < 2 + kPyrTH / 2;
        if (own && X < w1 && Y < h1) {
            stf((TN *)D.Ln + (size_t)Y * D.pitchn + X, vL);
            stf((TN *)D.Rn + (size_t)Y * D.pitchn + X, vR);
        }
    }
    __syncthreads();
    // Sobel-x/8 of level l+1 over its 32x16 tile
    TG *G1 = (TG *)E.G;
    for (int i = threadIdx.x; G1 != nullptr && i < (kPyrTW / 2) * (kPyrTH / 2); i += blockDim.x) {
        const int ly = i / (kPyrTW / 2), lx = i - ly * (kPyrTW / 2);
        const int X = X0 + 2 + lx, Y = Y0 + 2 + ly;
        if (X >= w1 || Y >= h1) continue;
        const int cx = lx + 2, cy = ly + 2;
        const float acc = (Lm[cy - 1][cx + 1] - Lm[cy - 1][cx - 1]) +
                          2.f * (Lm[cy][cx + 1] - Lm[cy][cx - 1]) +
                          (Lm[cy + 1][cx + 1] - Lm[cy + 1][cx - 1]);
        stf(G1 + (size_t)Y * E.gpitch + X, acc * 0.125f);
    }
    // level l+2 over its 16x8 tile
    for (int i = threadIdx.x; i < (kPyrTW / 4) * (kPyrTH / 4); i += blockDim.x) {
        const int oy = i / (kPyrTW / 4), ox = i - oy * (kPyrTW / 4);
        const int X = tx * (kPyrTW / 4) + ox, Y = ty * (kPyrTH / 4) + oy;
        if (X >= E.wn || Y >= E.hn) continue;
        const int cx = 2 * ox + 2, cy = 2 * oy + 2;
        float accL = 0.f, accR = 0.f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float sl = 0.f, sr = 0.f;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                sl += k5[q] * Lm[cy + j - 2][cx + q - 2];
                sr += k5[q] * Rm[cy + j - 2][cx + q - 2];
            }
            accL += k5[j] * sl;
            accR += k5[j] * sr;
        }
        stf((TN *)E.Ln + (size_t)Y * E.pitchn + X, accL * (1.f / 256.f));
        stf((TN *)E.Rn + (size_t)Y * E.pitchn + X, accR * (1.f / 256.f));
    }
}

template <typename TI, typename TN, typename TG>
__global__ void __launch_bounds__(256) k_pyramid2(LaunchArgs a) {
    __shared__ float sm[kPyr2SmemFloats];
    pdl_enter(a);
    if (blockIdx.x == 0 && a.acc_zero != nullptr)
        for (int i = threadIdx.x; i < a.acc_count; i += blockDim.x) a.acc_zero[i] = 0ull;
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) pyramid2_unit<TI, TN, TG>(a, unit, sm);
    pdl_leave(a);
}

template <typename TI, typename TN, typename TG>
__global__ void __launch_bounds__(256, 4) k_pyramid(LaunchArgs a) {
    __shared__ __align__(16) float Ls[kPyrSH][kPyrSP];
    __shared__ __align__(16) float Rs[kPyrSH][kPyrSP];
    __shared__ __align__(16) float Lh[kPyrSH][kPyrHP];
    __shared__ __align__(16) float Rh[kPyrSH][kPyrHP];
    pdl_enter(a);
    // the finest pyramid launch runs before every search: it clears the
    // sigma_r accumulators of all levels and pairs
    if (blockIdx.x == 0 && a.acc_zero != nullptr)
        for (int i = threadIdx.x; i < a.acc_count; i += blockDim.x) a.acc_zero[i] = 0ull;
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x)
        pyramid_unit<TI, TN, TG>(a, unit, Ls, Rs, Lh, Rh);
    pdl_leave(a);
}

// One-step pyramid with the staging of interior tiles by bulk asynchronous
// copies.  Each row of a tile's region is one cp.async.bulk of the storage
// type's raw bytes, from the region's first column rounded down to a 16-byte
// boundary (RAW_OFF elements before it) over RAW_SPAN_E elements, so both
// ends are 16-byte aligned; the copies of a tile complete on one mbarrier.
// A block walks its units with two raw buffers: the copies of the next unit
// are in flight while the current unit is widened to FP32 and computed.  A
// unit whose region is not inside the image (or whose rows do not allow the
// alignment) is staged by the block's own loads (pyramid_stage_loads).  The
// staged values, and so the results, are those of the one-step kernel.
template <typename TI>
struct PyrBulk {
    static constexpr int E = (int)sizeof(TI);
    static constexpr int A = 16 / E;                                   // elements per 16 bytes
    static constexpr int RAW_OFF = (kPyrOX + A - 1) / A * A - kPyrOX;  // region start in the raw row
    static constexpr int RAW_SPAN_E = (RAW_OFF + kPyrSW + A - 1) / A * A;
    static constexpr int RAW_SPAN_B = RAW_SPAN_E * E;                  // bytes per copied row
    static constexpr size_t kSmem = (size_t)2 * 2 * kPyrSH * RAW_SPAN_B;  // 2 buffers x (L, R)
};
static_assert(PyrBulk<uint8_t>::RAW_SPAN_B % 16 == 0 && PyrBulk<__half>::RAW_SPAN_B % 16 == 0 &&
                  PyrBulk<float>::RAW_SPAN_B % 16 == 0 && kPyrTW % 16 == 0,
              "bulk rows and tile columns on 16-byte boundaries");

// Polls of one wait for a tile's copies (a poll is a barrier test and a 32 ns
// sleep); past it the kernel records the failure and stops.
constexpr unsigned kCopyWaitLimit = 1u << 22;
__device__ __forceinline__ unsigned copy_limit(const LaunchArgs &a) {
    return a.copy_limit != 0u ? a.copy_limit : kCopyWaitLimit;
}
// bytes a wait expects beyond those its copies deliver (the test switch)
__device__ __forceinline__ unsigned copy_extra(const LaunchArgs &a) { return a.copy_test ? 16u : 0u; }

// Four raw elements at p (4-, 8- or 16-byte aligned) as floats.
__device__ __forceinline__ float4 raw4(const uint8_t *p) {
    const uchar4 u = *(const uchar4 *)p;
    return make_float4((float)u.x, (float)u.y, (float)u.z, (float)u.w);
}
__device__ __forceinline__ float4 raw4(const __half *p) {
    const uint2 u = *(const uint2 *)p;
    const float2 a = __half22float2(*(const __half2 *)&u.x);
    const float2 b = __half22float2(*(const __half2 *)&u.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 raw4(const float *p) { return *(const float4 *)p; }

template <typename TI, typename TN, typename TG>
__global__ void __launch_bounds__(256, 4) k_pyramid_bulk(LaunchArgs a) {
    using PB = PyrBulk<TI>;
    __shared__ __align__(16) float Ls[kPyrSH][kPyrSP];
    __shared__ __align__(16) float Rs[kPyrSH][kPyrSP];
    __shared__ __align__(16) float Lh[kPyrSH][kPyrHP];
    __shared__ __align__(16) float Rh[kPyrSH][kPyrHP];
    __shared__ __align__(8) uint64_t bar[2];
    extern __shared__ __align__(16) unsigned char raw[];  // [buffer][image][row][RAW_SPAN_B]
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    pdl_enter(a);
    if (blockIdx.x == 0 && a.acc_zero != nullptr)
        for (int i = tid; i < a.acc_count; i += blockDim.x) a.acc_zero[i] = 0ull;

    struct Tile {
        const LevelDesc *D;
        int tx, ty;
        bool bulk;
    };
    auto tile_of = [&](int unit) {
        Tile t;
        t.D = &a.descs[find_pair(a.descs, a.npairs, unit, W_PYR)];
        const LevelDesc &D = *t.D;
        const int tile = unit - D.work_begin[W_PYR];
        const int ntx = (D.w + kPyrTW - 1) / kPyrTW;
        t.ty = udiv_small(tile, recip(ntx));
        t.tx = tile - t.ty * ntx;
        const int xs = t.tx * kPyrTW - kPyrOX, y0 = t.ty * kPyrTH - 2;
        const int xr = xs - PB::RAW_OFF;
        const bool next = D.Ln != nullptr;
        const uintptr_t base = (uintptr_t)D.L | (next ? (uintptr_t)D.R : (uintptr_t)0);
        // region inside the image, copied span inside the row, 16-byte rows
        t.bulk = xr >= 0 && xs + kPyrSW <= D.w && xr + PB::RAW_SPAN_E <= D.pitch && y0 >= 0 &&
                 y0 + kPyrSH <= D.h && (base & 15u) == 0 && ((size_t)D.pitch * PB::E) % 16 == 0;
        return t;
    };
    // the copies of one tile into raw buffer b (block-uniform decision)
    auto issue = [&](const Tile &t, int b) {
        const LevelDesc &D = *t.D;
        const bool next = D.Ln != nullptr;
        const int nrows = next ? 2 * kPyrSH : kPyrSH;
        if (tid < nrows) {
            fence_proxy_async_smem();  // earlier reads of this buffer precede the copy
            if (tid == 0) mbar_arrive_expect_tx(&bar[b], (unsigned)(nrows * PB::RAW_SPAN_B) + copy_extra(a));
            const int img = tid / kPyrSH, r = tid - img * kPyrSH;
            const int xr = t.tx * kPyrTW - kPyrOX - PB::RAW_OFF, y = t.ty * kPyrTH - 2 + r;
            const TI *src = (const TI *)(img ? D.R : D.L) + (size_t)y * D.pitch + xr;
            unsigned char *dst = raw + ((size_t)(b * 2 + img) * kPyrSH + r) * PB::RAW_SPAN_B;
            bulk_copy_g2s(dst, src, (unsigned)PB::RAW_SPAN_B, &bar[b]);
        }
    };

    unsigned parity = 0u;  // bit b: parity of raw buffer b's next phase
    int unit = blockIdx.x;
    Tile cur;
    if (unit < a.total) {
        cur = tile_of(unit);
        if (cur.bulk) issue(cur, 0);
    }
    for (int i = 0; unit < a.total; ++i, unit += gridDim.x) {
        const int b = i & 1;
        // the next unit's copies go into the other buffer, whose last reads
        // (widening, iteration i - 1) finished before that iteration's barrier
        const int un = unit + gridDim.x;
        Tile nxt;
        nxt.bulk = false;
        if (un < a.total) {
            nxt = tile_of(un);
            if (nxt.bulk) issue(nxt, b ^ 1);
        }
        __syncthreads();  // the previous unit's readers are done with Ls, Rs
        if (cur.bulk) {
            const bool ok = mbar_wait_bounded(&bar[b], (parity >> b) & 1u, copy_limit(a));
            parity ^= 1u << b;
            if (__syncthreads_or(!ok)) {
                // a copy did not land: report it, wait (bounded) for the
                // copies still in flight and stop
                if (tid == 0 && a.err_host != nullptr) {
                    *(volatile int *)a.err_host = 1;
                    __threadfence_system();
                }
                if (nxt.bulk) mbar_wait_bounded(&bar[b ^ 1], (parity >> (b ^ 1)) & 1u, copy_limit(a));
                return;
            }
            // widen the raw rows to FP32 (exact for u8, f16, f32)
            const LevelDesc &D = *cur.D;
            const int nimg = D.Ln != nullptr ? 2 : 1;
            constexpr int QPR = kPyrSW / 4;  // four-element groups per row
            for (int q = tid; q < nimg * kPyrSH * QPR; q += blockDim.x) {
                const int img = q / (kPyrSH * QPR), rem = q - img * (kPyrSH * QPR);
                const int r = rem / QPR, c = 4 * (rem - r * QPR);
                const TI *src = (const TI *)(raw + ((size_t)(b * 2 + img) * kPyrSH + r) * PB::RAW_SPAN_B) +
                                PB::RAW_OFF + c;
                *(float4 *)&(img ? Rs : Ls)[r][c] = raw4(src);
            }
        } else {
            pyramid_stage_loads<TI>(*cur.D, cur.tx, cur.ty, Ls, Rs);
        }
        __syncthreads();
        pyramid_compute<TN, TG>(*cur.D, cur.tx, cur.ty, Ls, Rs, Lh, Rh);
        cur = nxt;
    }
    pdl_leave(a);
}

// ---------------------------------------------------------------- patch search

// Raw row pitch in bytes of the search's bulk band staging for element size
// esz: the band capacity rounded up to 16 bytes, plus 16.
__host__ __device__ __forceinline__ size_t search_raw_pitch(int band_cap, int esz) {
    return ((size_t)band_cap * esz + 15) / 16 * 16 + 16;
}

// The mbarrier of the bulk band staging: at the first 16-byte boundary past
// the right band, the left and gradient bands, the chunk's estimates and
// sigma_r terms and the reduction scratch (the layout of search_unit); the
// raw rows follow 16 bytes later.
__device__ __forceinline__ uint64_t *search_bulk_bar(float *smem, int P, int bp, int cp, int chunk) {
    const size_t off = sizeof(float) * ((size_t)P * bp + 2 * (size_t)P * cp + 4 * (size_t)chunk + 16);
    return (uint64_t *)((char *)smem + (off + 15) / 16 * 16);
}

// Block-wide min and max (all threads get the result).
__device__ __forceinline__ void block_minmax(float &lo, float &hi, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[wid] = lo;
        red[8 + wid] = hi;
    }
    __syncthreads();
    lo = red[0];
    hi = red[8];
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        lo = fminf(lo, red[i]);
        hi = fmaxf(hi, red[8 + i]);
    }
    __syncthreads();
}

// A block owns one chunk of consecutive patches of one patch row.  It stages
// in shared memory the left image and gradient over the chunk's columns and
// the right image over the column window that the chunk's estimates can
// reach: [cx0 - max d_init - margin, cx0 + cw - min d_init + margin], each
// shared column holding the image column clamped to [0, w-1], so the inner
// loops read with immediate offsets and no clamping.  A patch whose estimate
// leaves the window reads the image directly (same clamped values).  A group
// of G lanes handles one patch, lane r owning patch row r; reductions are
// xor shuffles inside the group; the iteration count is fixed, so every lane
// of a warp executes the same instruction stream.  The groups of a warp take
// patches spaced so that their rows fall in different shared-memory banks.
// With BULK and bit 2 of a.bulk, a band window inside the image is instead
// copied row by row by cp.async.bulk into a raw area behind the band
// (search_layout), then widened to FP32 in shared memory; the values staged,
// and so the results, are the same.  Returns false if the wait for those
// copies ran out (reported through a.err_host; the block stops).
template <int P, typename TI, typename TG, bool BULK>
__device__ __forceinline__ bool search_unit(const LaunchArgs &a, int unit, float *smem,
                                            unsigned &bphase) {

    constexpr int G = P <= 8 ? 8 : 16;
    constexpr int N = P * P;
    constexpr int GPW = 32 / G;  // groups per warp
    constexpr float invN = 1.f / (float)N;
    const int bp = a.band_pitch, cp = a.chunk_pitch, cap = a.band_cap;
    float *Rb = smem;
    float *Lb = Rb + P * bp;
    float *Gb = Lb + P * cp;
    float *dsh = Gb + P * cp;            // chunk d_init
    float *pe = dsh + a.chunk;           // chunk sigma_r terms: E(0), count, E(0)^2
    float *red = pe + 3 * a.chunk;       // 16 floats
    const int tid = threadIdx.x;
    const int gl = tid & (G - 1);
    const int q = (tid & 31) / G;
    const int warp = tid >> 5;
    const bool row_on = gl < P;
    const int S = a.S;
    const float h = a.window_step;
    const float dl[4] = {-h, h, -2.f * h, 2.f * h};
    // patch spacing between the groups of a warp (a power of two dividing 16)
    int sp = (32 / GPW) / S;
    sp = sp >= 16 ? 16 : sp >= 8 ? 8 : sp >= 4 ? 4 : sp >= 2 ? 2 : 1;
    // must divide the chunk's 8 x passes warp slots
    for (const int ns = 8 * (a.chunk / (8 * GPW)); ns % sp != 0;) sp >>= 1;
    const int margin = (int)ceilf(a.tau) + (int)ceilf(2.f * h) + 3;


    const LevelDesc &D = a.descs[find_pair(a.descs, a.npairs, unit, W_SEARCH)];
    const int u = unit - D.work_begin[W_SEARCH];
    const int py = udiv_small(u, recip(D.nchunks)), ch = u - py * D.nchunks;
    const int oy = origin(py, D.h, P, S, D.kyreg);
    const int k0 = ch * a.chunk;
    const int k1 = min(k0 + a.chunk, D.npx);
    const int nk = k1 - k0;
    const int cx0 = origin(k0, D.w, P, S, D.kxreg);
    const int cw = origin(k1 - 1, D.w, P, S, D.kxreg) + P - cx0;
    const int w = D.w;
    const TI *R = (const TI *)D.R;
    const TI *L = (const TI *)D.L;
    const TG *Gi = (const TG *)D.G;

    __syncthreads();  // the previous unit's readers are done with smem
    // the left-image and gradient bands do not depend on the estimates: the
    // first column's loads are issued before the initial estimates are read.
    // Only where the register budget has room (P > 8 runs 2 blocks per SM;
    // the 3-block instances would spill).
    constexpr bool kEarlyLG = P > 8;
    float vl0[P], vg0[P];
    const bool col0 = kEarlyLG && tid < cw;
    if (col0) {
#pragma unroll
        for (int r = 0; r < P; ++r) {
            vl0[r] = ldf(L + (size_t)(oy + r) * D.pitch + cx0 + tid);
            vg0[r] = ldf(Gi + (size_t)(oy + r) * D.gpitch + cx0 + tid);
        }
    }
    // initial estimates of the chunk (coarser fused map at the centre)
    float dlo = FLT_MAX, dhi = -FLT_MAX;
    for (int t = tid; t < nk; t += blockDim.x) {
        float di = 0.f;
        if (D.Dc != nullptr) {
            const float cxp = (float)origin(k0 + t, w, P, S, D.kxreg) + 0.5f * (float)(P - 1);
            const float cyp = (float)oy + 0.5f * (float)(P - 1);
            di = 2.f * coarse_bilin(D.Dc, D.wc, D.hc, cxp, cyp);
        }
        dsh[t] = di;
        dlo = fminf(dlo, di);
        dhi = fmaxf(dhi, di);
    }
    if (col0) {
#pragma unroll
        for (int r = 0; r < P; ++r) {
            Lb[r * cp + tid] = vl0[r];
            Gb[r * cp + tid] = vg0[r];
        }
    }
    block_minmax(dlo, dhi, red);
    // column window of the right band
    dhi = fminf(fmaxf(dhi, -(float)(2 * w)), (float)(2 * w));
    dlo = fminf(fmaxf(dlo, -(float)(2 * w)), (float)(2 * w));
    int xlo = cx0 - (int)ceilf(dhi) - margin;
    const int xhi = cx0 + cw - (int)floorf(dlo) + margin;
    int wwin = min(xhi - xlo, cap);
    // bulk staging of the right band (block-uniform decision): the window
    // starts at a 16-byte boundary at or left of xlo and lies inside the
    // image (no clamping), the copied span (the window rounded up to 16
    // bytes) inside the image row, rows 16-byte aligned
    constexpr int kE = (int)sizeof(TI), kA = 16 / kE;
    bool bulk_band = false;
    unsigned char *raw = nullptr;
    uint64_t *bbar = nullptr;
    if (BULK && (a.bulk & 2) != 0) {
        const int xa = xlo >= 0 ? xlo / kA * kA : -1;
        const int wb = min(xhi - xa, cap);
        const int span = (wb + kA - 1) / kA * kA;
        if (xa >= 0 && xhi <= w && xa + span <= w && ((uintptr_t)R & 15u) == 0 &&
            ((size_t)D.pitch * kE) % 16 == 0) {
            bulk_band = true;
            xlo = xa;
            wwin = wb;
            bbar = search_bulk_bar(smem, P, bp, cp, a.chunk);
            raw = (unsigned char *)(bbar + 2);
            if (tid < P) {
                fence_proxy_async_smem();  // the last unit's widening reads precede the copy
                if (tid == 0) mbar_arrive_expect_tx(bbar, (unsigned)(P * span * kE) + copy_extra(a));
                bulk_copy_g2s(raw + (size_t)tid * search_raw_pitch(cap, kE),
                              R + (size_t)(oy + tid) * D.pitch + xa, (unsigned)(span * kE), bbar);
            }
        }
    }
    // staging: the P rows of a column are loaded together (memory-level parallelism)
    for (int c = bulk_band ? wwin : tid; c < wwin; c += blockDim.x) {
        const int col = clampi(xlo + c, 0, w - 1);
        float v[P];
#pragma unroll
        for (int r = 0; r < P; ++r) v[r] = ldf(R + (size_t)(oy + r) * D.pitch + col);
#pragma unroll
        for (int r = 0; r < P; ++r) Rb[r * bp + c] = v[r];
    }
    // four columns per step where the rows allow aligned vector loads
    // (P <= 8: no early column; block-uniform decision)
    int c_first = kEarlyLG ? tid + blockDim.x : tid;
    if (!kEarlyLG && (cx0 & 3) == 0 && (D.pitch & 3) == 0 && (D.gpitch & 3) == 0 &&
        (((uintptr_t)L | (uintptr_t)Gi) & 15u) == 0) {
        const int nq = cw >> 2;
        for (int q = tid; q < nq; q += blockDim.x) {
            const int c = 4 * q;
            float4 v[P];
#pragma unroll
            for (int r = 0; r < P; ++r) v[r] = raw4(L + (size_t)(oy + r) * D.pitch + cx0 + c);
#pragma unroll
            for (int r = 0; r < P; ++r) {
                float *d = Lb + r * cp + c;
                d[0] = v[r].x; d[1] = v[r].y; d[2] = v[r].z; d[3] = v[r].w;
            }
#pragma unroll
            for (int r = 0; r < P; ++r) v[r] = raw4(Gi + (size_t)(oy + r) * D.gpitch + cx0 + c);
#pragma unroll
            for (int r = 0; r < P; ++r) {
                float *d = Gb + r * cp + c;
                d[0] = v[r].x; d[1] = v[r].y; d[2] = v[r].z; d[3] = v[r].w;
            }
        }
        c_first = 4 * nq + tid;
    }
    for (int c = c_first; c < cw; c += blockDim.x) {
        float vl[P], vg[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            vl[r] = ldf(L + (size_t)(oy + r) * D.pitch + cx0 + c);
            vg[r] = ldf(Gi + (size_t)(oy + r) * D.gpitch + cx0 + c);
        }
#pragma unroll
        for (int r = 0; r < P; ++r) {
            Lb[r * cp + c] = vl[r];
            Gb[r * cp + c] = vg[r];
        }
    }
    if (bulk_band) {
        const unsigned par = bphase & 1u;
        const bool ok = mbar_wait_bounded(bbar, par, copy_limit(a));
        bphase ^= 1u;
        if (__syncthreads_or(!ok)) {
            // the copies did not land: report it, wait (bounded) once more
            // for them to finish writing shared memory, and stop
            if (tid == 0 && a.err_host != nullptr) {
                *(volatile int *)a.err_host = 1;
                __threadfence_system();
            }
            mbar_wait_bounded(bbar, par, copy_limit(a));
            return false;
        }
        // widen to FP32: four raw elements per step (the copied span covers
        // the window rounded up to four), stored up to the window's end
        const int ng = (wwin + 3) >> 2;
        const size_t rpb = search_raw_pitch(cap, kE);
        const float rng = recip(ng);
        for (int i = tid; i < P * ng; i += blockDim.x) {
            const int r = udiv_small(i, rng), g = i - r * ng, c = 4 * g;
            const float4 f = raw4((const TI *)(raw + (size_t)r * rpb) + c);
            float *dst = Rb + r * bp + c;
            dst[0] = f.x;
            if (c + 1 < wwin) dst[1] = f.y;
            if (c + 2 < wwin) dst[2] = f.z;
            if (c + 3 < wwin) dst[3] = f.w;
        }
    }
    __syncthreads();

    const int passes = a.chunk / (8 * GPW);
    for (int pass = 0; pass < passes; ++pass) {
        // the slot of warp u, group q is (u / sp) sp GPW + u % sp + sp q,
        // increasing in u for q = 0, so the pass's smallest slot is that of
        // its first warp's first group; once it is past the chunk's last
        // patch, so is every slot of this pass and the later ones
        // (block-uniform).  With sp > 8 a pass's slots are not contiguous.
        if (((pass * 8) / sp) * (sp * GPW) + (pass * 8) % sp >= nk) break;
        const int uu = pass * 8 + warp;
        const int kk = (uu / sp) * (sp * GPW) + (uu % sp) + sp * q;  // patch slot in chunk
        const bool active = kk < nk;
        const int kl = min(kk, nk - 1);
        const int kx = k0 + kl;
        const int ox = origin(kx, w, P, S, D.kxreg);
        const int rr = row_on ? gl : 0;
        const float *Lrow = Lb + rr * cp + (ox - cx0);
        const float *Grow = Gb + rr * cp + (ox - cx0);
        const float *Rs = Rb + rr * bp;
        const TI *Rg = R + (size_t)(oy + rr) * D.pitch;

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
        float hp = 0.f, cpart = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            gt[j] = row_on ? gt[j] - gbar : 0.f;
            hp = fmaf(gt[j], gt[j], hp);
            cpart = fmaf(gt[j], T[j], cpart);
        }
        const float H = group_sum<G>(hp);
        const float cT = group_sum<G>(cpart);
        const bool flat = !(H >= a.hess_eps * (float)N);
        const float invH = flat ? 0.f : 1.f / H;
        const float dinit = dsh[kl];
        const float dlim = (float)w + 2.f * (float)P;

        // right-image values of this lane's row at columns base .. base + NV - 1
        // (staged band, else the image with the same clamping)
        auto load_vals = [&](int base, auto &v) {
            constexpr int NV = sizeof(v) / sizeof(float);
            const int o = base - xlo;
            if (o >= 0 && o + NV <= wwin) {
                const float *p = Rs + o;
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = p[j];
            } else {
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = ldf(Rg + clampi(base + j, 0, w - 1));
            }
        };

        // Gauss-Newton: d <- d + (sum gt_i s_i - cT) / H, s_i = I_r(x_i - d).
        // With x - d = base + j + t the sum is A + t (B - A), A and B the
        // correlations of gt with the row at integer offsets base and base + 1;
        // they change only when d crosses an integer, so the warp recomputes
        // them only when one of its patches did.
        float d = dinit, dlast = 0.f;
        int offc = INT_MIN;
        float At = 0.f, Bt = 0.f;
        for (int it = 0; it < a.iters; ++it) {
            int off;
            float t;
            split_shift(d, off, t);
            if (__any_sync(0xffffffffu, off != offc)) {
                float v[P + 1];
                load_vals(ox + off, v);
                float A = 0.f, B = 0.f;
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    A = fmaf(gt[j], v[j], A);
                    B = fmaf(gt[j], v[j + 1], B);
                }
                At = group_sum<G>(A);
                Bt = group_sum<G>(B);
                offc = off;
            }
            const float s = fmaf(t, Bt - At, At);
            if (!flat) {
                const float delta = (s - cT) * invH;
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
        // samples of the window offsets {-h, +h, -2h, +2h}: sw[k][j]
        // (general h: one split per offset; h = 1/2: the +-2h samples are the
        // centre samples one column over and -h is +h one column over, so two
        // interpolated rows cover all five)
        float su[4], suu[4];
        float sa = 0.f;
        const bool half = h == 0.5f;
        // S0: columns -1 .. P at d (the centre samples are S0[1 .. P]);
        // Sp (h = 1/2 only): columns 0 .. P at d + 1/2
        float S0[P + 2], Sp[P + 1];
        float v0[P + 3];
        load_vals(base0 - 1, v0);
#pragma unroll
        for (int j = 0; j < P + 2; ++j) S0[j] = fmaf(t0, v0[j + 1] - v0[j], v0[j]);
        if (half) {
            // the columns of d + 1/2 start at base0 or base0 - 1 (the half
            // pixel moves the split by at most one column), both held in v0
            int offp;
            float tp;
            split_shift(d + 0.5f, offp, tp);
            const bool same = offp == off0;
#pragma unroll
            for (int j = 0; j < P + 1; ++j) {
                const float a0 = same ? v0[j + 1] : v0[j];
                const float a1 = same ? v0[j + 2] : v0[j + 1];
                Sp[j] = fmaf(tp, a1 - a0, a0);
            }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) sa += row_on ? S0[j + 1] - T[j] : 0.f;
        // samples outside [0, w-1]: every row shares base0 and t0, so per
        // row j < -base0 on the left and base0 + j >= w - 1 (t0 > 0) or
        // >= w (t0 = 0) on the right
        const int nl = min(max(-base0, 0), P);
        const int nr = min(max(P + base0 - (t0 > 0.f ? w - 1 : w), 0), P);
        const int nout_all = P * (nl + nr);
        const float mean0 = group_sum<G>(sa) * invN;
        float e0 = 0.f;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            T[j] = row_on ? (S0[j + 1] - T[j]) - mean0 : 0.f;  // now the centred residual
            e0 = fmaf(T[j], T[j], e0);
        }
        // window energies.  E(0) in two passes; for the four offsets the
        // differences dE_k = E(delta_k) - E(0) directly from the sample
        // differences u_j = s_kj - s_0j (the template cancels):
        //   dE_k = sum u^2 - (sum u)^2 / N + 2 sum u (a_0j - mean a_0)
        //        = sum u (u + 2 c_j) - (sum u)^2 / N,  c_j the centred residual,
        // which keeps full relative precision when dE_k << E(0); two group
        // sums per offset.
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float sk[P];
            if (half) {
#pragma unroll
                for (int j = 0; j < P; ++j)
                    sk[j] = k == 0 ? Sp[j + 1] : k == 1 ? Sp[j] : k == 2 ? S0[j + 2] : S0[j];
            } else {
                int off;
                float t;
                split_shift(d + dl[k], off, t);
                float v[P + 1];
                load_vals(ox + off, v);
#pragma unroll
                for (int j = 0; j < P; ++j) sk[j] = fmaf(t, v[j + 1] - v[j], v[j]);
            }
            float p1 = 0.f, p2 = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const float uj = row_on ? sk[j] - S0[j + 1] : 0.f;
                p1 += uj;
                p2 = fmaf(uj, fmaf(2.f, T[j], uj), p2);
            }
            su[k] = p1;
            suu[k] = p2;
        }
        float E[5];  // E[0] = E(0); E[k] = E(delta_k) - E(0)
        E[0] = group_sum<G>(e0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float S1 = group_sum<G>(su[k]);
            const float S2 = group_sum<G>(suu[k]);
            E[k + 1] = fmaf(-S1 * invN, S1, S2);
        }

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
            // the 64-byte record as four 16-byte stores (layout of bdis_patch_record:
            // d dinit dlast H | E0..E3 | E4 cT flags nout+pdf_flags | pi rho sig2 mu)
            static_assert(sizeof(bdis_patch_record) == 64, "record layout");
            float4 *rp = (float4 *)(D.rec + (size_t)py * D.npx + kx);
            rp[0] = make_float4(d, dinit, dlast, H);
            rp[1] = make_float4(E[0], E[1], E[2], E[3]);
            rp[2] = make_float4(E[4], cT, __uint_as_float(f), __uint_as_float((uint32_t)nout_all & 0xffffu));
            rp[3] = make_float4(0.f, 0.f, 0.f, mean0);
            const bool kept = f == 0u;
            pe[3 * kk] = kept ? E[0] : 0.f;
            pe[3 * kk + 1] = kept ? 1.f : 0.f;
            pe[3 * kk + 2] = kept ? E[0] * E[0] : 0.f;
        }
    }
    __syncthreads();
    // sigma_r sums of the chunk in 64-bit fixed point: integer addition is
    // exactly associative, so the totals do not depend on the chunking or
    // on the order in which blocks add them
    if (warp == 0) {
        unsigned long long s1 = 0ull, s2 = 0ull, s3 = 0ull;
        for (int i = tid; i < nk; i += 32) {
            s1 += (unsigned long long)__float2ll_rn(pe[3 * i] * kSigmaFix1);
            s2 += (unsigned long long)pe[3 * i + 1];
            s3 += (unsigned long long)__float2ll_rn(pe[3 * i + 2]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        }
        if (tid == 0) {
            atomicAdd(D.acc, s1);
            atomicAdd(D.acc + 1, s2);
            atomicAdd(D.acc + 2, s3);
        }
    }
    return true;
}

// BULK: the instance with the bulk band staging (BDIS_OPT_BULK_COPY bit 2;
// compiled for P = 8 and 12), a kernel of its own so that the default
// instances keep their register allocation.
template <int P, typename TI, typename TG, bool BULK>
__global__ void __launch_bounds__(256, (P <= 8 ? 3 : 2)) k_search(LaunchArgs a) {
    extern __shared__ __align__(16) float smem[];
    if (BULK && (a.bulk & 2) != 0 && threadIdx.x == 0) {
        mbar_init(search_bulk_bar(smem, P, a.band_pitch, a.chunk_pitch, a.chunk), 1);
        mbar_init_fence();
    }
    // (the unit's first barrier orders the initialisation before any use)
    pdl_enter(a);
    unsigned bphase = 0u;
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x)
        if (!search_unit<P, TI, TG, BULK>(a, unit, smem, bphase)) break;
    pdl_leave(a);
}

// ---------------------------------------------------------------- posterior, fusion

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
    // one reciprocal of sigma per step (the other quotients are products
    // with it and with 1 / sum q^2), and ln sigma^2 = 2 ln sigma: a shorter
    // dependent chain for the same step
    const float iqq = 1.f / qq;
    float sg = sqrtf(0.1f), c = 1.f;
    for (int it = 0; it < iters; ++it) {
        const float isg = 1.f / sg;
        const float lc = logf(c), ls = 2.f * logf(sg);
        const float inv2s2 = 0.5f * isg * isg;
        float rbar = 0.f, qr = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float r = (lc - 0.5f * (ln2pi + ls) - d2[i] * inv2s2) - lnp[i];
            rbar += r;
            qr = fmaf(d2[i] - mu, r, qr);
        }
        rbar *= 0.2f;
        const float a = -isg, b = isg * isg * isg;
        float ds = -qr * iqq * (sg * sg * sg);  // -qr / (b qq)
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
        const float isg = 1.f / sg;
        const float lc = logf(c), ls = 2.f * logf(sg);
        const float inv2s2 = 0.5f * isg * isg;
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

// A pixel of an image whose element type is known only at run time.
__device__ __forceinline__ float ld_typed(const void *p, size_t i, int t) {
    if (t == E_U8) return (float)__ldg((const uint8_t *)p + i);
    if (t == E_F16) return __half2float(__ldg((const __half *)p + i));
    return __ldg((const float *)p + i);
}

// Schraudolph's exponential (Neural Computation 11(4), 1999) in single
// precision: the bits of the binary32 result are the integer
// A y + (B - C), A = 2^23 / ln 2, B = 127 * 2^23, C = 8 * 60801 (the paper's
// RMS-optimal correction moved to the 23-bit fraction), truncated.  Within
// about 4 % of exp(y); 0 below y = -87.
__device__ __forceinline__ float exp_schraudolph(float y) {
    if (y < -87.f) return 0.f;
    y = fminf(y, 88.f);
    const float A = 12102203.161561485f;        // 2^23 / ln 2
    const float BC = 1065353216.f - 486408.f;   // 127 * 2^23 - 8 * 60801
    return __int_as_float((int)floorf(fmaf(A, y, BC)));
}

// One thread per patch of a tile's patch set: pi_k = p_0 / sum_i p_i with
// p_i = exp(-E_i/(2 sigma_r^2 s^2)), rho_k = Gamma_n pi_k + Q^(n+1)(centre),
// and at the finest level with variance on the PDF fit.
// The memory inputs of one patch's posterior (loaded before sigma_r is
// known, so the loads overlap its reduction).
struct PostIn {
    float4 r0, r1, r2;  // d, dinit, dlast, H | E0, dE1, dE2, dE3 | dE4, cT, flags, nout + pdf_flags
    float mu, prop;     // mean offset; coarse probability at the centre (Eq. 10)
};

__device__ __forceinline__ PostIn posterior_load(const LaunchArgs &a, const LevelDesc &D, int kx,
                                                 int ky) {
    const bdis_patch_record *rec = D.rec + ky * D.npx + kx;
    // L2 loads: the record was written by another block, possibly earlier in
    // the same (persistent) launch
    PostIn in;
    in.r0 = __ldcg((const float4 *)rec);
    in.r1 = __ldcg((const float4 *)rec + 1);
    in.r2 = __ldcg((const float4 *)rec + 2);
    in.mu = __ldcg(&rec->mu);
    in.prop = 0.f;
    if (a.use_c2f && D.Qc != nullptr) {
        const float cx = (float)origin(kx, D.w, a.P, a.S, D.kxreg) + 0.5f * (float)(a.P - 1);
        const float cy = (float)origin(ky, D.h, a.P, a.S, D.kyreg) + 0.5f * (float)(a.P - 1);
        in.prop = coarse_bilin(D.Qc, D.wc, D.hc, cx, cy);
    }
    return in;
}

__device__ __forceinline__ float4 posterior_of(const LaunchArgs &a, const LevelDesc &D, int kx, int ky,
                               const PostIn &in, float sr, bool write) {
    const int k = ky * D.npx + kx;
    bdis_patch_record *rec = D.rec + k;
    const float4 r0 = in.r0, r1 = in.r1, r2 = in.r2;
    const uint32_t flags = __float_as_uint(r2.z);
    if (flags != 0u) {
        if (write) {
            rec->pi = rec->rho = rec->sig2 = 0.f;
            rec->pdf_flags = 0;
            D.fuse[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float mu = in.mu;
    const float h = a.window_step;
    const float dlt[5] = {0.f, -h, h, -2.f * h, 2.f * h};
    // 1 / (2 sigma_r^2 s^2): one division, the same for every patch of the pair
    const float iscale = 1.f / (2.f * sr * sr * (float)(kWindow * kWindow));
    // ln p_i - ln p_0 = -(E_i - E_0) / (2 sigma_r^2 s^2); the record holds E_i - E_0
    const float dE[5] = {0.f, r1.y, r1.z, r1.w, r2.x};
    float e[5], Z = 1.f;
    e[0] = 0.f;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        e[i] = -dE[i] * iscale;
        Z += expf(e[i]);
    }
    // pi = p_0 / sum_i p_i; with fast_exp every p_i (p_0 included) is
    // Schraudolph's approximation; the PDF fit keeps the exact log-probabilities
    float pi = 1.f / Z;
    if (a.fast_exp) {
        const float p0 = exp_schraudolph(0.f);
        float Zf = p0;
#pragma unroll
        for (int i = 1; i < 5; ++i) Zf += exp_schraudolph(e[i]);
        pi = p0 / Zf;
    }
    float rho;
    if (a.use_c2f) {
        rho = a.gamma_w * pi + in.prop;
    } else {
        rho = pi;
    }
    float sig2 = 0.f;
    uint32_t pf = 0u;
    if (a.level == a.finest && a.variance) {
        const float lnZ = logf(Z);
        float lnp[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) lnp[i] = e[i] - lnZ;
        sig2 = pdf_fit(lnp, dlt, a.pdf_iters, a.pdf_resid, a.tau0, pf);
    }
    // .w: the mean offset, read by the DIS-weighted fusion
    const float4 fz = make_float4(r0.x, rho, sig2, mu);
    if (write) {
        rec->pi = pi;
        rec->rho = rho;
        rec->sig2 = sig2;
        rec->pdf_flags = (uint16_t)pf;
        D.fuse[k] = fz;
    }
    return fz;
}

// Covering patch indices of pixel coordinate x along one axis: regular k
// with kS <= x < kS + P, plus the ragged one.
// rS = 1/S (udiv_small).
__device__ __forceinline__ void cover(int x, int n, int P, int S, float rS, int kreg, int np, int &lo,
                                      int &hi, bool &ext) {
    lo = x - P + 1 > 0 ? udiv_small(x - P + 1 + S - 1, rS) : 0;
    hi = min(kreg - 1, udiv_small(x, rS));
    ext = np > kreg && x >= n - P;
}

// A block owns a TW x TH pixel tile.  It reads sigma_r of its pair (reduced
// by the search), computes the posterior of every patch overlapping the tile
// into shared memory (the tile containing a patch's origin writes its
// record), then fuses its pixels by a gather over the covering kept patches
// (no atomics):
//   omega_k = rho_k m[x - ox] m[y - oy], D = sum omega d / sum omega,
//   Q = sum omega rho / sum omega, V = sum omega^2 sig2 / (sum omega)^2.
// The weight is separable, so the gather runs in two passes: per tile column
// and covering patch row, sums over the covering patch columns; then per
// pixel, sums over the covering patch rows.
template <int TW, int TH>
__device__ __forceinline__ void fuse_unit(const LaunchArgs &a, int unit, float4 *fz) {
    // fz: nkx * nky posteriors, then nky * TW column sums (dynamic shared memory).
    // The tile size is a compile-time constant (32x16, 64x32 or 64x64), so the pixel
    // index arithmetic is shifts and masks.
    __shared__ int cxlo[kFuseTileWMax], cxn[kFuseTileWMax], cxr[kFuseTileWMax];
    __shared__ int cylo[kFuseTileHMax], cyn[kFuseTileHMax], cyr[kFuseTileHMax];
    __shared__ float cxm[kFuseTileWMax][kMaxPatch + 2], cym[kFuseTileHMax][kMaxPatch + 2];
    const int P = a.P, S = a.S;

    // the descriptor is copied to registers: the pixel stores could alias it
    // as far as the compiler knows, which would reload its fields per pixel
    const LevelDesc D = a.descs[find_pair(a.descs, a.npairs, unit, W_FUSE)];
    const int tile = unit - D.work_begin[W_FUSE];
    const int ty = udiv_small(tile, recip(D.tiles_x)), tx = tile - ty * D.tiles_x;
    const float rS = recip(S);
    const int x0 = tx * TW, y0 = ty * TH;
    const int x1 = min(x0 + TW, D.w) - 1, y1 = min(y0 + TH, D.h) - 1;
    // patches overlapping the tile
    int kxlo, kxhi, kylo, kyhi, tmp;
    bool kxext, kyext, bext;
    cover(x0, D.w, P, S, rS, D.kxreg, D.npx, kxlo, tmp, bext);
    cover(x1, D.w, P, S, rS, D.kxreg, D.npx, tmp, kxhi, kxext);
    cover(y0, D.h, P, S, rS, D.kyreg, D.npy, kylo, tmp, bext);
    cover(y1, D.h, P, S, rS, D.kyreg, D.npy, tmp, kyhi, kyext);
    const int nkxr = max(0, kxhi - kxlo + 1), nkyr = max(0, kyhi - kylo + 1);
    const int nkx = nkxr + (kxext ? 1 : 0);
    const int nky = nkyr + (kyext ? 1 : 0);
    const float rnkx = recip(nkx);
    // the first patch's posterior inputs are loaded before sigma_r is known
    auto patch_of = [&](int i, int &kx, int &ky) {
        const int iy = udiv_small(i, rnkx), ix = i - iy * nkx;
        kx = ix < nkxr ? kxlo + ix : D.npx - 1;
        ky = iy < nkyr ? kylo + iy : D.npy - 1;
    };
    PostIn pre;
    if ((int)threadIdx.x < nkx * nky) {
        int kx, ky;
        patch_of(threadIdx.x, kx, ky);
        pre = posterior_load(a, D, kx, ky);
    }
    // sigma_r of the pair from the search's exact integer sums (text after
    // Eq. 6), converted once to FP32 by one thread and broadcast through
    // shared memory
    __shared__ float sr_sh;
    if (threadIdx.x == 0) {
        float sr;
        const unsigned long long n = __ldcg(D.acc + 1);
        const float S1 = __ull2float_rn(__ldcg(D.acc)) * (1.f / kSigmaFix1);  // sum E(0)
        const float S2 = __ull2float_rn(n);                                  // kept patches
        const float S3 = __ull2float_rn(__ldcg(D.acc + 2));                  // sum E(0)^2
        if (a.sigma_r_mode == BDIS_SIGMA_R_FIXED) {
            sr = a.sigma_r_fixed;
        } else if (n == 0ull) {
            sr = a.sigma_r_floor;
        } else if (a.sigma_r_mode == BDIS_SIGMA_R_LITERAL) {
            // population variance mean(E^2) - mean(E)^2, the square's
            // rounding error taken back by an FMA
            const float mean = S1 / S2;
            const float sq = mean * mean;
            const float var = (S3 / S2 - sq) - fmaf(mean, mean, -sq);
            sr = fmaxf(sqrtf(fmaxf(var, 0.f)), a.sigma_r_floor);
        } else {
            sr = fmaxf(sqrtf(S1 / (S2 * (float)(P * P))), a.sigma_r_floor);
        }
        if (tile == 0) *D.sigma_r = sr;
        sr_sh = sr;
    }
    __syncthreads();
    const float sr = sr_sh;

    for (int i = threadIdx.x; i < nkx * nky; i += blockDim.x) {
        int kx, ky;
        patch_of(i, kx, ky);
        const int ox = origin(kx, D.w, P, S, D.kxreg);
        const int oy = origin(ky, D.h, P, S, D.kyreg);
        const bool owner = ox >= x0 && ox < x0 + TW && oy >= y0 && oy < y0 + TH;
        const PostIn in = i == (int)threadIdx.x ? pre : posterior_load(a, D, kx, ky);
        fz[i] = posterior_of(a, D, kx, ky, in, sr, owner);
    }
    // covering patches (tile-local indices) and their weights per column / row,
    // by the block's last two warps (the posteriors start at thread 0, so the
    // two run side by side)
    for (int ci = (int)threadIdx.x - ((int)blockDim.x - 64); ci >= 0 && ci < TW + TH; ci += 64) {
        const bool col = ci < TW;
        const int c = col ? ci : ci - TW;
        const int xy = (col ? x0 : y0) + c;
        const int n = col ? D.w : D.h, kreg = col ? D.kxreg : D.kyreg, np = col ? D.npx : D.npy;
        const int klo = col ? kxlo : kylo, nr = col ? nkxr : nkyr, nt = col ? nkx : nky;
        int lo = 0, hi = -1;
        bool ext = false;
        if (xy < n) cover(xy, n, P, S, rS, kreg, np, lo, hi, ext);
        const int cnt = xy < n ? max(0, hi - lo + 1) + (ext ? 1 : 0) : 0;
        float *mrow = col ? cxm[c] : cym[c];
        for (int q = 0; q < cnt; ++q) {
            const bool isx = lo + q > hi;  // the ragged extra patch comes last
            const int k = isx ? np - 1 : lo + q;
            const int o = origin(k, n, P, S, kreg);
            mrow[q] = a.use_sgmm ? a.m[xy - o] : 1.f;
        }
        (col ? cxlo : cylo)[c] = lo - klo;  // first regular local index
        (col ? cxn : cyn)[c] = cnt;
        (col ? cxr : cyr)[c] = xy < n ? max(0, hi - lo + 1) : 0;  // regular entries
        (void)nr;
        (void)nt;
    }
    __syncthreads();

    // one fused pixel: D = sum omega d / sum omega, Q = sum omega rho / sum omega,
    // V = sum omega^2 sig2 / (sum omega)^2
    auto emit = [&](int x, int y, float swd, float sw, float swr, float sw2) {
        const size_t idx = (size_t)y * D.w + x;
        const bool any = sw > 0.f;
        float Dv, Qv, Vv;
        if (any) {
            const float inv = 1.f / sw;
            Dv = swd * inv;
            Qv = swr * inv;
            Vv = sw2 * inv * inv;
        } else {
            Dv = D.Dc != nullptr ? 2.f * coarse_bilin(D.Dc, D.wc, D.hc, (float)x, (float)y) : 0.f;
            Qv = 0.f;
            Vv = 0.f;
        }
        const float qnan = __int_as_float(0x7fc00000);
        if (D.wsum != nullptr) D.wsum[idx] = sw;
        if (a.level == a.finest) {
            const bool ok = any && Qv >= a.pix_thresh;
            if (a.level == 0) {
                D.valid[idx] = ok ? 1 : 0;
                D.disp[idx] = ok ? Dv : qnan;
                if (D.var != nullptr && a.variance) D.var[idx] = ok ? Vv : qnan;
            } else {
                // level-f maps for the full-resolution upsampling (NaN = invalid)
                D.D[idx] = ok ? Dv : qnan;
                if (D.var != nullptr && a.variance) D.var[idx] = Vv;
            }
        } else {
            D.D[idx] = Dv;
            D.Q[idx] = Qv;
        }
    };

    if (a.weight_mode == BDIS_WEIGHT_DIS) {
        // Eq. 2 weights depend on the pixel: direct gather over the covering
        // patches, omega = 1 / max(1, (I_r(x - d) - I_l(x) - mu)^2)
        for (int pix = threadIdx.x; pix < TW * TH; pix += blockDim.x) {
            const int c = pix % TW, r = pix / TW;
            const int x = x0 + c, y = y0 + r;
            if (x > x1 || y > y1) continue;
            const size_t row = (size_t)y * D.pitch;
            const float Il = ld_typed(D.L, row + x, a.img_type);
            const int cntx = cxn[c], lox = cxlo[c], nrx = cxr[c];
            const int cnty = cyn[r], loy = cylo[r], nry = cyr[r];
            float swd = 0.f, sw = 0.f, swr = 0.f, sw2 = 0.f;
            for (int qy = 0; qy < cnty; ++qy) {
                const int ly = qy < nry ? loy + qy : nky - 1;
                for (int qx = 0; qx < cntx; ++qx) {
                    const int lx = qx < nrx ? lox + qx : nkx - 1;
                    const float4 f = fz[ly * nkx + lx];
                    if (!(f.y > 0.f)) continue;  // rejected patch
                    const float X = fminf(fmaxf((float)x - f.x, 0.f), (float)(D.w - 1));
                    const int xa = (int)floorf(X);
                    const int xb = min(xa + 1, D.w - 1);
                    const float t = X - (float)xa;
                    const float ra = ld_typed(D.R, row + xa, a.img_type);
                    const float rb = ld_typed(D.R, row + xb, a.img_type);
                    const float res = fmaf(t, rb - ra, ra) - Il - f.w;
                    const float om = 1.f / fmaxf(res * res, 1.f);
                    swd = fmaf(om, f.x, swd);
                    sw += om;
                    swr = fmaf(om, f.y, swr);
                    sw2 = fmaf(om * om, f.z, sw2);
                }
            }
            emit(x, y, swd, sw, swr, sw2);
        }
        __syncthreads();
        return;
    }

    // pass 1: per tile column x and patch row iy, sums over the covering columns
    float4 *csum = fz + nkx * nky;  // [nky][TW] of (sum m rho d, sum m rho, sum m rho^2, sum m^2 rho^2 sig2)
    for (int i = threadIdx.x; i < nky * TW; i += blockDim.x) {
        const int iy = i / TW, c = i - iy * TW;
        const int cnt = cxn[c], lo = cxlo[c], nreg = cxr[c];
        float A = 0.f, Bw = 0.f, Cq = 0.f, V = 0.f;
        for (int q = 0; q < cnt; ++q) {
            const int lx = q < nreg ? lo + q : nkx - 1;
            const float4 f = fz[iy * nkx + lx];
            const float mr = cxm[c][q] * f.y;  // 0 for a rejected patch
            A = fmaf(mr, f.x, A);
            Bw += mr;
            Cq = fmaf(mr, f.y, Cq);
            V = fmaf(mr * mr, f.z, V);
        }
        csum[i] = make_float4(A, Bw, Cq, V);
    }
    __syncthreads();

    // pass 2: per pixel, sums over the covering patch rows
    for (int pix = threadIdx.x; pix < TW * TH; pix += blockDim.x) {
        const int c = pix % TW, r = pix / TW;
        const int x = x0 + c, y = y0 + r;
        if (x > x1 || y > y1) continue;
        const int cnt = cyn[r], lo = cylo[r], nreg = cyr[r];
        float swd = 0.f, sw = 0.f, swr = 0.f, sw2 = 0.f;
        for (int q = 0; q < cnt; ++q) {
            const int ly = q < nreg ? lo + q : nky - 1;
            const float4 cs = csum[ly * TW + c];
            const float my = cym[r][q];
            swd = fmaf(my, cs.x, swd);
            sw = fmaf(my, cs.y, sw);
            swr = fmaf(my, cs.z, swr);
            sw2 = fmaf(my * my, cs.w, sw2);
        }
        emit(x, y, swd, sw, swr, sw2);
    }
    __syncthreads();
    }

// Full-resolution output from the finest processed level f > 0: a unit is
// kUpUnitPixels consecutive level-0 pixels of one pair.  Level-f coordinate
// X = (x + 0.5) / 2^f - 0.5 (clamped), disp = 2^f bilinear(D_f),
// var = 4^f bilinear(V_f); valid iff every level-f pixel with a non-zero
// bilinear weight is valid (not NaN in D_f).
__device__ __forceinline__ void upsample_unit(const LaunchArgs &a, int unit) {
    const LevelDesc D = a.descs[find_pair(a.descs, a.npairs, unit, W_UP)];  // in registers (see fuse_unit)
    const int u = unit - D.work_begin[W_UP];
    const float sc = (float)(1 << a.finest), inv = 1.f / sc;  // exact (power of two)
    const long long npix = (long long)D.w * D.h;
    const float qnan = __int_as_float(0x7fc00000);
    for (int i = threadIdx.x; i < kUpUnitPixels; i += blockDim.x) {
        const long long pix = (long long)u * kUpUnitPixels + i;
        if (pix >= npix) break;
        const int y = (int)(pix / D.w), x = (int)(pix - (long long)y * D.w);
        const float X = fminf(fmaxf(((float)x + 0.5f) * inv - 0.5f, 0.f), (float)(D.wf - 1));
        const float Y = fminf(fmaxf(((float)y + 0.5f) * inv - 0.5f, 0.f), (float)(D.hf - 1));
        const int xa = (int)floorf(X), ya = (int)floorf(Y);
        const int xb = min(xa + 1, D.wf - 1), yb = min(ya + 1, D.hf - 1);
        const float fx = X - (float)xa, fy = Y - (float)ya;
        const int xs[4] = {xa, xb, xa, xb}, ys[4] = {ya, ya, yb, yb};
        const float wt[4] = {(1.f - fx) * (1.f - fy), fx * (1.f - fy), (1.f - fx) * fy, fx * fy};
        bool ok = true;
        float dv = 0.f, vv = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (wt[k] == 0.f) continue;
            const size_t j = (size_t)ys[k] * D.wf + xs[k];
            const float dk = __ldcg(D.Df + j);
            ok = ok && !isnan(dk);
            dv = fmaf(wt[k], dk, dv);
            if (D.Vf != nullptr) vv = fmaf(wt[k], __ldcg(D.Vf + j), vv);
        }
        D.valid[pix] = ok ? 1 : 0;
        D.disp[pix] = ok ? sc * dv : qnan;
        if (D.var != nullptr && a.variance) D.var[pix] = (ok && D.Vf != nullptr) ? sc * sc * vv : qnan;
    }
}

__global__ void __launch_bounds__(256) k_upsample(LaunchArgs a) {
    pdl_enter(a);
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) upsample_unit(a, unit);
    pdl_leave(a);
}

// Depth (Eq. 13) and its variance (the depth factor of Eq. 17), elementwise.
__device__ __forceinline__ void depth_px(float d, float v, float fb, float &z, float &zv) {
    const bool ok = d > 0.f && d < INFINITY;  // a positive finite disparity (false for NaN)
    const float q = fb / d;
    const float qd = q / d;   // fb / d^2
    z = ok ? q : __int_as_float(0x7fc00000);
    zv = ok ? qd * qd * v : __int_as_float(0x7fc00000);
}

// 16-byte vectors when every pointer allows it (the common case), scalars
// for the tail; grid-strided so each thread keeps several loads in flight.
__global__ void __launch_bounds__(256) k_depth(const float *__restrict__ disp,
                                               const float *__restrict__ var, long long n, float fb,
                                               float *__restrict__ depth,
                                               float *__restrict__ depth_var) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool hv = depth_var != nullptr;
    const uintptr_t al = (uintptr_t)disp | (uintptr_t)depth | (uintptr_t)var | (uintptr_t)depth_var;
    const long long n4 = (al & 15u) == 0 ? n / 4 : 0;
    for (long long i = tid; i < n4; i += stride) {
        const float4 d = __ldg((const float4 *)disp + i);
        const float4 v = hv ? __ldg((const float4 *)var + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 z, zv;
        depth_px(d.x, v.x, fb, z.x, zv.x);
        depth_px(d.y, v.y, fb, z.y, zv.y);
        depth_px(d.z, v.z, fb, z.z, zv.z);
        depth_px(d.w, v.w, fb, z.w, zv.w);
        __stcs((float4 *)depth + i, z);
        if (hv) __stcs((float4 *)depth_var + i, zv);
    }
    for (long long i = 4 * n4 + tid; i < n; i += stride) {
        float z, zv;
        depth_px(__ldg(disp + i), hv ? __ldg(var + i) : 0.f, fb, z, zv);
        depth[i] = z;
        if (hv) depth_var[i] = zv;
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(256, 4) k_fuse(LaunchArgs a) {
    extern __shared__ float4 fz[];
    pdl_enter(a);
    for (int unit = blockIdx.x; unit < a.total; unit += gridDim.x) fuse_unit<TW, TH>(a, unit, fz);
    pdl_leave(a);
}

// ---------------------------------------------------------------- persistent form

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// Thread 0 of each block arrives on a counter; the last arrival resets it and
// bumps the generation, the others wait for the generation to change.  Every
// wait is bounded: past `limit` polls the block records the timeout and goes
// on, so the kernel always terminates.  `unreachable` (a test of that path)
// makes no arrival the last one, so every wait runs out.
__device__ void grid_barrier(unsigned *bar, int *err, int *err_host, unsigned limit, int unreachable) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (!unreachable && arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g) {
                if (++it > limit) {
                    atomicOr(err, 1);
                    if (err_host != nullptr) {
                        *(volatile int *)err_host = 1;  // the host takes it on its next call
                        __threadfence_system();
                    }
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// All stages of one call: the pyramid levels, then search and fuse per level
// coarse to fine, each stage striding its units over the persistent grid.
template <int P, typename TG>
__global__ void __launch_bounds__(256) k_mega(MegaArgs m) {
    extern __shared__ __align__(16) float smem[];
    pdl_wait();
    for (int s = 0; s < m.nstages; ++s) {
        const LaunchArgs &a = m.stages[s];
        const int total = a.total;
        if (a.kind == 0) {
            if (blockIdx.x == 0 && a.acc_zero != nullptr)
                for (int i = threadIdx.x; i < a.acc_count; i += blockDim.x) a.acc_zero[i] = 0ull;
            float(*Ls)[kPyrSP] = (float(*)[kPyrSP])smem;
            float(*Rs)[kPyrSP] = Ls + kPyrSH;
            float(*Lh)[kPyrHP] = (float(*)[kPyrHP])(smem + 2 * kPyrSH * kPyrSP);
            float(*Rh)[kPyrHP] = Lh + kPyrSH;
            if (a.level == 0) {
                for (int u = blockIdx.x; u < total; u += gridDim.x)
                    pyramid_unit<uint8_t, TG, TG>(a, u, Ls, Rs, Lh, Rh);
            } else {
                for (int u = blockIdx.x; u < total; u += gridDim.x) pyramid_unit<TG, TG, TG>(a, u, Ls, Rs, Lh, Rh);
            }
        } else if (a.kind == 4) {
            if (blockIdx.x == 0 && a.acc_zero != nullptr)
                for (int i = threadIdx.x; i < a.acc_count; i += blockDim.x) a.acc_zero[i] = 0ull;
            if (a.level == 0) {
                for (int u = blockIdx.x; u < total; u += gridDim.x) pyramid2_unit<uint8_t, TG, TG>(a, u, smem);
            } else {
                for (int u = blockIdx.x; u < total; u += gridDim.x) pyramid2_unit<TG, TG, TG>(a, u, smem);
            }
        } else if (a.kind == 1) {
            unsigned ph = 0u;  // (no bulk staging in the persistent form)
            if (a.level == 0) {
                for (int u = blockIdx.x; u < total; u += gridDim.x) search_unit<P, uint8_t, TG, false>(a, u, smem, ph);
            } else {
                for (int u = blockIdx.x; u < total; u += gridDim.x) search_unit<P, TG, TG, false>(a, u, smem, ph);
            }
        } else if (a.kind == 2) {
            if (a.tile_w == 64 && a.tile_h == 64) {
                for (int u = blockIdx.x; u < total; u += gridDim.x) fuse_unit<64, 64>(a, u, (float4 *)smem);
            } else if (a.tile_w == 64) {
                for (int u = blockIdx.x; u < total; u += gridDim.x) fuse_unit<64, 32>(a, u, (float4 *)smem);
            } else {
                for (int u = blockIdx.x; u < total; u += gridDim.x) fuse_unit<32, 16>(a, u, (float4 *)smem);
            }
        } else {
            for (int u = blockIdx.x; u < total; u += gridDim.x) upsample_unit(a, u);
        }
        if (s + 1 < m.nstages) grid_barrier(m.bar, m.err, m.err_host, m.spin_limit, m.unreachable);
    }
    pdl_release();
}

const void *mega_kernel(int P, int st_type) {
    const bool h = st_type == E_F16;
    switch (P) {
        case 6: return h ? (const void *)k_mega<6, __half> : (const void *)k_mega<6, float>;
        case 8: return h ? (const void *)k_mega<8, __half> : (const void *)k_mega<8, float>;
        case 10: return h ? (const void *)k_mega<10, __half> : (const void *)k_mega<10, float>;
        case 12: return h ? (const void *)k_mega<12, __half> : (const void *)k_mega<12, float>;
        case 16: return h ? (const void *)k_mega<16, __half> : (const void *)k_mega<16, float>;
        default: return nullptr;
    }
}

// ---------------------------------------------------------------- dispatch

// (image type, gradient type): (u8, f32), (u8, f16), (f32, f32), (f32, f16), (f16, f16)
template <int P, bool BULK = false>
const void *search_fn(int in_type, int g_type) {
    if (in_type == E_U8)
        return g_type == E_F32 ? (const void *)k_search<P, uint8_t, float, BULK>
                               : (const void *)k_search<P, uint8_t, __half, BULK>;
    if (in_type == E_F32)
        return g_type == E_F32 ? (const void *)k_search<P, float, float, BULK>
                               : (const void *)k_search<P, float, __half, BULK>;
    if (in_type == E_F16 && g_type == E_F16) return (const void *)k_search<P, __half, __half, BULK>;
    return nullptr;
}

// bulk: the instance with the bulk band staging where one is compiled (P = 8
// and 12), else the default one (same results)
const void *search_kernel(int P, int in_type, int g_type, bool bulk) {
    if (bulk && P == 8) return search_fn<8, true>(in_type, g_type);
    if (bulk && P == 12) return search_fn<12, true>(in_type, g_type);
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

cudaError_t raise_smem_limit(const void *f, size_t bytes);

bool search_supported(int P) { return P >= kMinPatch && P <= kMaxPatch; }

void search_layout(int P, int S, float tau, float window_step, int passes, int &band_pitch,
                   int &band_cap, int &chunk_pitch, size_t &bytes, bool bulk) {
    const int chunk = search_chunk(P, passes);
    const int cw = (chunk - 1) * S + P;
    const int margin = (int)ceilf(tau) + (int)ceilf(2.f * window_step) + 3;
    band_cap = cw + 2 * margin + kBandSpread;
    band_pitch = (band_cap + 31) / 32 * 32 + 1;  // rows land in different banks
    chunk_pitch = cw | 1;
    bytes = sizeof(float) * ((size_t)P * band_pitch + 2 * (size_t)P * chunk_pitch + 4 * (size_t)chunk + 16);
    // bulk staging of the right band: a 16-byte aligned mbarrier slot, then P
    // raw rows of the widest storage type (FP32)
    if (bulk) bytes = (bytes + 15) / 16 * 16 + 16 + (size_t)P * search_raw_pitch(band_cap, 4);
}

size_t fuse_smem(int P, int S, int tile_w, int tile_h) {
    const int nkx = (tile_w + P - 2) / S + 2, nky = (tile_h + P - 2) / S + 2;
    return sizeof(float4) * ((size_t)nkx * nky + (size_t)nky * tile_w);
}

cudaError_t prepare_fuse(size_t smem_bytes) {
    cudaError_t e = raise_smem_limit((const void *)k_fuse<32, 16>, smem_bytes);
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_fuse<64, 32>, smem_bytes);
    return e != cudaSuccess ? e : raise_smem_limit((const void *)k_fuse<64, 64>, smem_bytes);
}

bool mega_supported(int P) { return mega_kernel(P, E_F32) != nullptr; }

int mega_grid(int P, int st_type, size_t smem) {
    const void *f = mega_kernel(P, st_type);
    if (f == nullptr || raise_smem_limit(f, smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem) != cudaSuccess) return 0;
    return nb * num_sms();
}

cudaError_t launch_mega(const MegaArgs &m, int P, int st_type, int grid, size_t smem, bool pdl,
                        cudaStream_t s) {
    const void *f = mega_kernel(P, st_type);
    if (f == nullptr || grid < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    void *args[] = {(void *)&m};
    return cudaLaunchKernelExC(&cfg, f, args);
}
int search_group(int P) { return P <= 8 ? 8 : 16; }
int search_chunk(int P, int passes) { return passes * (256 / search_group(P)); }

// Raises (never lowers) a kernel's dynamic shared-memory limit to `bytes`
// (the default limit is 48 KB less the kernel's static shared memory).
cudaError_t raise_smem_limit(const void *f, size_t bytes) {
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, f);
    if (e != cudaSuccess) return e;
    if ((size_t)at.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t prepare_search(int P, size_t smem_bytes) {
    const int combos[5][2] = {{E_U8, E_F32}, {E_U8, E_F16}, {E_F32, E_F32}, {E_F32, E_F16},
                              {E_F16, E_F16}};
    for (const auto &c : combos)
        for (const bool bulk : {false, true}) {
            const void *f = search_kernel(P, c[0], c[1], bulk);
            if (f == nullptr) return cudaErrorInvalidValue;
            cudaError_t e = raise_smem_limit(f, smem_bytes);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

int search_occupancy(int P, int in_type, int g_type, size_t smem_bytes, bool bulk) {
    int nb = 0;
    const void *f = search_kernel(P, in_type, g_type, bulk);
    if (f == nullptr) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem_bytes) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

namespace {
// One 256-thread launch of a LaunchArgs kernel; with a.pdl the launch allows
// programmatic stream serialisation (the kernel waits in pdl_wait()).
int resident_blocks(const void *f, size_t smem);

cudaError_t launch_args_kernel(const void *f, const LaunchArgs &args, int grid, size_t smem,
                               cudaStream_t s) {
    LaunchArgs a = args;
    a.early = a.pdl == 2 && grid <= num_sms() * resident_blocks(f, smem) ? 1 : 0;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 1 : 0;
    void *kargs[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, f, kargs);
}
}  // namespace

namespace {
// Resident blocks per SM of a kernel at a dynamic shared-memory size (cached).
int resident_blocks(const void *f, size_t smem) {
    static const void *keys[16];
    static size_t sizes[16];
    static int vals[16];
    static int n = 0;
    for (int i = 0; i < n; ++i)
        if (keys[i] == f && sizes[i] == smem) return vals[i];
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    if (n < 16) {
        keys[n] = f;
        sizes[n] = smem;
        vals[n] = nb;
        ++n;
    }
    return nb;
}

template <typename TI, typename TN, typename TG>
cudaError_t launch_pyramid_bulk(const LaunchArgs &a, cudaStream_t s) {
    const void *f = (const void *)k_pyramid_bulk<TI, TN, TG>;
    const size_t smem = PyrBulk<TI>::kSmem;
    const cudaError_t e = raise_smem_limit(f, smem);
    if (e != cudaSuccess) return e;
    // every block resident: each walks its units with the copies of the next
    // one in flight
    return launch_args_kernel(f, a, grid_for(a.total, resident_blocks(f, smem)), smem, s);
}

// The (read, next level, gradient) element types of a pyramid launch: FP32
// or FP16 pyramids with gradients of the same type, or 8-bit pyramids with
// FP16 gradients; the images read are the level-0 input (8-bit or FP32) or
// the stored type.
#define BDIS_PYR_TYPES(X)                                                                  \
    X(E_U8, E_F32, E_F32, uint8_t, float, float)                                           \
    X(E_F32, E_F32, E_F32, float, float, float)                                            \
    X(E_U8, E_F16, E_F16, uint8_t, __half, __half)                                         \
    X(E_F32, E_F16, E_F16, float, __half, __half)                                          \
    X(E_F16, E_F16, E_F16, __half, __half, __half)                                         \
    X(E_U8, E_U8, E_F16, uint8_t, uint8_t, __half)                                         \
    X(E_F32, E_U8, E_F16, float, uint8_t, __half)

const void *pyramid_kernel(int in_type, int img_type, int g_type) {
#define BDIS_PYR_CASE(a, b, c, TI, TN, TG) \
    if (in_type == a && img_type == b && g_type == c) return (const void *)k_pyramid<TI, TN, TG>;
    BDIS_PYR_TYPES(BDIS_PYR_CASE)
#undef BDIS_PYR_CASE
    return nullptr;
}

const void *pyramid2_kernel(int in_type, int img_type, int g_type) {
#define BDIS_PYR_CASE(a, b, c, TI, TN, TG) \
    if (in_type == a && img_type == b && g_type == c) return (const void *)k_pyramid2<TI, TN, TG>;
    BDIS_PYR_TYPES(BDIS_PYR_CASE)
#undef BDIS_PYR_CASE
    return nullptr;
}

cudaError_t launch_pyramid_bulk_typed(const LaunchArgs &a, int in_type, int img_type, int g_type,
                                      cudaStream_t s) {
#define BDIS_PYR_CASE(a_, b, c, TI, TN, TG) \
    if (in_type == a_ && img_type == b && g_type == c) return launch_pyramid_bulk<TI, TN, TG>(a, s);
    BDIS_PYR_TYPES(BDIS_PYR_CASE)
#undef BDIS_PYR_CASE
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_pyramid(const LaunchArgs &a, int in_type, int img_type, int g_type, cudaStream_t s) {
    if (a.bulk & 1) return launch_pyramid_bulk_typed(a, in_type, img_type, g_type, s);
    const void *f = pyramid_kernel(in_type, img_type, g_type);
    if (f == nullptr) return cudaErrorInvalidValue;
    return launch_args_kernel(f, a, grid_for(a.total, 8), 0, s);
}

cudaError_t launch_pyramid2(const LaunchArgs &a, int in_type, int img_type, int g_type, cudaStream_t s) {
    const void *f = pyramid2_kernel(in_type, img_type, g_type);
    if (f == nullptr) return cudaErrorInvalidValue;
    return launch_args_kernel(f, a, grid_for(a.total, 8), 0, s);
}

cudaError_t launch_search(const LaunchArgs &a, int in_type, int g_type, size_t smem, int grid,
                          cudaStream_t s) {
    const void *f = search_kernel(a.P, in_type, g_type, (a.bulk & 2) != 0);
    if (f == nullptr) return cudaErrorInvalidValue;
    return launch_args_kernel(f, a, grid, smem, s);
}

cudaError_t launch_fuse(const LaunchArgs &a, size_t smem, cudaStream_t s) {
    const void *f = a.tile_w == 64 ? (a.tile_h == 64 ? (const void *)k_fuse<64, 64> : (const void *)k_fuse<64, 32>)
                                   : (const void *)k_fuse<32, 16>;
    return launch_args_kernel(f, a, grid_for(a.total, 8), smem, s);
}

cudaError_t launch_upsample(const LaunchArgs &a, cudaStream_t s) {
    return launch_args_kernel((const void *)k_upsample, a, grid_for(a.total, 8), 0, s);
}

cudaError_t launch_depth(const float *disp, const float *var, long long n, float fb, float *depth,
                         float *depth_var, cudaStream_t s) {
    const long long blocks = (n / 4 + 255) / 256 + 1;
    const int grid = (int)std::max<long long>(1, std::min<long long>(blocks, (long long)num_sms() * 8));
    k_depth<<<grid, 256, 0, s>>>(disp, var, n, fb, depth, depth_var);
    return cudaGetLastError();
}

}  // namespace bdis
