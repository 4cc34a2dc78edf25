// bdis_device.cuh -- small device helpers shared by the kernels of libbdis.
#pragma once

#include <cmath>

#include "bdis_internal.cuh"

namespace bdis {
namespace {

__device__ __forceinline__ float ldf(const uint8_t *p) { return (float)__ldg(p); }
__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(__half *p, float v) { *p = __float2half_rn(v); }
// an 8-bit image value: nearest integer, ties to even, within 0..255
__device__ __forceinline__ void stf(uint8_t *p, float v) {
    *p = (uint8_t)__float2uint_rn(fminf(fmaxf(v, 0.f), 255.f));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Four consecutive elements as floats; p aligned to four elements.
__device__ __forceinline__ float4 ld4f(const uint8_t *p) {
    const uchar4 u = __ldg((const uchar4 *)p);
    return make_float4((float)u.x, (float)u.y, (float)u.z, (float)u.w);
}
__device__ __forceinline__ float4 ld4f(const float *p) { return __ldg((const float4 *)p); }
__device__ __forceinline__ float4 ld4f(const __half *p) {
    const uint2 u = __ldg((const uint2 *)p);
    const float2 a = __half22float2(*(const __half2 *)&u.x);
    const float2 b = __half22float2(*(const __half2 *)&u.y);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Eight consecutive values stored as floats or halves (rounded to nearest);
// p aligned to 16 bytes.
__device__ __forceinline__ void st8(float *p, const float *v) {
    ((float4 *)p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    ((float4 *)p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void st8(__half *p, const float *v) {
    const __half2 h0 = __floats2half2_rn(v[0], v[1]), h1 = __floats2half2_rn(v[2], v[3]);
    const __half2 h2 = __floats2half2_rn(v[4], v[5]), h3 = __floats2half2_rn(v[6], v[7]);
    uint4 u;
    u.x = *(const unsigned *)&h0;
    u.y = *(const unsigned *)&h1;
    u.z = *(const unsigned *)&h2;
    u.w = *(const unsigned *)&h3;
    *(uint4 *)p = u;
}
// Two consecutive values; p aligned to two elements.
__device__ __forceinline__ void st2(float *p, float a, float b) { *(float2 *)p = make_float2(a, b); }
__device__ __forceinline__ void st2(__half *p, float a, float b) { *(__half2 *)p = __floats2half2_rn(a, b); }
__device__ __forceinline__ void st2(uint8_t *p, float a, float b) {
    *(uchar2 *)p = make_uchar2((uint8_t)__float2uint_rn(fminf(fmaxf(a, 0.f), 255.f)),
                               (uint8_t)__float2uint_rn(fminf(fmaxf(b, 0.f), 255.f)));
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while its predecessor on the stream still runs;
// pdl_wait() returns once the predecessor has completed and its memory is
// visible (at once when there is no programmatic predecessor), so it comes
// before the first global-memory access.  pdl_release() lets the next
// kernel of the stream be scheduled early (it still waits in pdl_wait()).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- bulk asynchronous copies from global to shared memory
// cp.async.bulk moves a contiguous run of bytes (16-byte aligned at both
// ends, a multiple of 16 long) through the async proxy and reports its bytes
// to an mbarrier (complete_tx); a phase of the barrier completes when its
// one expected arrival (arrive.expect_tx, which also announces the bytes)
// has happened and all announced bytes have landed.

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the async proxy (before any copy)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// true once the phase with the given parity has completed (non-blocking)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}
// generic-proxy accesses of shared memory ordered before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Waits for a phase of `bar` with at most `limit` polls; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit) {
    for (unsigned it = 0; !mbar_test(bar, parity); ++it) {
        if (it >= limit) return false;
        __nanosleep(32);
    }
    return true;
}

// x / d for 0 <= x < 2^22 and d >= 1 from the correctly rounded reciprocal
// r = 1/d: floor((x + 1/2) r) is exact there (the half step keeps the product
// at least 1/(2d) away from the next integer, more than its rounding error),
// four instructions where an integer division by a run-time divisor takes
// about twenty.
__device__ __forceinline__ int udiv_small(int x, float r) {
    return (int)__fmul_rn(__fadd_rn((float)x, 0.5f), r);
}
__device__ __forceinline__ float recip(int d) { return __frcp_rn((float)d); }

// reflect about the edge pixel without repeating it (-1 -> 1, n -> n-2); n >= 3
__device__ __forceinline__ int refl(int i, int n) {
    i = i < 0 ? -i : i;
    return i >= n ? 2 * (n - 1) - i : i;
}

// Patch origin k along an axis of length n: k*S for the regular origins,
// n-P for the extra ragged one.
__device__ __forceinline__ int origin(int k, int n, int P, int S, int kreg) {
    return k < kreg ? k * S : n - P;
}

// Largest descriptor whose work range starts at or before `unit`.
__device__ __forceinline__ int find_pair(const LevelDesc *d, int n, int unit, int kind) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].work_begin[kind] <= unit) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Bilinear lookup of a coarse map at fine position (x, y): coarse
// coordinate (x + 0.5)/2 - 0.5, clamped to the map.
__device__ __forceinline__ float coarse_bilin(const float *__restrict__ m, int wc, int hc,
                                              float x, float y) {
    float X = (x + 0.5f) * 0.5f - 0.5f, Y = (y + 0.5f) * 0.5f - 0.5f;
    X = fminf(fmaxf(X, 0.f), (float)(wc - 1));
    Y = fminf(fmaxf(Y, 0.f), (float)(hc - 1));
    int x0 = (int)floorf(X), y0 = (int)floorf(Y);
    int x1 = min(x0 + 1, wc - 1), y1 = min(y0 + 1, hc - 1);
    float fx = X - (float)x0, fy = Y - (float)y0;
    // L2 loads: the map may have been written earlier in the same (persistent) launch
    float a = (1.f - fx) * __ldcg(m + (size_t)y0 * wc + x0) + fx * __ldcg(m + (size_t)y0 * wc + x1);
    float b = (1.f - fx) * __ldcg(m + (size_t)y1 * wc + x0) + fx * __ldcg(m + (size_t)y1 * wc + x1);
    return (1.f - fy) * a + fy * b;
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Split x - d into an integer base and a fraction: x - d = base + t with
// t in [0, 1), computed from d alone so it is exact for any x.
__device__ __forceinline__ void split_shift(float d, int &off, float &t) {
    float fl = floorf(d);
    float f = d - fl;                 // exact
    int di = (int)fl;
    if (f > 0.f) { off = -di - 1; t = 1.f - f; }
    else { off = -di; t = 0.f; }
}

}  // namespace
}  // namespace bdis
