// bdis_probe.cu -- the L2 read-bandwidth probe behind bdis_probe_l2_read:
// the denominator of the L2 roofline fractions the benchmark reports (the
// HBM denominator is a measured device copy; the L2 has no such figure).
#include <cstdint>

#include "bdis_internal.cuh"

namespace bdis {
namespace {

// Every thread reads 16-byte words of the buffer in a grid-stride loop,
// `reps` times over the whole buffer, through L2 (L1 bypassed).  The XOR of
// the words is stored only when it equals a constant the buffer of the
// probe never produces, so the loads are kept and nothing is written.
__global__ void __launch_bounds__(256) k_l2_read(const uint4 *__restrict__ buf, size_t n16, int reps,
                                                 unsigned *__restrict__ sink) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    unsigned acc = 0u;
    for (int r = 0; r < reps; ++r) {
#pragma unroll 4
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9e3779b9u && sink != nullptr) sink[0] = acc;
}

}  // namespace
}  // namespace bdis

using namespace bdis;

extern "C" bdis_status bdis_probe_l2_read(const void *buf, size_t bytes, int reps, void *stream) {
    if (!buf || bytes < 16 || reps < 1 || ((uintptr_t)buf & 15u) != 0) return BDIS_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BDIS_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return BDIS_ECUDA;
    k_l2_read<<<sms * 8, 256, 0, (cudaStream_t)stream>>>((const uint4 *)buf, bytes / 16, reps,
                                                         nullptr);
    return cudaGetLastError() == cudaSuccess ? BDIS_OK : BDIS_ECUDA;
}
