// orca_peak.cu -- FP32 FMA throughput microbenchmark (measurement only; the paper has no
// counterpart).  The ORCA kernel is bound by plain FP32 issue, not by a dense contraction
// or HBM, so its arithmetic roofline needs the GPU's FP32 FMA rate as measured on the
// machine, under the clocks the machine runs at, rather than the nominal product of unit
// counts and the maximum clock.
//
// Every thread runs kChains independent FMA chains x <- x * m + c (m, c kernel arguments,
// so nothing folds at compile time) for `iters` rounds; with 8 CTAs of 256 threads per SM
// the 4 schedulers of an SM have 16 warps x kChains independent FMAs each to issue, which
// hides the FMA latency.  One float per CTA is written so the work stays live.
#include "../../include/orca_gb300.h"
#include "orca_common.cuh"

namespace orca {

constexpr int kFmaThreads = 256;
constexpr int kChains = 16;

__global__ void __launch_bounds__(kFmaThreads) fma_peak_kernel(int iters, float m, float c, float* out) {
    float x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = (float)(threadIdx.x + q) * 1e-3f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = __fmaf_rn(x[q], m, c);
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = __fmaf_rn(x[q], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float s_w[kFmaThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kFmaThreads / 32; ++w) t += s_w[w];
        out[blockIdx.x] = t;
    }
}

}  // namespace orca

using namespace orca;

extern "C" ORCA_API int orca_fma_bench(int32_t blocks, int32_t iters, float* out, int64_t* flops,
                                       void* stream) {
    if (!out || !flops || iters < 1) return ORCA_ERR_ARG;
    if (blocks <= 0) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ORCA_ERR_CUDA;
        blocks = 8 * sms;
    }
    fma_peak_kernel<<<blocks, kFmaThreads, 0, (cudaStream_t)stream>>>(iters, 0.99999994f, 1e-7f, out);
    if (cudaGetLastError() != cudaSuccess) return ORCA_ERR_CUDA;
    *flops = (int64_t)blocks * kFmaThreads * iters * (2 * kChains) * 2;
    return ORCA_OK;
}
