// FP32 FMA throughput of the device, measured by the library itself: the denominator of
// the compositing kernels' roofline (their work is FP32 arithmetic on the CUDA cores).
#include <cstdint>

#include <cuda_runtime.h>

#include "sgad.h"

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);
}

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

// Every thread runs kChains independent chains of `iters` dependent FMAs (2 flops each);
// the result is stored only when it could not be predicted, so nothing is optimised away.
__global__ void __launch_bounds__(kThreads) k_fma_burn(int iters, float seed, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.9999999f, k = 1e-7f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 1234.5f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" sgad_status sgad_fma_burn(int32_t blocks, int32_t iters, float *sink, double *flops, void *stream)
{
    if (blocks < 1 || iters < 1 || !sink || !flops)
        return sgad::report_error(SGAD_ERR_INVALID_ARG, "sgad_fma_burn: bad arguments");
    k_fma_burn<<<blocks, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.5f, sink);
    *flops = 2.0 * (double)blocks * kThreads * kChains * 16.0 * (double)iters;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGAD_OK : sgad::report_error(SGAD_ERR_CUDA, "sgad_fma_burn: launch failed");
}
