// Throughput probe of the FP32 fused multiply-add pipe (a measurement helper; the
// paper has no counterpart).  The accelerated kernels are bound by FP32 FMA issue,
// and the GPU's FP32 rate is not among the measured peaks, so the benchmark times
// this kernel on the same GPU, at the same clock, to obtain the denominator of
// their roofline.  Every thread runs kChains independent dependency chains of
// a <- a * m + c, as scalar FFMA or as packed f32x2 FMA (two lanes per
// instruction); the chains are independent so that the pipe, not the latency of
// one chain, limits the rate.  With m = 1 - 2^-20 and c = 2^-20 every value stays
// in [0, 1], so no denormal or overflow changes the timing.
#include "accel_common.cuh"
#include "../../include/rcscm_probe.h"

namespace rcscm {
namespace {

constexpr int kChains = 16;

template <bool PACKED>
__global__ void __launch_bounds__(256) fma_probe_kernel(long long n_loops, float* sink) {
    const float m = 1.0f - 9.5367431640625e-07f, c = 9.5367431640625e-07f;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if constexpr (PACKED) {
        f32x2 a[kChains / 2];
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) a[k] = pk(0.001f * (float)((t + 2 * k) & 255), 0.002f * (float)k);
        const f32x2 M2 = pk(m, m), C2 = pk(c, c);
        for (long long i = 0; i < n_loops; ++i) {
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) a[k] = fma2(a[k], M2, C2);
        }
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) acc += lo_of(a[k]) + hi_of(a[k]);
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 0.001f * (float)((t + k) & 255);
        for (long long i = 0; i < n_loops; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += a[k];
    }
    if (acc == -1.0f) sink[t] = acc;     // never true; keeps the chains live
}

}  // namespace
}  // namespace rcscm

extern "C" int rcscm_probe_fma(int packed, int n_blocks, long long n_loops, float* sink, void* stream,
                               double* lane_ops) {
    if (n_blocks < 1 || n_loops < 1 || !sink) return RCSCM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (packed)
        rcscm::fma_probe_kernel<true><<<n_blocks, 256, 0, s>>>(n_loops, sink);
    else
        rcscm::fma_probe_kernel<false><<<n_blocks, 256, 0, s>>>(n_loops, sink);
    if (lane_ops) *lane_ops = (double)n_blocks * 256.0 * (double)n_loops * (double)rcscm::kChains;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RCSCM_OK : RCSCM_ECUDA;
}
