// Measurement aid: a kernel that does nothing but FP32 fused multiply-adds, so
// that the ceiling of the FMA pipe that bounds the filter and adjoint kernels
// is measured on the GPU at hand (with its clock) instead of taken from
// nominal lane counts.  Every thread runs independent chains x <- x m + c,
// which no compiler can fold, and writes one float so that none is dead code.
#include <cuda_runtime.h>

#include "../../include/dpd.h"
#include "dpd_internal.h"

namespace dpd {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 16;   // FMAs per iteration and thread

template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, float *__restrict__ sink)
{
    const float s = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
    float out = 0.f;
    if constexpr (PACKED) {
        float2 a[kProbeChains / 2];
#pragma unroll
        for (int j = 0; j < kProbeChains / 2; ++j) a[j] = make_float2(s + (float)j, s - (float)j);
        const float2 m = make_float2(0.99993f, 1.00007f), c = make_float2(1e-6f, -1e-6f);
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kProbeChains / 2; ++j) a[j] = __ffma2_rn(a[j], m, c);
        }
#pragma unroll
        for (int j = 0; j < kProbeChains / 2; ++j) out += a[j].x + a[j].y;
    } else {
        float a[kProbeChains];
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) a[j] = s + (float)j;
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kProbeChains; ++j) a[j] = fmaf(a[j], 0.99993f, 1e-6f);
        }
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) out += a[j];
    }
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = out;
}

}  // namespace
}  // namespace dpd

extern "C" dpd_status dpd_probe_fma(int blocks, int iters, int packed, void *sink, void *stream)
{
    if (blocks < 1 || iters < 0 || !sink || (reinterpret_cast<uintptr_t>(sink) & 3u) != 0)
        return DPD_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *out = static_cast<float *>(sink);
    if (packed)
        dpd::fma_probe_kernel<true><<<blocks, dpd::kProbeThreads, 0, s>>>(iters, out);
    else
        dpd::fma_probe_kernel<false><<<blocks, dpd::kProbeThreads, 0, s>>>(iters, out);
    dpd::count_launch();
    return cudaGetLastError() == cudaSuccess ? DPD_OK : DPD_ERR_CUDA;
}
