// Zero-copy forward filter: the kernel reads the input from and writes the
// output to pinned host memory mapped into the device address space, with no
// staging copy (the zero-copy access of Sec. 3.3.1, here over the CPU-GPU
// link of a Grace host).  Host memory is reached through the link at cache-line
// granularity, so every byte must cross it exactly once and in whole lines:
// each CTA stages its tile of S samples plus the kHalo history samples in
// front with coalesced 16-byte loads (the tile overlap is the only re-read,
// kHalo / S of the input), computes from shared memory, stages the outputs in
// shared memory and writes them back with coalesced 16-byte stores.  One tile
// per CTA, many CTAs per SM: the loads of resident CTAs keep the link busy
// while others compute.
#pragma once

#include "dpd_fwd.cuh"
#include "dpd_zc.h"

namespace dpd {

constexpr int kZcThreads = 256;
constexpr int kZcV = 8;
constexpr int kZcTile = kZcThreads * kZcV;   // samples per CTA

template <int B, int T, int MODE>
__global__ void __launch_bounds__(kZcThreads)
    fwd_zc_kernel(FwdArgs a, const __grid_constant__ ParamTab<B, T> ptab)
{
    constexpr int V = kZcV, S = kZcTile, W = V + T - 1;
    constexpr int TABF = wl_table_floats(B, T);
    constexpr int NIN4 = (kHalo + S) / 2;                       // float4 of the staged input
    constexpr int PER = (NIN4 + kZcThreads - 1) / kZcThreads;   // loads per thread
    __shared__ __align__(16) float2 xin[kHalo + S];             // samples s0 - kHalo .. s0 + S - 1
    __shared__ __align__(16) float2 yout[S];
    __shared__ __align__(16) float tab[(MODE & kModeParamCoef) ? 4 : ((TABF + 3) / 4) * 4];
    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * S;

    // Stage the input: element pair (g, g + 1), g = s0 - kHalo + 2 i, zero outside [0, n).
    float4 v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = tid + q * kZcThreads;
        const int64_t g = s0 - kHalo + 2 * (int64_t)i;
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < NIN4 && g >= 0) {
            if (g + 1 < a.n) {
                v[q] = *reinterpret_cast<const float4 *>(a.x + g);
            } else if (g < a.n) {
                const float2 u = a.x[g];
                v[q] = make_float4(u.x, u.y, 0.f, 0.f);
            }
        }
    }
    if constexpr ((MODE & kModeParamCoef) == 0)
        for (int i = tid; i < TABF; i += kZcThreads) tab[i] = a.tab[i];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = tid + q * kZcThreads;
        if (i < NIN4) reinterpret_cast<float4 *>(xin)[i] = v[q];
    }
    __syncthreads();

    // Window of thread tid: samples s0 + tid V - (T-1) .. s0 + tid V + V - 1,
    // read as 16-byte pairs from a pair-aligned start.
    constexpr int MP = ((T - 1) + 1) & ~1;
    constexpr int E = V + MP;
    constexpr int D = MP - (T - 1);
    const float4 *src = reinterpret_cast<const float4 *>(xin + tid * V + kHalo - MP);
    float er[E], ei[E];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
        const float4 q = src[i];
        er[2 * i] = q.x;
        ei[2 * i] = q.y;
        er[2 * i + 1] = q.z;
        ei[2 * i + 1] = q.w;
    }
    float wr[W], wi[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        wr[j] = er[j + D];
        wi[j] = ei[j + D];
    }
    float yr[V], yi[V];
    fwd_compute<B, T, V, MODE>(tab, ptab, wr, wi, yr, yi);
#pragma unroll
    for (int i = 0; i < V / 2; ++i)
        reinterpret_cast<float4 *>(yout + tid * V)[i] = make_float4(yr[2 * i], yi[2 * i], yr[2 * i + 1], yi[2 * i + 1]);
    __syncthreads();

    // Coalesced write-back of the S outputs (pairs), clipped at n.
#pragma unroll
    for (int q = 0; q < S / 2 / kZcThreads; ++q) {
        const int i = tid + q * kZcThreads;
        const int64_t g = s0 + 2 * (int64_t)i;
        const float4 w = reinterpret_cast<const float4 *>(yout)[i];
        if (g + 1 < a.n)
            *reinterpret_cast<float4 *>(a.y + g) = w;
        else if (g < a.n)
            a.y[g] = make_float2(w.x, w.y);
    }
}

template <int B, int T, int MODE>
cudaError_t launch_zc_tm(const FwdArgs &a, cudaStream_t s)
{
    ParamTab<B, T> ptab{};
    if constexpr ((MODE & kModeParamCoef) != 0) {
        if (!a.host_tab) return cudaErrorInvalidValue;
        for (int i = 0; i < wl_table_floats(B, T); ++i) ptab.v[i] = a.host_tab->v[i];
    }
    const int64_t grid = (a.n + kZcTile - 1) / kZcTile;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    fwd_zc_kernel<B, T, MODE><<<(unsigned)grid, kZcThreads, 0, s>>>(a, ptab);
    count_launch();
    return cudaGetLastError();
}

template <int B, int T>
cudaError_t launch_zc_t(const FwdArgs &a, bool param_coef, cudaStream_t s)
{
    return param_coef ? launch_zc_tm<B, T, kModePackedFma | kModeParamCoef>(a, s)
                      : launch_zc_tm<B, T, kModePackedFma>(a, s);
}

#define DPD_DEFINE_LAUNCH_ZC(BB)                                                                   \
    template <>                                                                                    \
    cudaError_t launch_zc<BB>(int T, const FwdArgs &a, bool param_coef, cudaStream_t s)            \
    {                                                                                              \
        switch (T) {                                                                               \
        case 1: return launch_zc_t<BB, 1>(a, param_coef, s);                                       \
        case 2: return launch_zc_t<BB, 2>(a, param_coef, s);                                       \
        case 3: return launch_zc_t<BB, 3>(a, param_coef, s);                                       \
        case 4: return launch_zc_t<BB, 4>(a, param_coef, s);                                       \
        case 5: return launch_zc_t<BB, 5>(a, param_coef, s);                                       \
        case 6: return launch_zc_t<BB, 6>(a, param_coef, s);                                       \
        case 7: return launch_zc_t<BB, 7>(a, param_coef, s);                                       \
        case 8: return launch_zc_t<BB, 8>(a, param_coef, s);                                       \
        default: return cudaErrorInvalidValue;                                                     \
        }                                                                                          \
    }

}  // namespace dpd
