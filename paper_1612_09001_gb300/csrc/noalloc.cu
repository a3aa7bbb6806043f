// Coefficient gradient for callers that may not allocate device memory.
//
// dpd_grad reduces the coefficient gradient through a per-handle workspace that
// dpd_create obtains with cudaMalloc.  This entry point needs no handle: its
// per-CTA partial rows live in a fixed array of device memory that belongs to
// the library image (g_partials below), so a call allocates nothing.  The
// array is reserved on every device that loads the library until the process
// exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/dpd.h"
#include "dpd_model.h"
#include "dpd_adj.cuh"

namespace {

constexpr int kRows = 512;                         // partial rows (one per CTA of a tap group)
constexpr int kMaxK = (6 + 6) * dpd::kMaxT + 1;    // 97: P = Q = 11, M = 7

// Shared by every call on a device; each call overwrites the rows it sums.
__device__ __align__(256) float2 g_partials[kRows * kMaxK];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float2 *g_partials_addr[kMaxDevices];   // device address of g_partials, per device
int g_sm_count[kMaxDevices];

// Once per device, with that device current: look up the device address of
// g_partials (the host-side name is only a stand-in for it).
dpd_status setup_device(int dev)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_partials_addr[dev]) return DPD_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || p == nullptr) return DPD_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DPD_ERR_CUDA;
    g_sm_count[dev] = sms;
    g_partials_addr[dev] = static_cast<float2 *>(p);
    return DPD_OK;
}

int nbranch(int order) { return order > 0 ? (order + 1) / 2 : 0; }

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

cudaError_t launch_gh(int B, const dpd::AdjArgs &a, const dpd::AdjLaunch &L, int T, int Bp, int Bq, int K,
                      cudaStream_t s)
{
    switch (B) {
    case 1: return dpd::launch_adj_gh<1>(a, L, T, Bp, Bq, K, s);
    case 2: return dpd::launch_adj_gh<2>(a, L, T, Bp, Bq, K, s);
    case 3: return dpd::launch_adj_gh<3>(a, L, T, Bp, Bq, K, s);
    case 4: return dpd::launch_adj_gh<4>(a, L, T, Bp, Bq, K, s);
    case 5: return dpd::launch_adj_gh<5>(a, L, T, Bp, Bq, K, s);
    case 6: return dpd::launch_adj_gh<6>(a, L, T, Bp, Bq, K, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" dpd_status dpd_grad_coeffs_noalloc(int P, int Q, int M, const void *x, const void *gy, int64_t n,
                                              void *gh, void *stream)
{
    const dpd_status mst = dpd::model_status(P, Q, M);
    if (mst != DPD_OK) return mst;
    if (n < 0 || !gh || !aligned8(gh)) return DPD_ERR_INVALID_ARGUMENT;
    const int Bp = nbranch(P), Bq = nbranch(Q), B = Bp > Bq ? Bp : Bq, T = M + 1;
    const int K = (Bp + Bq) * T + 1;
    if (K > kMaxK) return DPD_ERR_UNSUPPORTED;
    if (n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
    const size_t bytes = (size_t)n * sizeof(float2), kbytes = sizeof(float2) * K;
    if (n > 0) {
        if (!x || !gy || !aligned8(x) || !aligned8(gy)) return DPD_ERR_INVALID_ARGUMENT;
        if (overlap(gh, kbytes, x, bytes) || overlap(gh, kbytes, gy, bytes)) return DPD_ERR_INVALID_ARGUMENT;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DPD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DPD_ERR_UNSUPPORTED;
    dpd_status st = setup_device(dev);
    if (st != DPD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return cudaMemsetAsync(gh, 0, kbytes, s) == cudaSuccess ? DPD_OK : DPD_ERR_CUDA;

    // One partial row per CTA; every row that is summed is fully written by
    // this call, so nothing has to be cleared first.
    int64_t rows = (n + 1023) / 1024;
    if (rows > 2 * (int64_t)g_sm_count[dev]) rows = 2 * (int64_t)g_sm_count[dev];
    if (rows > kRows) rows = kRows;
    if (rows < 1) rows = 1;
    if (rows * K > (int64_t)kRows * kMaxK) return DPD_ERR_UNSUPPORTED;

    dpd::AdjArgs a;
    a.x = static_cast<const float2 *>(x);
    a.gy = static_cast<const float2 *>(gy);
    a.n = n;
    a.gx = nullptr;
    a.partials = g_partials_addr[dev];
    a.adj_tab = nullptr;
    a.status = nullptr;
    dpd::AdjLaunch L;
    L.gh_blocks = (int)rows;
    L.tap_group = B <= 2 ? 4 : 2;
    if (launch_gh(B, a, L, T, Bp, Bq, K, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (dpd::launch_adj_finalize(a.partials, (int)rows, K, static_cast<float2 *>(gh), s) != cudaSuccess)
        return DPD_ERR_CUDA;
    return DPD_OK;
}
