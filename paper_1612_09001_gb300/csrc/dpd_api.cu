// libdpd C ABI: handle management, argument checks and kernel dispatch.
// Declarations and the contract of every entry point are in include/dpd.h.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/dpd.h"
#include "dpd_model.h"
#include "dpd_internal.h"

static_assert(dpd::kModelMaxOrder == 2 * dpd::kMaxB - 1 && dpd::kModelMaxTaps == dpd::kMaxT,
              "model limits match the kernels' limits");

#include "dpd_handle.h"
#include "dpd_zc.h"

namespace dpd {
static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

cudaError_t launch_adj_any(int B, const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K,
                           int sm_count, cudaStream_t s)
{
    switch (B) {
    case 1: return launch_adj<1>(a, L, T, Bp, Bq, K, sm_count, s);
    case 2: return launch_adj<2>(a, L, T, Bp, Bq, K, sm_count, s);
    case 3: return launch_adj<3>(a, L, T, Bp, Bq, K, sm_count, s);
    case 4: return launch_adj<4>(a, L, T, Bp, Bq, K, sm_count, s);
    case 5: return launch_adj<5>(a, L, T, Bp, Bq, K, sm_count, s);
    case 6: return launch_adj<6>(a, L, T, Bp, Bq, K, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj_gh_many_any(int B, const AdjArgs *args, int count, int blocks, int tap_group, int T, int Bp,
                                   int Bq, int K, cudaStream_t s)
{
    switch (B) {
    case 1: return launch_adj_gh_many<1>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    case 2: return launch_adj_gh_many<2>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    case 3: return launch_adj_gh_many<3>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    case 4: return launch_adj_gh_many<4>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    case 5: return launch_adj_gh_many<5>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    case 6: return launch_adj_gh_many<6>(args, count, blocks, tap_group, T, Bp, Bq, K, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zc_any(int B, int T, const FwdArgs &a, bool param_coef, cudaStream_t s)
{
    switch (B) {
    case 1: return launch_zc<1>(T, a, param_coef, s);
    case 2: return launch_zc<2>(T, a, param_coef, s);
    case 3: return launch_zc<3>(T, a, param_coef, s);
    case 4: return launch_zc<4>(T, a, param_coef, s);
    case 5: return launch_zc<5>(T, a, param_coef, s);
    case 6: return launch_zc<6>(T, a, param_coef, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fwd_any(int B, int T, const FwdArgs &a, const FwdLaunch &L, int sm_count,
                           cudaStream_t s)
{
    switch (B) {
    case 1: return launch_fwd<1>(T, a, L, sm_count, s);
    case 2: return launch_fwd<2>(T, a, L, sm_count, s);
    case 3: return launch_fwd<3>(T, a, L, sm_count, s);
    case 4: return launch_fwd<4>(T, a, L, sm_count, s);
    case 5: return launch_fwd<5>(T, a, L, sm_count, s);
    case 6: return launch_fwd<6>(T, a, L, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace dpd

namespace {

int nbranch(int order) { return order > 0 ? (order + 1) / 2 : 0; }

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

dpd_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DPD_OK : DPD_ERR_CUDA; }

}  // namespace

extern "C" {

const char *dpd_status_string(dpd_status s)
{
    switch (s) {
    case DPD_OK: return "DPD_OK";
    case DPD_ERR_INVALID_ARGUMENT: return "DPD_ERR_INVALID_ARGUMENT";
    case DPD_ERR_UNSUPPORTED: return "DPD_ERR_UNSUPPORTED";
    case DPD_ERR_NO_COEFFS: return "DPD_ERR_NO_COEFFS";
    case DPD_ERR_CUDA: return "DPD_ERR_CUDA";
    case DPD_ERR_ALLOC: return "DPD_ERR_ALLOC";
    case DPD_ERR_NOT_SPD: return "DPD_ERR_NOT_SPD";
    case DPD_ERR_TIMEOUT: return "DPD_ERR_TIMEOUT";
    }
    return "DPD_ERR_UNKNOWN";
}

uint64_t dpd_kernel_launches(void) { return dpd::g_launches.load(std::memory_order_relaxed); }

dpd_status dpd_create(int P, int Q, int M, dpd_handle *out)
{
    if (!out) return DPD_ERR_INVALID_ARGUMENT;
    const dpd_status mst = dpd::model_status(P, Q, M);
    if (mst != DPD_OK) return mst;
    dpd_filter *f = new (std::nothrow) dpd_filter();
    if (!f) return DPD_ERR_ALLOC;
    f->P = P;
    f->Q = Q;
    f->M = M;
    f->Bp = nbranch(P);
    f->Bq = nbranch(Q);
    f->B = f->Bp > f->Bq ? f->Bp : f->Bq;
    f->T = M + 1;
    f->K = (f->Bp + f->Bq) * f->T + 1;
    f->has_coeffs = false;
    f->host_tab_valid = false;
    if (cudaGetDevice(&f->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&f->sm_count, cudaDevAttrMultiProcessorCount, f->device) != cudaSuccess) {
        delete f;
        return DPD_ERR_CUDA;
    }
    f->rows_max = 4 * f->sm_count;
    // Coefficient-gradient schedule: as few tap groups as keep a thread's
    // accumulators (4 B TG + 2 floats) within about a hundred registers, with
    // the taps spread evenly over the groups, and the CTAs of all groups in one
    // wave of one CTA per SM (the staged kernel's ring takes most of an SM's
    // shared memory): sm_count / groups CTAs per group.
    {
        int tg_max = 25 / f->B;
        if (tg_max > 5) tg_max = 5;
        if (tg_max < 1) tg_max = 1;
        const int groups = (f->T + tg_max - 1) / tg_max;
        f->adj.tap_group = (f->T + groups - 1) / groups;
        f->adj.gh_blocks = f->sm_count / groups > 0 ? f->sm_count / groups : 1;
    }
    f->d_h = nullptr;
    f->d_tab = nullptr;
    f->d_status = nullptr;
    f->d_adj_tab = nullptr;
    f->d_partials = nullptr;
    f->d_hist = nullptr;
    f->d_loss_part = nullptr;
    if (cudaMalloc(&f->d_h, sizeof(float2) * f->K) != cudaSuccess ||
        cudaMalloc(&f->d_tab, sizeof(float) * dpd::wl_table_floats(f->B, f->T)) != cudaSuccess ||
        cudaMalloc(&f->d_adj_tab, sizeof(float) * dpd::adj_table_floats(f->B, f->T)) != cudaSuccess ||
        cudaMalloc(&f->d_partials, sizeof(float2) * (size_t)f->rows_max * f->K) != cudaSuccess ||
        cudaMalloc(&f->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&f->d_hist, sizeof(float2) * dpd::kHalo) != cudaSuccess ||
        cudaMalloc(&f->d_loss_part, sizeof(double) * dpd::kLossBlocks) != cudaSuccess) {
        dpd_destroy(f);
        return DPD_ERR_ALLOC;
    }
    if (cudaMallocHost(&f->h_tab_pin, sizeof(float) * dpd::wl_table_floats(f->B, f->T)) != cudaSuccess ||
        cudaMallocHost(&f->h_adj_pin, sizeof(float) * dpd::adj_table_floats(f->B, f->T)) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->ev_tab, cudaEventDisableTiming) != cudaSuccess) {
        dpd_destroy(f);
        return DPD_ERR_ALLOC;
    }
    if (cudaMemset(f->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(f->d_hist, 0, sizeof(float2) * dpd::kHalo) != cudaSuccess) {
        dpd_destroy(f);
        return DPD_ERR_CUDA;
    }
    *out = f;
    return DPD_OK;
}

dpd_status dpd_destroy(dpd_handle h)
{
    if (!h) return DPD_OK;
    cudaFree(h->d_h);
    cudaFree(h->d_tab);
    cudaFree(h->d_adj_tab);
    cudaFree(h->d_partials);
    cudaFree(h->d_status);
    cudaFree(h->d_hist);
    cudaFree(h->d_loss_part);
    cudaFreeHost(h->h_tab_pin);
    cudaFreeHost(h->h_adj_pin);
    if (h->ev_tab) cudaEventDestroy(h->ev_tab);
    free_estimate_workspace(h->est);
    free_host_pipeline(h->host);
    delete h;
    return DPD_OK;
}

namespace {

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// Whether launches on `s` may pass the coefficient tables by value (kernel
// parameter bank).  Coefficients set from host memory: always.  Coefficients
// set from device memory: once the queued copy of the derived tables back to
// host memory has landed, and not while `s` is being captured -- a captured
// graph then keeps reading the tables on the device at every replay, as it
// did before the copy existed.
bool param_tables(dpd_handle h, cudaStream_t s)
{
    if (h->tab_pending && !capturing(s)) {
        const cudaError_t q = cudaEventQuery(h->ev_tab);
        if (q == cudaSuccess) {
            std::memcpy(h->h_tab.v, h->h_tab_pin, sizeof(float) * dpd::wl_table_floats(h->B, h->T));
            std::memcpy(h->h_adj_tab, h->h_adj_pin, sizeof(float) * dpd::adj_table_floats(h->B, h->T));
            h->host_tab_valid = true;
            h->tab_from_device = true;
            h->tab_pending = false;
        } else if (q != cudaErrorNotReady) {
            (void)cudaGetLastError();   // the copy failed: keep reading the device tables
            h->tab_pending = false;
        }
    }
    return h->host_tab_valid && !(h->tab_from_device && capturing(s));
}

}  // namespace

dpd_status dpd_num_coeffs(dpd_handle h, int *K)
{
    if (!h || !K) return DPD_ERR_INVALID_ARGUMENT;
    *K = h->K;
    return DPD_OK;
}

dpd_status dpd_set_coeffs(dpd_handle h, const void *coeffs, int K, int where, void *stream)
{
    if (!h || !coeffs || K != h->K) return DPD_ERR_INVALID_ARGUMENT;
    if (where != DPD_HOST && where != DPD_DEVICE) return DPD_ERR_INVALID_ARGUMENT;
    if (!aligned(coeffs, 4)) return DPD_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2 *src = static_cast<const float2 *>(coeffs);
    if (where == DPD_HOST) {
        cudaError_t e = cudaMemcpyAsync(h->d_h, coeffs, sizeof(float2) * K, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return DPD_ERR_CUDA;
        src = h->d_h;
    } else if (!aligned(coeffs, 8)) {
        return DPD_ERR_INVALID_ARGUMENT;
    } else if (src != h->d_h) {
        cudaError_t e = cudaMemcpyAsync(h->d_h, coeffs, sizeof(float2) * K, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return DPD_ERR_CUDA;
        src = h->d_h;
    }
    h->host_tab_valid = false;
    h->tab_from_device = false;
    h->tab_pending = false;
    cudaError_t e = dpd::launch_wl_table(src, h->Bp, h->Bq, h->T, h->d_tab, h->d_adj_tab, s);
    if (e != cudaSuccess) return DPD_ERR_CUDA;
    if (where == DPD_DEVICE && !capturing(s)) {
        // Copy the derived tables back to pinned host memory without waiting:
        // later calls pass them by value once the copy has landed.
        if (cudaMemcpyAsync(h->h_tab_pin, h->d_tab, sizeof(float) * dpd::wl_table_floats(h->B, h->T),
                            cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemcpyAsync(h->h_adj_pin, h->d_adj_tab, sizeof(float) * dpd::adj_table_floats(h->B, h->T),
                            cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaEventRecord(h->ev_tab, s) == cudaSuccess)
            h->tab_pending = true;
        else
            return DPD_ERR_CUDA;
    }
    if (where == DPD_HOST) {
        // Keep host copies of the tables so that dpd_apply and dpd_grad can pass
        // them by value.
        e = cudaMemcpyAsync(h->h_tab.v, h->d_tab, sizeof(float) * dpd::wl_table_floats(h->B, h->T),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->h_adj_tab, h->d_adj_tab, sizeof(float) * dpd::adj_table_floats(h->B, h->T),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return DPD_ERR_CUDA;
        h->host_tab_valid = true;
    }
    h->has_coeffs = true;
    return DPD_OK;
}

// Launch shape for n samples.  With the default shape, an input too short to
// give every SM a few tiles gets 4 samples per thread and fewer warps per tile
// (tiles of 128 to 512 samples): such calls are bound by latency, and more,
// smaller tiles spread them over more SMs.
static dpd::FwdLaunch launch_for(dpd_handle h, int64_t n, bool param_tab)
{
    dpd::FwdLaunch L = h->fwd;
    if (!param_tab) L.mode &= ~dpd::kModeParamCoef;
    const int64_t tile = (int64_t)L.warps * 32 * L.V;
    if (h->fwd_auto && (n + tile - 1) / tile < 4 * (int64_t)h->sm_count) {
        L.V = 4;
        L.warps = 1;
        for (int w : {4, 2})
            if ((n + w * 128 - 1) / (w * 128) * 2 >= 3 * (int64_t)h->sm_count) {
                L.warps = w;
                break;
            }
        L.stages = L.warps >= 4 ? 3 : 2;
        L.group = 0;
    }
    return L;
}

dpd_status dpd_apply(dpd_handle h, const void *x, void *y, int64_t n, void *stream)
{
    if (!h || n < 0) return DPD_ERR_INVALID_ARGUMENT;
    if (!h->has_coeffs) return DPD_ERR_NO_COEFFS;
    if (n == 0) return DPD_OK;
    if (!x || !y || !aligned(x, 8) || !aligned(y, 8)) return DPD_ERR_INVALID_ARGUMENT;
    if (n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
    const size_t bytes = (size_t)n * sizeof(float2);
    if (overlap(x, bytes, y, bytes)) return DPD_ERR_INVALID_ARGUMENT;
    dpd::FwdArgs a;
    a.x = static_cast<const float2 *>(x);
    a.y = static_cast<float2 *>(y);
    a.n = n;
    a.tab = h->d_tab;
    a.status = h->d_status;
    a.vec_store = aligned(y, 16) ? 1 : 0;
    const bool pt = param_tables(h, static_cast<cudaStream_t>(stream));
    a.host_tab = pt ? &h->h_tab : nullptr;
    dpd::FwdLaunch L = launch_for(h, n, pt);
    if (!aligned(x, 16)) {
        // 8-byte aligned input: plain-load kernel (built for V = 4)
        L.use_tma = 0;
        L.V = 4;
    }
    return cuda_status(dpd::launch_fwd_any(h->B, h->T, a, L, h->sm_count, static_cast<cudaStream_t>(stream)));
}

dpd_status dpd_grad(dpd_handle h, const void *x, const void *gy, int64_t n, void *gh, void *gx,
                    void *stream)
{
    if (!h || n < 0) return DPD_ERR_INVALID_ARGUMENT;
    if (!gh && !gx) return DPD_ERR_INVALID_ARGUMENT;
    if (gx && !h->has_coeffs) return DPD_ERR_NO_COEFFS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (gh && !aligned(gh, 8)) return DPD_ERR_INVALID_ARGUMENT;
    if (n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
    const size_t bytes = (size_t)n * sizeof(float2), kbytes = sizeof(float2) * h->K;
    if (n > 0) {
        if (!x || !gy || !aligned(x, 8) || !aligned(gy, 8)) return DPD_ERR_INVALID_ARGUMENT;
        if (gx && (!aligned(gx, 8) || overlap(gx, bytes, x, bytes) || overlap(gx, bytes, gy, bytes)))
            return DPD_ERR_INVALID_ARGUMENT;
        if (gh && (overlap(gh, kbytes, x, bytes) || overlap(gh, kbytes, gy, bytes) ||
                   (gx && overlap(gh, kbytes, gx, bytes))))
            return DPD_ERR_INVALID_ARGUMENT;
    }
    if (n == 0) {
        if (gh && cudaMemsetAsync(gh, 0, kbytes, s) != cudaSuccess) return DPD_ERR_CUDA;
        return DPD_OK;
    }
    dpd::AdjArgs a;
    a.x = static_cast<const float2 *>(x);
    a.gy = static_cast<const float2 *>(gy);
    a.n = n;
    a.gx = static_cast<float2 *>(gx);
    a.partials = gh ? h->d_partials : nullptr;
    a.adj_tab = h->d_adj_tab;
    a.status = h->d_status;
    a.host_adj_tab = param_tables(h, s) ? h->h_adj_tab : nullptr;
    dpd::AdjLaunch L = h->adj;
    int64_t need = (n + 1023) / 1024;
    if (L.gh_blocks > need) L.gh_blocks = (int)need;
    if (L.gh_blocks > h->rows_max) L.gh_blocks = h->rows_max;
    if (L.gh_blocks < 1) L.gh_blocks = 1;
    cudaError_t e = dpd::launch_adj_any(h->B, a, L, h->T, h->Bp, h->Bq, h->K, h->sm_count, s);
    if (e != cudaSuccess) return DPD_ERR_CUDA;
    if (gh) {
        e = dpd::launch_adj_finalize(h->d_partials, L.gh_blocks, h->K, static_cast<float2 *>(gh), s);
        if (e != cudaSuccess) return DPD_ERR_CUDA;
    }
    return DPD_OK;
}

namespace {

// Host pointer kinds: 0 pinned / registered / managed (device-accessible), 1 pageable, -1 device or error.
int host_kind(const void *p, void **dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged) {
        *dev = at.devicePointer;
        return at.devicePointer ? 0 : -1;
    }
    if (at.type == cudaMemoryTypeUnregistered) {
        *dev = const_cast<void *>(p);
        return 1;
    }
    return -1;
}

dpd_status apply_zero_copy(dpd_handle h, const void *x, void *y, int64_t n, cudaStream_t stream);
dpd_status apply_pipelined(dpd_handle h, const void *x, void *y, int64_t n, cudaStream_t stream);

}  // namespace

dpd_status dpd_apply_host(dpd_handle h, const void *x, void *y, int64_t n, int mode, void *stream)
{
    if (!h || n < 0) return DPD_ERR_INVALID_ARGUMENT;
    if (mode != DPD_HOST_PIPELINED && mode != DPD_HOST_ZERO_COPY) return DPD_ERR_INVALID_ARGUMENT;
    if (!h->has_coeffs) return DPD_ERR_NO_COEFFS;
    if (n == 0) return DPD_OK;
    if (!x || !y || !aligned(x, 8) || !aligned(y, 8)) return DPD_ERR_INVALID_ARGUMENT;
    if (n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
    const size_t bytes = (size_t)n * sizeof(float2);
    if (overlap(x, bytes, y, bytes)) return DPD_ERR_INVALID_ARGUMENT;
    void *dx = nullptr, *dy = nullptr;
    const int kx = host_kind(x, &dx), ky = host_kind(y, &dy);
    if (kx < 0 || ky < 0) return DPD_ERR_INVALID_ARGUMENT;   // device memory: use dpd_apply
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode == DPD_HOST_ZERO_COPY) return apply_zero_copy(h, x, y, n, s);
    return apply_pipelined(h, x, y, n, s);
}

namespace {

dpd_status apply_zero_copy(dpd_handle h, const void *x, void *y, int64_t n, cudaStream_t stream)
{
    // Resolve each buffer to an address the kernel can dereference.
    const void *ptrs[2] = {x, y};
    void *dev[2] = {nullptr, nullptr};
    int pageable_ok = 0;
    if (cudaDeviceGetAttribute(&pageable_ok, cudaDevAttrPageableMemoryAccess, h->device) != cudaSuccess)
        return DPD_ERR_CUDA;
    for (int i = 0; i < 2; ++i) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
            cudaGetLastError();
            return DPD_ERR_INVALID_ARGUMENT;
        }
        if (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged) {
            if (!at.devicePointer) return DPD_ERR_INVALID_ARGUMENT;
            dev[i] = at.devicePointer;
        } else if (at.type == cudaMemoryTypeUnregistered && pageable_ok) {
            dev[i] = const_cast<void *>(ptrs[i]);
        } else {
            return DPD_ERR_INVALID_ARGUMENT;   // device memory: use dpd_apply
        }
    }
    dpd::FwdArgs a;
    a.x = static_cast<const float2 *>(dev[0]);
    a.y = static_cast<float2 *>(dev[1]);
    a.n = n;
    a.tab = h->d_tab;
    a.status = h->d_status;
    a.vec_store = 0;
    const bool pt = param_tables(h, stream);
    a.host_tab = pt ? &h->h_tab : nullptr;
    if (aligned(a.x, 16) && aligned(a.y, 16))   // staged, coalesced 16-byte accesses
        return cuda_status(dpd::launch_zc_any(h->B, h->T, a, pt, stream));
    dpd::FwdLaunch L = h->fwd;
    L.use_tma = 0;   // 8-byte aligned buffers: plain loads and stores straight to host memory
    L.V = 4;
    L.mode &= dpd::kModePackedFma | (pt ? dpd::kModeParamCoef : 0);
    return cuda_status(dpd::launch_fwd_any(h->B, h->T, a, L, h->sm_count, stream));
}

constexpr int64_t kHostChunk = (int64_t)1 << 21;

dpd_status ensure_pipeline(dpd_handle h)
{
    HostPipeline &P = h->host;
    if (P.chunk) return DPD_OK;
    for (int i = 0; i < kHostSlots; ++i) {
        if (cudaMalloc(&P.in[i], sizeof(float2) * (kHostChunk + dpd::kHalo)) != cudaSuccess ||
            cudaMalloc(&P.out[i], sizeof(float2) * (kHostChunk + dpd::kHalo)) != cudaSuccess) {
            free_host_pipeline(P);
            return DPD_ERR_ALLOC;
        }
        if (cudaStreamCreateWithFlags(&P.streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P.done[i], cudaEventDisableTiming) != cudaSuccess) {
            free_host_pipeline(P);
            return DPD_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming) != cudaSuccess) {
        free_host_pipeline(P);
        return DPD_ERR_CUDA;
    }
    P.chunk = kHostChunk;
    return DPD_OK;
}

// Chunks of the input are copied in (with kHalo samples of history), filtered
// and copied out on kHostSlots streams in turn, so host-to-device copies,
// kernels and device-to-host copies of different chunks overlap.  Ordered
// after `stream`'s earlier work; `stream` waits for every chunk at the end.
dpd_status apply_pipelined(dpd_handle h, const void *x, void *y, int64_t n, cudaStream_t stream)
{
    dpd_status st = ensure_pipeline(h);
    if (st != DPD_OK) return st;
    HostPipeline &P = h->host;
    const bool pt = param_tables(h, stream);
    if (cudaEventRecord(P.start, stream) != cudaSuccess) return DPD_ERR_CUDA;
    for (int i = 0; i < kHostSlots; ++i)
        if (cudaStreamWaitEvent(P.streams[i], P.start, 0) != cudaSuccess) return DPD_ERR_CUDA;
    const float2 *xs = static_cast<const float2 *>(x);
    float2 *ys = static_cast<float2 *>(y);
    const int64_t nchunks = (n + P.chunk - 1) / P.chunk;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int slot = (int)(c % kHostSlots);
        cudaStream_t s = P.streams[slot];
        const int64_t c0 = c * P.chunk, len = std::min(P.chunk, n - c0);
        const int64_t hs = std::min<int64_t>(c0, dpd::kHalo);   // history samples copied in front
        if (cudaMemcpyAsync(P.in[slot], xs + c0 - hs, sizeof(float2) * (hs + len), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return DPD_ERR_CUDA;
        dpd::FwdArgs a;
        a.x = P.in[slot];
        a.y = P.out[slot];
        a.n = hs + len;
        a.tab = h->d_tab;
        a.status = h->d_status;
        a.vec_store = 1;
        a.host_tab = pt ? &h->h_tab : nullptr;
        dpd::FwdLaunch L = h->fwd;
        if (!pt) L.mode &= ~dpd::kModeParamCoef;
        if (dpd::launch_fwd_any(h->B, h->T, a, L, h->sm_count, s) != cudaSuccess) return DPD_ERR_CUDA;
        if (cudaMemcpyAsync(ys + c0, P.out[slot] + hs, sizeof(float2) * len, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return DPD_ERR_CUDA;
    }
    for (int i = 0; i < kHostSlots; ++i)
        if (cudaEventRecord(P.done[i], P.streams[i]) != cudaSuccess || cudaStreamWaitEvent(stream, P.done[i], 0) != cudaSuccess)
            return DPD_ERR_CUDA;
    return DPD_OK;
}

}  // namespace

extern "C++" void free_host_pipeline(HostPipeline &P)
{
    for (int i = 0; i < kHostSlots; ++i) {
        cudaFree(P.in[i]);
        cudaFree(P.out[i]);
        if (P.streams[i]) cudaStreamDestroy(P.streams[i]);
        if (P.done[i]) cudaEventDestroy(P.done[i]);
    }
    if (P.start) cudaEventDestroy(P.start);
    P = HostPipeline();
}

dpd_status dpd_set_adj_launch(dpd_handle h, int gh_blocks, int tap_group)
{
    if (!h) return DPD_ERR_INVALID_ARGUMENT;
    if (gh_blocks < 1 || gh_blocks > h->rows_max) return DPD_ERR_INVALID_ARGUMENT;
    if (tap_group < 1 || tap_group > 5) return DPD_ERR_INVALID_ARGUMENT;
    h->adj.gh_blocks = gh_blocks;
    h->adj.tap_group = tap_group;
    return DPD_OK;
}

dpd_status dpd_apply_stream(dpd_handle h, const void *x, void *y, int64_t n, void *stream)
{
    if (!h || n < 0) return DPD_ERR_INVALID_ARGUMENT;
    if (!h->has_coeffs) return DPD_ERR_NO_COEFFS;
    if (n == 0) return DPD_OK;
    const dpd_status st = dpd_apply(h, x, y, n, stream);   // zero history; checks the buffers
    if (st != DPD_OK) return st;
    return cuda_status(dpd::launch_stream_head(h->d_tab, h->B, h->T, static_cast<const float2 *>(x), n, h->d_hist,
                                               static_cast<float2 *>(y), static_cast<cudaStream_t>(stream)));
}

dpd_status dpd_sq_error(dpd_handle h, const void *y, const void *x, int64_t n, float gain_re, float gain_im,
                        double scale, float *loss, void *gy, void *stream)
{
    if (!h || n < 0 || !loss || !aligned(loss, 4)) return DPD_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!y || !x || !aligned(y, 8) || !aligned(x, 8))) return DPD_ERR_INVALID_ARGUMENT;
    if (n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
    const size_t bytes = (size_t)n * sizeof(float2);
    if (gy && (!aligned(gy, 8) || overlap(gy, bytes, x, bytes) || overlap(gy, bytes, y, bytes)))
        return DPD_ERR_INVALID_ARGUMENT;
    return cuda_status(dpd::launch_sq_error(static_cast<const float2 *>(y), static_cast<const float2 *>(x), n,
                                            make_float2(gain_re, gain_im), scale, h->d_loss_part, loss,
                                            static_cast<float2 *>(gy), static_cast<cudaStream_t>(stream)));
}

dpd_status dpd_reset_stream(dpd_handle h, void *stream)
{
    if (!h) return DPD_ERR_INVALID_ARGUMENT;
    return cuda_status(cudaMemsetAsync(h->d_hist, 0, sizeof(float2) * dpd::kHalo, static_cast<cudaStream_t>(stream)));
}

dpd_status dpd_set_fwd_launch(dpd_handle h, int mode, int V, int warps, int stages, int ctas_per_sm,
                              int use_tma, int group)
{
    if (!h) return DPD_ERR_INVALID_ARGUMENT;
    if (mode < 0 || mode > 3) return DPD_ERR_INVALID_ARGUMENT;
    if ((V != 2 && V != 4 && V != 6 && V != 8) || warps < 1 || warps > dpd::kFwdMaxWarps || stages < 2 || stages > 8 ||
        ctas_per_sm < 0 || (use_tma != 0 && use_tma != 1) || group < 0 || (group > 0 && warps % group != 0))
        return DPD_ERR_INVALID_ARGUMENT;
    if (use_tma) {   // the rings of all groups must fit in one CTA's shared memory
        const int gw = group > 0 ? group : warps, ng = warps / gw;
        const size_t smem = (size_t)((4 * h->B * h->T + 2) * 4 + 127) / 128 * 128 +
                            (size_t)((2 * ng * stages * 8 + 127) / 128) * 128 +
                            (size_t)ng * stages * (size_t)(dpd::kHalo + gw * 32 * V) * sizeof(float2);
        if (smem > (size_t)227 * 1024) return DPD_ERR_UNSUPPORTED;
    }
    h->fwd.group = group;
    h->fwd.mode = mode;
    h->fwd.V = V;
    h->fwd.warps = warps;
    h->fwd.stages = stages;
    h->fwd.ctas_per_sm = ctas_per_sm;
    h->fwd.use_tma = use_tma;
    h->fwd_auto = false;
    return DPD_OK;
}

dpd_status dpd_sync_status(dpd_handle h, void *stream)
{
    if (!h) return DPD_ERR_INVALID_ARGUMENT;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return DPD_ERR_CUDA;
    int flags = 0;
    if (cudaMemcpy(&flags, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DPD_ERR_CUDA;
    if (flags && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) return DPD_ERR_CUDA;
    if (flags & dpd::kFlagTimeout) return DPD_ERR_TIMEOUT;
    if (flags) return DPD_ERR_CUDA;
    return DPD_OK;
}

}  // extern "C"
