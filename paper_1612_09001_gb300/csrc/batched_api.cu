// libdpd C ABI, batched part: plans of many independent streams executed by
// one persistent launch (see dpd_batched.cuh and include/dpd.h).
#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dpd.h"
#include "dpd_model.h"
#include "dpd_batched.cuh"

struct dpd_plan_s {
    int device = 0, sm_count = 0;
    std::vector<dpd::BatchStream> streams;   // host copy (device pointers, sizes, table offsets)
    dpd::BatchStream *d_streams = nullptr;
    dpd::BatchItem *d_items = nullptr;
    float *d_tabs = nullptr;
    float *d_h = nullptr;          // raw coefficients, 2*K floats per stream
    int *d_status = nullptr;
    int nitems = 0;
    int64_t tab_floats = 0;
    int small = 1;            // every stream has B <= 5 and T <= 7
    int V = 8, warps = 8, stages = 4, ctas_per_sm = 0, group = 0;
    int nsub = dpd::batch_nsub(8, 8, 4, 8);   // sub-blocks per thread and item (follows the launch shape)
};

namespace {

int nbranch(int order) { return order > 0 ? (order + 1) / 2 : 0; }
bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return na && nb && x < y + nb && y < x + na;
}

void free_plan(dpd_plan p)
{
    cudaFree(p->d_streams);
    cudaFree(p->d_items);
    cudaFree(p->d_tabs);
    cudaFree(p->d_h);
    cudaFree(p->d_status);
    delete p;
}

// Work list for tile size S = nsub * warps * 32 * V: streams by decreasing per-sample
// cost (B * T), every tile of a stream in order.  Launched CTAs take items
// round-robin.  The list goes to a new device buffer that replaces the plan's
// only once it holds the list, so on failure the plan keeps its previous list
// (and tiling) unchanged.
dpd_status build_items(dpd_plan p, int V, int warps, int nsub)
{
    const int S = nsub * warps * 32 * V;
    std::vector<int> order(p->streams.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    // Costliest models first (B T per sample), and streams of the same model
    // next to each other, so that the items a CTA takes one after another
    // mostly run the same (B, T) code path.
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int ca = p->streams[a].B * p->streams[a].T, cb = p->streams[b].B * p->streams[b].T;
        if (ca != cb) return ca > cb;
        return p->streams[a].B > p->streams[b].B;
    });
    std::vector<dpd::BatchItem> items;
    for (int si : order) {
        const int64_t nt = (p->streams[si].n + S - 1) / S;
        if (nt > INT32_MAX) return DPD_ERR_UNSUPPORTED;
        for (int64_t t = 0; t < nt; ++t) items.push_back({si, (int)t});
    }
    if (items.size() > (size_t)INT32_MAX) return DPD_ERR_UNSUPPORTED;
    dpd::BatchItem *d_new = nullptr;
    const size_t cap = std::max<size_t>(items.size(), 1);
    if (cudaMalloc(&d_new, cap * sizeof(dpd::BatchItem)) != cudaSuccess) return DPD_ERR_ALLOC;
    if (!items.empty() &&
        cudaMemcpy(d_new, items.data(), items.size() * sizeof(dpd::BatchItem), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(d_new);
        return DPD_ERR_CUDA;
    }
    cudaFree(p->d_items);
    p->d_items = d_new;
    p->nitems = (int)items.size();
    return DPD_OK;
}

}  // namespace

extern "C" {

dpd_status dpd_plan_batched(const dpd_stream_desc *descs, int count, int where, dpd_plan *out)
{
    if (!out || count < 0 || (count > 0 && !descs)) return DPD_ERR_INVALID_ARGUMENT;
    if (where != DPD_HOST && where != DPD_DEVICE) return DPD_ERR_INVALID_ARGUMENT;
    // validate every stream before touching the device
    size_t hfloats = 0, tfloats = 0;
    for (int i = 0; i < count; ++i) {
        const dpd_stream_desc &d = descs[i];
        const dpd_status mst = dpd::model_status(d.P, d.Q, d.M);
        if (mst != DPD_OK) return mst;
        if (d.n < 0 || !d.h) return DPD_ERR_INVALID_ARGUMENT;
        if (d.n > (int64_t)(INT64_MAX / sizeof(float2))) return DPD_ERR_INVALID_ARGUMENT;
        if (d.n > 0 && (!d.x || !d.y || !aligned(d.x, 16) || !aligned(d.y, 8))) return DPD_ERR_INVALID_ARGUMENT;
        if (!aligned(d.h, where == DPD_HOST ? 4 : 8)) return DPD_ERR_INVALID_ARGUMENT;
        const int Bp = nbranch(d.P), Bq = nbranch(d.Q), B = std::max(Bp, Bq), T = d.M + 1;
        hfloats += 2 * (size_t)((Bp + Bq) * T + 1);
        tfloats += (size_t)((dpd::wl_table_floats(B, T) * 4 + 15) / 16) * 4;
    }
    for (int i = 0; i < count; ++i) {   // outputs overlap no input and no other output
        const size_t bi = (size_t)descs[i].n * sizeof(float2);
        for (int j = 0; j < count; ++j) {
            const size_t bj = (size_t)descs[j].n * sizeof(float2);
            if (overlap(descs[i].y, bi, descs[j].x, bj)) return DPD_ERR_INVALID_ARGUMENT;
            if (j != i && overlap(descs[i].y, bi, descs[j].y, bj)) return DPD_ERR_INVALID_ARGUMENT;
        }
    }
    dpd_plan p = new (std::nothrow) dpd_plan_s();
    if (!p) return DPD_ERR_ALLOC;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        delete p;
        return DPD_ERR_CUDA;
    }
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->d_h, std::max<size_t>(hfloats, 2) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_tabs, std::max<size_t>(tfloats, 4) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_streams, std::max(count, 1) * sizeof(dpd::BatchStream)) != cudaSuccess) {
        free_plan(p);
        return DPD_ERR_ALLOC;
    }
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) {
        free_plan(p);
        return DPD_ERR_CUDA;
    }
    size_t hoff = 0, toff = 0;
    for (int i = 0; i < count; ++i) {
        const dpd_stream_desc &d = descs[i];
        const int Bp = nbranch(d.P), Bq = nbranch(d.Q), B = std::max(Bp, Bq), T = d.M + 1;
        const int K = (Bp + Bq) * T + 1;
        float2 *hdst = reinterpret_cast<float2 *>(p->d_h + hoff);
        const cudaMemcpyKind kind = where == DPD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (cudaMemcpy(hdst, d.h, sizeof(float2) * K, kind) != cudaSuccess ||
            dpd::launch_wl_table(hdst, Bp, Bq, T, p->d_tabs + toff, nullptr, 0) != cudaSuccess) {
            free_plan(p);
            return DPD_ERR_CUDA;
        }
        dpd::BatchStream st;
        st.x = static_cast<const float2 *>(d.x);
        st.y = static_cast<float2 *>(d.y);
        st.n = d.n;
        st.B = B;
        st.T = T;
        st.tab_off = (int)toff;
        st.tab_bytes = ((dpd::wl_table_floats(B, T) * 4 + 15) / 16) * 16;
        p->streams.push_back(st);
        if (B > 5 || T > 7) p->small = 0;
        hoff += 2 * (size_t)K;
        toff += (size_t)st.tab_bytes / 4;
    }
    p->tab_floats = (int64_t)toff;
    if (count > 0 &&
        cudaMemcpy(p->d_streams, p->streams.data(), count * sizeof(dpd::BatchStream), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        free_plan(p);
        return DPD_ERR_CUDA;
    }
    dpd_status st = build_items(p, p->V, p->warps, p->nsub);
    if (st == DPD_OK && cudaDeviceSynchronize() != cudaSuccess) st = DPD_ERR_CUDA;
    if (st != DPD_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return DPD_OK;
}

dpd_status dpd_plan_set_launch(dpd_plan p, int V, int warps, int stages, int ctas_per_sm, int group)
{
    if (!p) return DPD_ERR_INVALID_ARGUMENT;
    if ((V != 4 && V != 6 && V != 8) || warps < 1 || warps > 16 || stages < 2 || stages > 8 || ctas_per_sm < 0 || group < 0 ||
        (group > 0 && warps % group != 0))
        return DPD_ERR_INVALID_ARGUMENT;
    const int gw = group > 0 ? group : warps;
    if (dpd::batch_smem(warps, gw, stages, V) > dpd::kBatchSmemMax) return DPD_ERR_UNSUPPORTED;
    const int nsub = dpd::batch_nsub(warps, gw, stages, V);
    if (V != p->V || warps != p->warps || nsub != p->nsub) {
        // Re-tile first: the new shape is kept only once its work list is on
        // the device; on failure the plan runs with its previous shape.
        const dpd_status st = build_items(p, V, warps, nsub);
        if (st != DPD_OK) return st;
    }
    p->V = V;
    p->warps = warps;
    p->nsub = nsub;
    p->stages = stages;
    p->ctas_per_sm = ctas_per_sm;
    p->group = group;
    return DPD_OK;
}

dpd_status dpd_exec_batched(dpd_plan p, void *stream)
{
    if (!p) return DPD_ERR_INVALID_ARGUMENT;
    if (p->nitems == 0) return DPD_OK;
    if (!p->d_items || !p->d_streams || !p->d_tabs || !p->d_status) return DPD_ERR_INVALID_ARGUMENT;
    dpd::BatchArgs a;
    a.streams = p->d_streams;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.nstreams = (int)p->streams.size();
    a.tabs = p->d_tabs;
    a.tab_floats = p->tab_floats;
    a.status = p->d_status;
    a.gw = p->group;
    a.nsub = p->nsub;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = p->small ? dpd::launch_batched_57(a, p->V, p->warps, p->stages, p->ctas_per_sm, p->sm_count, s)
                             : dpd::launch_batched_68(a, p->V, p->warps, p->stages, p->ctas_per_sm, p->sm_count, s);
    return e == cudaSuccess ? DPD_OK : DPD_ERR_CUDA;
}

dpd_status dpd_plan_sync_status(dpd_plan p, void *stream)
{
    if (!p) return DPD_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return DPD_ERR_CUDA;
    int flags = 0;
    if (cudaMemcpy(&flags, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DPD_ERR_CUDA;
    if (flags && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return DPD_ERR_CUDA;
    if (flags & dpd::kFlagTimeout) return DPD_ERR_TIMEOUT;
    if (flags) return DPD_ERR_CUDA;
    return DPD_OK;
}

dpd_status dpd_plan_destroy(dpd_plan p)
{
    if (p) free_plan(p);
    return DPD_OK;
}

}  // extern "C"
