// Batched APH DPD: many independent antenna streams of uneven length and
// model order (P, Q, M) filtered by ONE persistent launch.
//
// The host plan cuts every stream into tiles of S samples and orders the
// (stream, tile) work items by cost; CTA b takes items b, b + grid, ...  One
// producer thread per CTA streams each item into a shared-memory ring slot
// with two bulk copies completed on the slot's mbarrier: the stream's
// widely-linear coefficient table (see dpd_internal.h) and the tile with its
// kHalo samples of history (zero before the stream's first sample, Eq. 2).
// The producer also writes the item's description (pointers, length, tile
// start, model, validity) into the slot's header before it arrives on the
// barrier, so the consumers read it from shared memory instead of every
// thread loading the item and stream records from global memory.  Consumer
// warps dispatch on the item's (B, T) to the same per-sample compute as the
// single-stream kernel, with coefficients read from the slot.
#pragma once

#include "dpd_fwd.cuh"

namespace dpd {

struct BatchStream {
    const float2 *x;
    float2 *y;
    int64_t n;
    int B, T;          // branch pairs, taps
    int tab_off;       // offset of the stream's table in the table pool (floats, 16-byte aligned)
    int tab_bytes;     // bytes copied per item (multiple of 16)
    const float2 *sub = nullptr;   // if set, y = sub - filter output (a least-squares residual)
};

struct BatchItem {
    int stream;
    int tile;
};

struct BatchArgs {
    const BatchStream *streams;
    const BatchItem *items;
    int nitems;
    int nstreams;
    const float *tabs;
    int64_t tab_floats;   // size of the table pool
    int *status;
    int gw = 0;           // consumer warps per group (0: one group of all warps)
    int nsub = 1;         // sub-blocks of V samples per thread and item
};

constexpr int kBatchTabBytes = ((kMaxTabFloats * 4 + 15) / 16) * 16;   // table area of a slot

// Item description written by the producer at the start of a slot.
struct BatchSlotHeader {
    const float2 *x;
    float2 *y;
    int64_t n;     // stream length
    int64_t s0;    // first sample of the tile
    int bt;        // B * 16 + T
    int ok;        // item passed item_ok (else skipped by both sides)
    const float2 *sub;   // the stream's subtrahend or null
};
constexpr int kBatchHdrBytes = 64;
static_assert(sizeof(BatchSlotHeader) <= kBatchHdrBytes, "slot header");

// Slot: header, table, tile (kHalo history samples + S samples).
__host__ __device__ constexpr size_t batch_slot_bytes(int S)
{
    return (size_t)kBatchHdrBytes + (size_t)kBatchTabBytes + (size_t)(kHalo + S) * sizeof(float2);
}

// Range checks of a work item against the plan (stream index, table inside
// the pool and the slot, tile inside the stream, 16-byte aligned input).  The
// producer and the consumers evaluate the same predicate on the same item, so
// a bad item is skipped by both sides and no wait is left unmatched.
__device__ __forceinline__ bool item_ok(const BatchArgs &a, const BatchItem &w, const BatchStream &st, int S)
{
    return w.stream >= 0 && w.stream < a.nstreams && st.tab_off >= 0 && st.tab_bytes > 0 &&
           st.tab_bytes <= kBatchTabBytes && (st.tab_bytes & 15) == 0 && (st.tab_off & 3) == 0 &&
           (int64_t)st.tab_off + st.tab_bytes / 4 <= a.tab_floats && w.tile >= 0 &&
           (int64_t)w.tile * S < st.n && ((reinterpret_cast<uintptr_t>(st.x) & 15u) == 0);
}

template <int B, int T, int V>
__device__ __forceinline__ void batched_item(const unsigned char *slot, const BatchSlotHeader &hd, int S,
                                             int t_in_tile)
{
    constexpr int W = V + T - 1;
    const float *tab = reinterpret_cast<const float *>(slot + kBatchHdrBytes);
    const float2 *xs = reinterpret_cast<const float2 *>(slot + kBatchHdrBytes + kBatchTabBytes);
    float wr[W], wi[W];
    const bool full = load_window<T, V>(xs, hd.s0, S, hd.n, hd.x, t_in_tile, wr, wi);
    float yr[V], yi[V];
    // Coefficients come from the slot (shared memory); the parameter-bank
    // table argument is not read in this mode.
    fwd_compute<B, T, V, kModePackedFma>(tab, *reinterpret_cast<const ParamTab<B, T> *>(tab), wr, wi, yr,
                                         yi);
    const int64_t g0 = hd.s0 + (int64_t)t_in_tile * V;
    if (hd.sub) {   // residual: y = sub - Psi h
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float2 t = g0 + v < hd.n ? __ldcs(hd.sub + g0 + v) : make_float2(0.f, 0.f);
            yr[v] = t.x - yr[v];
            yi[v] = t.y - yi[v];
        }
    }
    const bool vec = full && ((reinterpret_cast<uintptr_t>(hd.y) & 15u) == 0);
    store_outputs<V>(hd.y, g0, hd.n, vec, yr, yi);
}

#define DPD_BCASE(b, t)                                                                            \
    case (b) * 16 + (t):                                                                           \
        if constexpr ((b) <= BMAX && (t) <= TMAX) {                                                \
            for (int sb = 0; sb < a.nsub; ++sb)                                                    \
                batched_item<(b), (t), V>(slot, hd, SG, sb * gw * 32 + t_in_tile);                 \
            break;                                                                                 \
        }                                                                                          \
        bad = true;                                                                                \
        break;
#define DPD_BCASES(b)                                                                              \
    DPD_BCASE(b, 1) DPD_BCASE(b, 2) DPD_BCASE(b, 3) DPD_BCASE(b, 4) DPD_BCASE(b, 5)               \
    DPD_BCASE(b, 6) DPD_BCASE(b, 7) DPD_BCASE(b, 8)

template <int BMAX, int TMAX, int V>
__global__ void __launch_bounds__(32 * 17) fwd_batched_kernel(BatchArgs a, int stages)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int nwarps = blockDim.x / 32 - 1;
    const int gw = (a.gw > 0 && nwarps % a.gw == 0) ? a.gw : nwarps;   // warps per group
    const int ngroups = nwarps / gw;
    // per group g: full[s] at bars[2 stages g + s], empty[s] at bars[2 stages g + stages + s]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *ring = smem + ((2 * ngroups * stages * 8 + 127) / 128) * 128;
    const int S = a.nsub * nwarps * 32 * V;   // the item's tile
    const int SG = a.nsub * gw * 32 * V;      // a group's part of it: nsub sub-blocks of gw * 32 * V
    const size_t slot_bytes = batch_slot_bytes(SG);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int g = 0; g < ngroups; ++g)
            for (int s = 0; s < stages; ++s) {
                mbar_init(smem_addr(&bars[2 * stages * g + s]), 1);
                mbar_init(smem_addr(&bars[2 * stages * g + stages + s]), gw);
            }
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == nwarps) {
        // ---------------------------------------------------------------- producer
        // Every group's slot receives the item's header and table and the
        // group's sub-tile (with its history), so each group runs on its own
        // ring, independently of the CTA's other groups.
        if (lane != 0) return;
        const uint64_t pol = policy_evict_first();
        int it = 0, gfail = -1, fail_it = 0;
        int s = 0;          // slot of item `it`, kept incrementally
        uint32_t ph = 0;
        for (int i = blockIdx.x; i < a.nitems && gfail < 0; i += gridDim.x, ++it) {
            const BatchItem w = a.items[i];
            const BatchStream st = a.streams[(w.stream >= 0 && w.stream < a.nstreams) ? w.stream : 0];
            const bool good = item_ok(a, w, st, S);
            if (!good) atomicOr(a.status, kFlagBadWork);
            for (int g = 0; g < ngroups; ++g) {
                uint64_t *gb = bars + 2 * stages * g;
                if (it >= stages && !mbar_wait(smem_addr(&gb[stages + s]), ph ^ 1u, a.status)) {
                    gfail = g;
                    fail_it = it;
                    break;
                }
                const uint32_t fb = smem_addr(&gb[s]);
                unsigned char *slot = ring + ((size_t)g * stages + s) * slot_bytes;
                BatchSlotHeader *hd = reinterpret_cast<BatchSlotHeader *>(slot);
                const int64_t s0 = (int64_t)w.tile * S + (int64_t)g * SG;
                hd->x = st.x;
                hd->y = st.y;
                hd->n = st.n;
                hd->s0 = s0;
                hd->bt = st.B * 16 + st.T;
                hd->ok = good ? 1 : 0;
                hd->sub = st.sub;
                if (!good) {
                    mbar_arrive_expect_tx(fb, 0);   // complete the phase with no copies (releases the header)
                    continue;
                }
                int64_t lo = 0, cnt = 0;
                int off = 0;
                if (s0 < st.n) tile_copy_range(s0, SG, st.n, lo, cnt, off);
                if (cnt < 0) cnt = 0;
                const uint32_t xbytes = (uint32_t)(cnt * (int64_t)sizeof(float2));
                // The arrive releases the header stores; the consumers' wait acquires them.
                mbar_arrive_expect_tx(fb, xbytes + (uint32_t)st.tab_bytes);
                bulk_copy_g2s(smem_addr(slot + kBatchHdrBytes), a.tabs + st.tab_off, (uint32_t)st.tab_bytes, fb);
                if (xbytes)
                    bulk_copy_g2s_stream(
                        smem_addr(slot + kBatchHdrBytes + kBatchTabBytes + (size_t)off * sizeof(float2)), st.x + lo,
                        xbytes, fb, pol);
            }
            if (gfail < 0 && ++s == stages) {
                s = 0;
                ph ^= 1u;
            }
        }
        if (gfail >= 0) {
            // Let the copies already issued land before the CTA exits: group g
            // has items [0, fail_it] issued if g < gfail, else [0, fail_it - 1].
            for (int g = 0; g < ngroups; ++g) {
                const int last = g < gfail ? fail_it : fail_it - 1;
                const int first = last - stages + 1 > 0 ? last - stages + 1 : 0;
                for (int j = first; j <= last; ++j)
                    mbar_wait(smem_addr(&bars[2 * stages * g + j % stages]), (uint32_t)((j / stages) & 1), a.status);
            }
        }
        return;
    }

    // -------------------------------------------------------------------- consumers
    const int g = warp / gw;
    const int t_in_tile = (warp - g * gw) * 32 + lane;   // position in the group's sub-tile
    uint64_t *gb = bars + 2 * stages * g;
    int s = 0;
    uint32_t ph = 0;
    for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
        if (!mbar_wait(smem_addr(&gb[s]), ph, a.status)) return;
        const unsigned char *slot = ring + ((size_t)g * stages + s) * slot_bytes;
        const BatchSlotHeader &hd = *reinterpret_cast<const BatchSlotHeader *>(slot);   // read in place
        bool bad = hd.ok == 0;
        if (!bad && hd.s0 < hd.n) switch (hd.bt) {   // a group past the stream's end has nothing to do
            DPD_BCASES(1)
            DPD_BCASES(2)
            DPD_BCASES(3)
            DPD_BCASES(4)
            DPD_BCASES(5)
            DPD_BCASES(6)
        default: bad = true;
        }
        if (bad && hd.ok != 0 && lane == 0) atomicOr(a.status, kFlagBadWork);   // model outside this kernel
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&gb[stages + s]));   // slot (header, table, tile) no longer read
        if (++s == stages) {
            s = 0;
            ph ^= 1u;
        }
    }
}

#undef DPD_BCASES
#undef DPD_BCASE

// Shared-memory bytes of the batched kernel: barrier pairs of every group and
// stage, then per group `stages` slots of its sub-tile.
__host__ __device__ constexpr size_t batch_smem(int warps, int gw, int stages, int V, int nsub = 1)
{
    return (size_t)((2 * (warps / gw) * stages * 8 + 127) / 128) * 128 +
           (size_t)(warps / gw) * stages * batch_slot_bytes(nsub * gw * 32 * V);
}

// Sub-blocks per thread and item: each item costs a barrier wait, a header read
// and a dispatch, so an item carries up to 4 sub-blocks of V samples per
// thread, as many as the ring still fits in shared memory.
constexpr size_t kBatchSmemMax = 227 * 1024;
__host__ __device__ constexpr int batch_nsub(int warps, int gw, int stages, int V)
{
    return batch_smem(warps, gw, stages, V, 4) <= kBatchSmemMax   ? 4
           : batch_smem(warps, gw, stages, V, 2) <= kBatchSmemMax ? 2
                                                                   : 1;
}

// One persistent launch over the work items: orders up to 9 (B <= 5) and up
// to 7 taps (batched_57.cu), or up to 11 and 8 (batched_68.cu).
cudaError_t launch_batched_57(const BatchArgs &a, int V, int warps, int stages, int cps, int sm_count,
                              cudaStream_t s);
cudaError_t launch_batched_68(const BatchArgs &a, int V, int warps, int stages, int cps, int sm_count,
                              cudaStream_t s);

template <int BMAX, int TMAX, int V>
cudaError_t launch_batched_impl(const BatchArgs &a, int warps, int stages, int ctas_per_sm, int sm_count,
                                cudaStream_t s)
{
    const int threads = (warps + 1) * 32;
    const int gw = (a.gw > 0 && warps % a.gw == 0) ? a.gw : warps;
    if (a.nsub < 1 || a.nsub > 4) return cudaErrorInvalidValue;
    const size_t smem = batch_smem(warps, gw, stages, V, a.nsub);
    auto kern = fwd_batched_kernel<BMAX, TMAX, V>;
    static SmemAttr smem_rec;
    cudaError_t e = ensure_smem(smem_rec, (const void *)kern, smem);
    if (e != cudaSuccess) return e;
    static OccCache occ_rec;
    int occ = 0;
    e = occupancy(occ_rec, (const void *)kern, threads, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int cps = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    int grid = sm_count * cps;
    if (grid > a.nitems) grid = a.nitems;
    if (grid < 1) return cudaSuccess;
    kern<<<grid, threads, smem, s>>>(a, stages);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
