// Forward APH DPD filter kernels (Eq. 1 / Algorithm 1), templated on the
// branch count B = max((P+1)/2, (Q+1)/2), the tap count T = M + 1 and the
// number V of consecutive samples each thread produces.
//
// Arithmetic.  Per tap k the main and conjugate branches of Algorithm 1 are
// regrouped into a widely-linear form: with r = |x|^2,
//   sum_p h_{p,k} |x|^{p-1} x + sum_q hbar_{q,k} |x|^{q-1} conj(x)
//     = A_k(r) x + C_k(r) conj(x)
//     = (P0(r) a + P1(r) b) + j (P2(r) a + P3(r) b),   x = a + j b,
// four real polynomials of degree B-1 evaluated by Horner's rule: 4B fused
// multiply-adds per (sample, tap) instead of 8B for the complex products.  The
// polynomial basis is formed from r without a square root, lowest order first
// (Sec. 3.2.1).
//
// Data movement.  The TMA kernel is persistent: each CTA walks tiles of
// S = warps*32*V samples.  One producer thread streams every tile, together
// with the kHalo samples in front of it (the filter history, Eq. 2's shifted
// rows), into a ring of shared-memory slots with one-dimensional bulk copies
// completed on mbarriers; consumer warps read their window from shared memory,
// release the slot and write the outputs with 16-byte streaming stores.  No
// lane is redundant: the history comes from the staged halo instead of the
// overlapping warps of the paper's Sec. 3.3.2 design.
#pragma once

#include "dpd_device.cuh"
#include "dpd_internal.h"

namespace dpd {

// Coefficient table passed by value (kernel parameter bank).  16-byte aligned
// so that every {P0, P2} / {P1, P3} pair sits at an 8-byte aligned offset of
// the bank, where a packed FMA can take it as a 64-bit constant operand (a
// misaligned table costs a register move per pair).  The alignment is stated
// rather than left to the parameters before it: with 8, FwdArgs growing by 8
// bytes moved the table and took the P = Q = 9, M = 4 kernel from 75 to 82
// registers.
template <int B, int T>
struct alignas(16) ParamTab {
    float v[wl_table_floats(B, T)];
};

// V outputs from a window of V + T - 1 inputs (window index j is sample n0 - (T-1) + j).
// MODE bit kModeParamCoef: coefficients come from the parameter bank and are
// used directly as FMA operands; otherwise one tap's B float4s are loaded from
// shared memory.  MODE bit kModePackedFma: the polynomial pairs {P0,P2} and
// {P1,P3} are evaluated with packed f32x2 FMAs.
template <int B, int T, int V, int MODE>
__device__ __forceinline__ void fwd_compute(const float *__restrict__ stab, const ParamTab<B, T> &ptab,
                                            const float (&wr)[V + T - 1],
                                            const float (&wi)[V + T - 1], float (&yr)[V],
                                            float (&yi)[V])
{
    constexpr int W = V + T - 1;
    constexpr bool PARAM = (MODE & kModeParamCoef) != 0;
    constexpr bool PACKED = (MODE & kModePackedFma) != 0;
    float r[W];
#pragma unroll
    for (int j = 0; j < W; ++j) r[j] = fmaf(wr[j], wr[j], wi[j] * wi[j]);
    const float cr = PARAM ? ptab.v[4 * B * T] : stab[4 * B * T];
    const float ci = PARAM ? ptab.v[4 * B * T + 1] : stab[4 * B * T + 1];
    float2 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float2(cr, ci);
#pragma unroll
    for (int k = 0; k < T; ++k) {
        float4 cf[B];   // per order m: {P0, P2, P1, P3}
#pragma unroll
        for (int m = 0; m < B; ++m) {
            if constexpr (PARAM)
                cf[m] = make_float4(ptab.v[(k * B + m) * 4 + 0], ptab.v[(k * B + m) * 4 + 1],
                                    ptab.v[(k * B + m) * 4 + 2], ptab.v[(k * B + m) * 4 + 3]);
            else
                cf[m] = reinterpret_cast<const float4 *>(stab)[k * B + m];
        }
        if constexpr (PACKED) {
            // All V samples advance one Horner step together: 2V independent
            // chains of packed {P0,P2} and {P1,P3} evaluations.
            float2 pa[V], pb[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                pa[v] = make_float2(cf[B - 1].x, cf[B - 1].y);
                pb[v] = make_float2(cf[B - 1].z, cf[B - 1].w);
            }
#pragma unroll
            for (int m = B - 2; m >= 0; --m) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = v + (T - 1) - k;   // window index of sample n - k
                    const float2 rr = make_float2(r[j], r[j]);
                    pa[v] = __ffma2_rn(pa[v], rr, make_float2(cf[m].x, cf[m].y));
                    pb[v] = __ffma2_rn(pb[v], rr, make_float2(cf[m].z, cf[m].w));
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int j = v + (T - 1) - k;
                acc[v] = __ffma2_rn(pa[v], make_float2(wr[j], wr[j]), acc[v]);   // {P0 a, P2 a}
                acc[v] = __ffma2_rn(pb[v], make_float2(wi[j], wi[j]), acc[v]);   // {P1 b, P3 b}
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int j = v + (T - 1) - k;   // window index of sample n - k
                float p0 = cf[B - 1].x, p2 = cf[B - 1].y, p1 = cf[B - 1].z, p3 = cf[B - 1].w;
#pragma unroll
                for (int m = B - 2; m >= 0; --m) {
                    p0 = fmaf(p0, r[j], cf[m].x);
                    p2 = fmaf(p2, r[j], cf[m].y);
                    p1 = fmaf(p1, r[j], cf[m].z);
                    p3 = fmaf(p3, r[j], cf[m].w);
                }
                acc[v].x = fmaf(p0, wr[j], acc[v].x);
                acc[v].x = fmaf(p1, wi[j], acc[v].x);
                acc[v].y = fmaf(p2, wr[j], acc[v].y);
                acc[v].y = fmaf(p3, wi[j], acc[v].y);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        yr[v] = acc[v].x;
        yi[v] = acc[v].y;
    }
}

template <int B, int T>
__host__ __device__ constexpr int tab_bytes()
{
    return ((wl_table_floats(B, T) * 4 + 127) / 128) * 128;
}

// Read the window of thread t_in_tile of a tile that starts at sample s0 from a
// shared-memory slot holding global samples [s0 - kHalo, ...).  Samples in
// [lo, vhi) are in the slot; the sample just past vhi (odd tail) comes from
// global memory; samples outside [0, n) are zero.  Returns true when the whole
// tile and its history are in the slot (the vectorised fast path).
template <int T, int V>
__device__ __forceinline__ bool load_window(const float2 *slot, int64_t s0, int S, int64_t n,
                                            const float2 *__restrict__ x, int t_in_tile,
                                            float (&wr)[V + T - 1], float (&wi)[V + T - 1])
{
    constexpr int W = V + T - 1;
    const int64_t g0 = s0 + (int64_t)t_in_tile * V;
    const int64_t lo = (s0 - kHalo > 0) ? s0 - kHalo : 0;
    const int64_t hi = (s0 + S < n) ? s0 + S : n;
    const int64_t vhi = lo + ((hi - lo) & ~int64_t(1));
    const bool full = (s0 >= kHalo) && (s0 + S <= vhi);
    if (full) {
        constexpr int MP = ((T - 1) + 1) & ~1;   // history rounded up to a 16-byte unit
        constexpr int E = V + MP;
        constexpr int D = MP - (T - 1);
        const float4 *src = reinterpret_cast<const float4 *>(slot + t_in_tile * V + kHalo - MP);
        float er[E], ei[E];
#pragma unroll
        for (int i = 0; i < E / 2; ++i) {
            const float4 q = src[i];
            er[2 * i] = q.x;
            ei[2 * i] = q.y;
            er[2 * i + 1] = q.z;
            ei[2 * i + 1] = q.w;
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            wr[j] = er[j + D];
            wi[j] = ei[j + D];
        }
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int64_t g = g0 - (T - 1) + j;
            float2 v = make_float2(0.f, 0.f);
            if (g >= lo && g < vhi)
                v = slot[g - (s0 - kHalo)];
            else if (g >= 0 && g < n)
                v = x[g];
            wr[j] = v.x;
            wi[j] = v.y;
        }
    }
    return full;
}

// Bulk-copy geometry of a tile: global sample range [lo, lo + cnt) (cnt even)
// lands at slot element `off`.
__device__ __forceinline__ void tile_copy_range(int64_t s0, int S, int64_t n, int64_t &lo, int64_t &cnt,
                                                int &off)
{
    lo = s0 - kHalo;
    off = 0;
    if (lo < 0) {
        off = (int)(-lo);
        lo = 0;
    }
    const int64_t hi = (s0 + S < n) ? s0 + S : n;
    cnt = (hi - lo) & ~int64_t(1);
}

template <int V>
__device__ __forceinline__ void store_outputs(float2 *__restrict__ y, int64_t g0, int64_t n, bool full_vec,
                                              const float (&yr)[V], const float (&yi)[V])
{
    if (full_vec) {
        float4 *yp = reinterpret_cast<float4 *>(y + g0);
#pragma unroll
        for (int i = 0; i < V / 2; ++i)
            st_stream_f4(yp + i, make_float4(yr[2 * i], yi[2 * i], yr[2 * i + 1], yi[2 * i + 1]));
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (g0 + v < n) y[g0 + v] = make_float2(yr[v], yi[v]);
    }
}

// Shared-memory bytes of the TMA kernel for a launch shape: the table area, the
// barrier pairs of every group and stage, and per group `stages` slots of the
// group's sub-tile (gw * 32 * V samples) with kHalo history samples each;
// kModeNorms adds as many slots for the minuend's sub-tiles (no history).
template <int B, int T, int V>
__host__ __device__ constexpr size_t fwd_tma_smem(int warps, int gw, int stages, bool sub = false)
{
    return (size_t)tab_bytes<B, T>() + (size_t)((2 * (warps / gw) * stages * 8 + 127) / 128) * 128 +
           (size_t)(warps / gw) * stages * (size_t)(kHalo + gw * 32 * V) * sizeof(float2) +
           (sub ? (size_t)(warps / gw) * stages * (size_t)(gw * 32 * V) * sizeof(float2) : 0);
}

// The consumer warps form groups of gw warps; every group has its own ring of
// `stages` slots and its own full / empty barriers, and the producer thread
// fills each group's slot with its own bulk copy (the group's sub-tile and the
// kHalo samples in front of it).  A group starts on its sub-tile as soon as its
// own copy has landed and releases its slot on its own, so the groups of a CTA
// drift apart instead of waiting for one another at every tile: at start-up
// the first (small) sub-tiles arrive sooner, and in the steady state the FMA
// and memory phases of the groups overlap.
//
// Shapes.  SH = 0 takes the warp count from the launch and the group size and
// ring depth from its arguments; SH > 0 fixes all three at compile time (the
// kFwdShapes entry), which turns the tile, sub-tile and slot arithmetic into
// constants and lets a 12-warp shape ask for two CTAs per SM: the shapes the
// autotuner picks for the benchmarked models run that way (measured: 59.0 ->
// 55.5 us per 2^24 samples at P = Q = 9, M = 4, 16 warps in groups of 4).
struct FwdShape {
    int warps, gw, stages;
};
constexpr FwdShape kFwdShapes[] = {{0, 0, 0}, {16, 4, 4}, {12, 3, 3}, {12, 2, 4}, {16, 8, 4}};
constexpr int kFwdNumShapes = sizeof(kFwdShapes) / sizeof(kFwdShapes[0]);

template <int SH>
constexpr int fwd_lb_threads()
{
    return SH > 0 ? 32 * (kFwdShapes[SH].warps + 1) : 32 * (kFwdMaxWarps + 1);
}
template <int SH>
constexpr int fwd_lb_blocks()
{
    return (SH > 0 && kFwdShapes[SH].warps <= 12) ? 2 : 1;
}

template <int B, int T, int V, int MODE, int SH>
__global__ void __launch_bounds__(fwd_lb_threads<SH>(), fwd_lb_blocks<SH>())
    fwd_tma_kernel(FwdArgs a, int stages_arg, int gw_arg, int64_t ntiles, const __grid_constant__ ParamTab<B, T> ptab)
{
    constexpr bool FIXED = SH > 0;
    constexpr int W = V + T - 1;
    constexpr int TABF = wl_table_floats(B, T);
    extern __shared__ __align__(128) unsigned char smem[];
    float *tab = reinterpret_cast<float *>(smem);
    const int nwarps = FIXED ? kFwdShapes[SH].warps : (int)(blockDim.x / 32) - 1;   // the last warp produces
    const int gw = FIXED ? kFwdShapes[SH].gw : gw_arg;
    const int stages = FIXED ? kFwdShapes[SH].stages : stages_arg;
    const int ngroups = nwarps / gw;
    // per group g: full[s] at bars[2 stages g + s], empty[s] at bars[2 stages g + stages + s]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + tab_bytes<B, T>());
    float2 *ring = reinterpret_cast<float2 *>(smem + tab_bytes<B, T>() + ((2 * ngroups * stages * 8 + 127) / 128) * 128);
    const int S = nwarps * 32 * V;    // tile
    const int SG = gw * 32 * V;       // a group's sub-tile
    const int slot_elems = kHalo + SG;
    // kModeNorms stages the minuend's sub-tiles through shared memory too (per
    // group `stages` slots): there its global loads, issued after the filter
    // arithmetic, would wait in full (measured 39.3 -> 36.4 us per 2^22
    // samples at P = Q = 11, M = 7).  The plain subtract mode keeps them in
    // global memory: staging held its slots longer and gained nothing there.
    constexpr bool STAGE = (MODE & kModeNorms) != 0;
    const float2 *sring = ring + (size_t)ngroups * stages * slot_elems;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Prologue that touches no global memory (overlaps the previous grid's tail
    // under programmatic dependent launch), then wait for that grid.
    if (tid == 0) {
        for (int g = 0; g < ngroups; ++g)
            for (int s = 0; s < stages; ++s) {
                mbar_init(smem_addr(&bars[2 * stages * g + s]), 1);
                mbar_init(smem_addr(&bars[2 * stages * g + stages + s]), gw);
            }
        fence_barrier_init();
    }
    grid_dep_launch_dependents();
    grid_dep_wait();
    if constexpr ((MODE & kModeParamCoef) == 0)
        for (int i = tid; i < TABF; i += blockDim.x) tab[i] = a.tab[i];
    __syncthreads();

    if (warp == nwarps) {
        // ---------------------------------------------------------------- producer
        if (lane != 0) return;
        const uint64_t pol = policy_evict_first();
        int64_t it = 0;
        int gfail = -1;   // group whose slot wait ran out, at tile index fail_it
        int64_t fail_it = 0;
        int s = 0;        // slot of tile `it` (it % stages, kept incrementally: no division in the loop)
        uint32_t ph = 0;  // parity of its use of the slot ((it / stages) & 1)
        for (int64_t tile = blockIdx.x; tile < ntiles && gfail < 0; tile += gridDim.x, ++it) {
            for (int g = 0; g < ngroups; ++g) {
                uint64_t *gb = bars + 2 * stages * g;
                if (it >= stages && !mbar_wait(smem_addr(&gb[stages + s]), ph ^ 1u, a.status)) {
                    gfail = g;
                    fail_it = it;
                    break;
                }
                int64_t lo, cnt;
                int off;
                const int64_t s0 = tile * S + (int64_t)g * SG;
                tile_copy_range(s0, SG, a.n, lo, cnt, off);
                if (cnt < 0) cnt = 0;   // a group past the end of the input: nothing to copy
                const uint32_t bytes = (uint32_t)(cnt * (int64_t)sizeof(float2));
                // STAGE: the minuend's sub-tile when all of it is in the input
                // (the consumers read a partial one from global memory).  s0 is
                // even and SG * 8 a multiple of 16: a 16-byte aligned copy.
                const uint32_t sbytes = (STAGE && s0 + SG <= a.n) ? (uint32_t)SG * (uint32_t)sizeof(float2) : 0u;
                const uint32_t fb = smem_addr(&gb[s]);
                mbar_arrive_expect_tx(fb, bytes + sbytes);
                if (bytes)
                    bulk_copy_g2s_stream(smem_addr(ring + ((size_t)g * stages + s) * slot_elems + off), a.x + lo,
                                         bytes, fb, pol);
                if (sbytes)
                    bulk_copy_g2s_stream(smem_addr(sring + ((size_t)g * stages + s) * SG), a.sub + s0, sbytes, fb,
                                         pol);
            }
            if (gfail < 0 && ++s == stages) {
                s = 0;
                ph ^= 1u;
            }
        }
        if (gfail >= 0) {
            // Let the copies already issued land before the CTA exits: group g
            // has tiles [0, fail_it] issued if g < gfail, else [0, fail_it - 1].
            for (int g = 0; g < ngroups; ++g) {
                const int64_t last = g < gfail ? fail_it : fail_it - 1;
                const int64_t first = last - stages + 1 > 0 ? last - stages + 1 : 0;
                for (int64_t j = first; j <= last; ++j)
                    mbar_wait(smem_addr(&bars[2 * stages * g + j % stages]), (uint32_t)((j / stages) & 1), a.status);
            }
        }
        return;
    }

    // -------------------------------------------------------------------- consumers
    const int g = warp / gw;
    const int t_in_tile = (warp - g * gw) * 32 + lane;   // position in the group's sub-tile
    uint64_t *gb = bars + 2 * stages * g;
    const float2 *ring_g = ring + (size_t)g * stages * slot_elems;
    constexpr bool NORMS = (MODE & kModeNorms) != 0;
    int s = 0;        // slot and parity of the current tile, kept incrementally
    uint32_t ph = 0;
    int64_t it = 0;
    // NORMS: this thread's sums |sub - y|^2 and |sub|^2 over its tiles as FP32
    // (hi, lo) pairs; no FP64 arithmetic runs in the kernel (FP64 on this GPU
    // is a small fraction of the FP32 rate).
    float2 pe = make_float2(0.f, 0.f), pt = make_float2(0.f, 0.f);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        if constexpr (FIXED) {   // constant ring depth: a cheap modulo
            s = (int)(it % kFwdShapes[SH].stages);
            ph = (uint32_t)((it / kFwdShapes[SH].stages) & 1);
        }
        if (!mbar_wait(smem_addr(&gb[s]), ph, a.status)) {
            if constexpr (NORMS) break;   // still take part in the completion count
            else return;
        }
        const float2 *slot = ring_g + (size_t)s * slot_elems;
        const int s_cur = s;
        const int64_t s0 = tile * S + (int64_t)g * SG;
        float wr[W], wi[W];
        const bool full = load_window<T, V>(slot, s0, SG, a.n, a.x, t_in_tile, wr, wi);
        if constexpr (!STAGE) {   // the slot is free once the window is in registers
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&gb[stages + s]));
        }
        if (!FIXED && ++s == stages) {
            s = 0;
            ph ^= 1u;
        }

        float yr[V], yi[V];
        fwd_compute<B, T, V, MODE & (kModeParamCoef | kModePackedFma)>(tab, ptab, wr, wi, yr, yi);
        const int64_t g0 = s0 + (int64_t)t_in_tile * V;
        if constexpr ((MODE & kModeSubtract) != 0) {   // y <- sub - y
            float ea = 0.f, ta = 0.f;   // NORMS: the tile's |sub - y|^2 and |sub|^2 in FP32
            if (full) {   // STAGE: the minuend's sub-tile is in the slot (full implies s0 + SG <= n)
                const float4 *sp =
                    STAGE ? reinterpret_cast<const float4 *>(sring + ((size_t)g * stages + s_cur) * SG + t_in_tile * V)
                          : reinterpret_cast<const float4 *>(a.sub + g0);
#pragma unroll
                for (int i = 0; i < V / 2; ++i) {
                    float4 q;
                    if constexpr (STAGE)
                        q = sp[i];
                    else
                        q = __ldcs(sp + i);
                    yr[2 * i] = q.x - yr[2 * i];
                    yi[2 * i] = q.y - yi[2 * i];
                    yr[2 * i + 1] = q.z - yr[2 * i + 1];
                    yi[2 * i + 1] = q.w - yi[2 * i + 1];
                    if constexpr (NORMS) {
                        ea = fmaf(yr[2 * i], yr[2 * i], fmaf(yi[2 * i], yi[2 * i], ea));
                        ea = fmaf(yr[2 * i + 1], yr[2 * i + 1], fmaf(yi[2 * i + 1], yi[2 * i + 1], ea));
                        ta = fmaf(q.x, q.x, fmaf(q.y, q.y, ta));
                        ta = fmaf(q.z, q.z, fmaf(q.w, q.w, ta));
                    }
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (g0 + v < a.n) {
                        const float2 q = a.sub[g0 + v];
                        yr[v] = q.x - yr[v];
                        yi[v] = q.y - yi[v];
                        if constexpr (NORMS) {
                            ea = fmaf(yr[v], yr[v], fmaf(yi[v], yi[v], ea));
                            ta = fmaf(q.x, q.x, fmaf(q.y, q.y, ta));
                        }
                    }
            }
            if constexpr (NORMS) {
                two_sum_acc(pe.x, pe.y, ea);
                two_sum_acc(pt.x, pt.y, ta);
            }
            if constexpr (STAGE) {   // both parts of the slot have been read
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&gb[stages + s_cur]));
            }
        }
        if constexpr (!NORMS) store_outputs<V>(a.y, g0, a.n, full && a.vec_store, yr, yi);
    }
    if constexpr (NORMS) {
        // The consumer warps' pairs meet in shared memory (named barrier 1: the
        // producer warp has left), warp 0 writes the CTA's pairs as one float4,
        // and the last CTA of the grid to finish adds those in CTA order
        // (deterministic), writes the two sums in FP64 and clears the counter
        // for the next launch.
        __shared__ float4 red[kFwdMaxWarps];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pe = pair_add(pe, shfl_xor_pair(pe, o));
            pt = pair_add(pt, shfl_xor_pair(pt, o));
        }
        if (lane == 0) red[warp] = make_float4(pe.x, pe.y, pt.x, pt.y);
        asm volatile("bar.sync 1, %0;" ::"r"(nwarps * 32) : "memory");
        if (warp != 0) return;
        const float4 r = lane < nwarps ? red[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        pe = make_float2(r.x, r.y);
        pt = make_float2(r.z, r.w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pe = pair_add(pe, shfl_xor_pair(pe, o));
            pt = pair_add(pt, shfl_xor_pair(pt, o));
        }
        float4 *part = reinterpret_cast<float4 *>(a.norms);
        unsigned *count = reinterpret_cast<unsigned *>(a.norms + 2 * kFwdNormSlots + 2);
        int last = 0;
        if (lane == 0) {
            part[blockIdx.x] = make_float4(pe.x, pe.y, pt.x, pt.y);
            __threadfence();
            last = atomicAdd(count, 1u) == gridDim.x - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __threadfence();
        pe = make_float2(0.f, 0.f);
        pt = make_float2(0.f, 0.f);
        for (int i = lane; i < (int)gridDim.x; i += 32) {
            const float4 v = __ldcg(part + i);
            pe = pair_add(pe, make_float2(v.x, v.y));
            pt = pair_add(pt, make_float2(v.z, v.w));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pe = pair_add(pe, shfl_xor_pair(pe, o));
            pt = pair_add(pt, shfl_xor_pair(pt, o));
        }
        if (lane == 0) {
            a.norms[2 * kFwdNormSlots] = (double)pe.x + (double)pe.y;
            a.norms[2 * kFwdNormSlots + 1] = (double)pt.x + (double)pt.y;
            *count = 0u;
        }
    }
}

// Plain-load variant: every thread reads its window straight from global
// memory (through L1).  Used for buffers that are only 8-byte aligned and as
// the no-TMA baseline.
template <int B, int T, int V, int MODE>
__global__ void __launch_bounds__(256)
    fwd_ldg_kernel(FwdArgs a, const __grid_constant__ ParamTab<B, T> ptab)
{
    constexpr int W = V + T - 1;
    constexpr int TABF = wl_table_floats(B, T);
    __shared__ __align__(16) float tab[((TABF + 3) / 4) * 4];
    for (int i = threadIdx.x; i < TABF; i += blockDim.x) tab[i] = a.tab[i];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    for (int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; g0 < a.n; g0 += stride) {
        float wr[W], wi[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int64_t g = g0 - (T - 1) + j;
            float2 v = make_float2(0.f, 0.f);
            if (g >= 0 && g < a.n) v = __ldg(a.x + g);
            wr[j] = v.x;
            wi[j] = v.y;
        }
        float yr[V], yi[V];
        fwd_compute<B, T, V, MODE>(tab, ptab, wr, wi, yr, yi);
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (g0 + v < a.n) a.y[g0 + v] = make_float2(yr[v], yi[v]);
    }
}

// Instantiated launch shapes.  Every (B, T) gets the default packed modes
// (2: shared-memory coefficients, 3: parameter-bank coefficients) at V = 4, 6
// and 8 plus the scalar mode 0 at V = 4; the plain-load kernel gets V = 4 in
// modes 0, 2 and 3.  The (B, T) pairs of the benchmarked workloads
// get every combination, for tuning and ablation.
template <int B, int T>
constexpr bool fwd_all_modes()
{
    return (B == 5 && T == 5) || (B == 3 && T == 3) || (B == 4 && T == 4) || (B == 6 && T == 8);
}

// Fixed-shape kernels (kFwdShapes) exist for the benchmarked filter models
// (B = T = 3, 4, 5) at V = 8 with packed FMAs on parameter-bank coefficients
// (mode 3); larger models would spill in the two-CTA shapes.
template <int B, int T, int V, int MODE>
constexpr bool fwd_fixed_shapes()
{
    return fwd_all_modes<B, T>() && B * T <= 25 && V == 8 && MODE == (kModeParamCoef | kModePackedFma);
}

// kFwdShapes index of a launch shape when it is built as a fixed kernel, else 0.
template <int B, int T, int V, int MODE>
int fwd_shape_index(int warps, int gw, int stages)
{
    if constexpr (fwd_fixed_shapes<B, T, V, MODE>()) {
        for (int i = 1; i < kFwdNumShapes; ++i)
            if (kFwdShapes[i].warps == warps && kFwdShapes[i].gw == gw && kFwdShapes[i].stages == stages) return i;
    }
    return 0;
}

template <int B, int T, int V, int MODE, bool TMA>
constexpr bool fwd_built()
{
    if constexpr ((MODE & kModeSubtract) != 0)
        return TMA && V == 6 &&
               (MODE == (kModePackedFma | kModeSubtract) || MODE == (kModePackedFma | kModeSubtract | kModeNorms));
    if (fwd_all_modes<B, T>()) return true;
    if (!TMA) return V == 4 && (MODE == 0 || MODE == 2 || MODE == 3);
    return (V == 4 && MODE == 0) || ((V == 4 || V == 6 || V == 8) && (MODE == 2 || MODE == 3));
}

template <int B, int T, int V, int MODE>
cudaError_t launch_fwd_tv(const FwdArgs &a, const FwdLaunch &L, int sm_count, cudaStream_t s)
{
    ParamTab<B, T> ptab{};
    if constexpr ((MODE & kModeParamCoef) != 0) {
        if (!a.host_tab) return cudaErrorInvalidValue;
        for (int i = 0; i < wl_table_floats(B, T); ++i) ptab.v[i] = a.host_tab->v[i];
    }
    if (L.use_tma) {
        if constexpr (fwd_built<B, T, V, MODE, true>()) {
            const int threads = (L.warps + 1) * 32;
            const int S = L.warps * 32 * V;
            const int gw = (L.group > 0 && L.warps % L.group == 0) ? L.group : L.warps;
            const int64_t ntiles = (a.n + S - 1) / S;
            const size_t smem = fwd_tma_smem<B, T, V>(L.warps, gw, L.stages, (MODE & kModeNorms) != 0);
            const int sh = fwd_shape_index<B, T, V, MODE>(L.warps, gw, L.stages);
            void (*kern)(FwdArgs, int, int, int64_t, const ParamTab<B, T>) = fwd_tma_kernel<B, T, V, MODE, 0>;
            if constexpr (fwd_fixed_shapes<B, T, V, MODE>()) {
                if (sh == 1) kern = fwd_tma_kernel<B, T, V, MODE, 1>;
                if (sh == 2) kern = fwd_tma_kernel<B, T, V, MODE, 2>;
                if (sh == 3) kern = fwd_tma_kernel<B, T, V, MODE, 3>;
                if (sh == 4) kern = fwd_tma_kernel<B, T, V, MODE, 4>;
            }
            static SmemAttr smem_rec[kFwdNumShapes];   // per instantiation
            cudaError_t ae = ensure_smem(smem_rec[sh], (const void *)kern, smem);
            if (ae != cudaSuccess) return ae;
            static OccCache occ_rec[kFwdNumShapes];
            int occ = 0;
            ae = occupancy(occ_rec[sh], (const void *)kern, threads, smem, &occ);
            if (ae != cudaSuccess) return ae;
            if (occ < 1) return cudaErrorInvalidConfiguration;
            const int cps = (L.ctas_per_sm > 0 && L.ctas_per_sm < occ) ? L.ctas_per_sm : occ;
            int64_t grid = (int64_t)sm_count * cps;
            if (grid > ntiles) grid = ntiles;
            if constexpr ((MODE & kModeNorms) != 0)
                if (!a.norms || grid > kFwdNormSlots || L.warps > kFwdMaxWarps) return cudaErrorInvalidValue;
            // Programmatic dependent launch: this grid may begin launching while
            // the previous one in the stream drains (the kernel waits for it
            // before touching global memory).
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3((unsigned)threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, L.stages, gw, ntiles, ptab);
            count_launch();
            return e != cudaSuccess ? e : cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    if constexpr (fwd_built<B, T, V, MODE, false>()) {
        const int threads = 256;
        static OccCache occ_rec;
        int occ = 0;
        cudaError_t oe = occupancy(occ_rec, (const void *)fwd_ldg_kernel<B, T, V, MODE>, threads, 0, &occ);
        if (oe != cudaSuccess) return oe;
        if (occ < 1) occ = 1;
        const int64_t need = (a.n + (int64_t)threads * V - 1) / ((int64_t)threads * V);
        int64_t grid = (int64_t)sm_count * occ;
        if (grid > need) grid = need;
        fwd_ldg_kernel<B, T, V, MODE><<<(unsigned)grid, threads, 0, s>>>(a, ptab);
        count_launch();
        return cudaGetLastError();
    }
    return cudaErrorNotSupported;
}

template <int B, int T, int MODE>
cudaError_t launch_fwd_mode(const FwdArgs &a, const FwdLaunch &L, int sm_count, cudaStream_t s)
{
    switch (L.V) {
    case 2: return launch_fwd_tv<B, T, 2, MODE>(a, L, sm_count, s);
    case 4: return launch_fwd_tv<B, T, 4, MODE>(a, L, sm_count, s);
    case 6: return launch_fwd_tv<B, T, 6, MODE>(a, L, sm_count, s);
    case 8: return launch_fwd_tv<B, T, 8, MODE>(a, L, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int B, int T>
cudaError_t launch_fwd_t(const FwdArgs &a, const FwdLaunch &L, int sm_count, cudaStream_t s)
{
    switch (L.mode) {
    case 0: return launch_fwd_mode<B, T, 0>(a, L, sm_count, s);
    case 1: return launch_fwd_mode<B, T, 1>(a, L, sm_count, s);
    case 2: return launch_fwd_mode<B, T, 2>(a, L, sm_count, s);
    case 3: return launch_fwd_mode<B, T, 3>(a, L, sm_count, s);
    case kModePackedFma | kModeSubtract: return launch_fwd_mode<B, T, kModePackedFma | kModeSubtract>(a, L, sm_count, s);
    case kModePackedFma | kModeSubtract | kModeNorms:
        return launch_fwd_mode<B, T, kModePackedFma | kModeSubtract | kModeNorms>(a, L, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

#define DPD_DEFINE_LAUNCH_FWD(BB)                                                                  \
    template <>                                                                                    \
    cudaError_t launch_fwd<BB>(int T, const FwdArgs &a, const FwdLaunch &L, int sm_count,         \
                               cudaStream_t s)                                                     \
    {                                                                                              \
        switch (T) {                                                                               \
        case 1: return launch_fwd_t<BB, 1>(a, L, sm_count, s);                                     \
        case 2: return launch_fwd_t<BB, 2>(a, L, sm_count, s);                                     \
        case 3: return launch_fwd_t<BB, 3>(a, L, sm_count, s);                                     \
        case 4: return launch_fwd_t<BB, 4>(a, L, sm_count, s);                                     \
        case 5: return launch_fwd_t<BB, 5>(a, L, sm_count, s);                                     \
        case 6: return launch_fwd_t<BB, 6>(a, L, sm_count, s);                                     \
        case 7: return launch_fwd_t<BB, 7>(a, L, sm_count, s);                                     \
        case 8: return launch_fwd_t<BB, 8>(a, L, sm_count, s);                                     \
        default: return cudaErrorInvalidValue;                                                     \
        }                                                                                          \
    }

}  // namespace dpd
