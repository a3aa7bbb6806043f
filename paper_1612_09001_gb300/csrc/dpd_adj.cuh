// Adjoint of the APH DPD filter: gradients of a real loss L through y = DPD(x)
// with respect to the input samples and the coefficients, given gy = dL/dy,
// all under the convention grad = dL/dRe + j dL/dIm.
//
// With r = |x|^2, branch polynomials A_k(r) = sum_b h_{2b+1,k} r^b and
// C_k(r) = sum_b hbar_{2b+1,k} r^b (so that y_n = sum_k A_k(r_{n-k}) x_{n-k}
// + C_k(r_{n-k}) conj(x_{n-k}) + c, Eq. 1), the Wirtinger derivatives of the
// term of tap k are
//   dy/dx       = E_k(r) + G_k(r) conj(x)^2,   E = A + r A',  G = C'
//   dy/dconj(x) = F_k(r) x^2 + H_k(r),         F = A',        H = C + r C'
// and
//   gx_i = sum_k conj(dy_{i+k}/dx_i) gy_{i+k} + (dy_{i+k}/dconj(x_i)) conj(gy_{i+k})
//        = sum_k [conj(E_k) g + H_k conj(g)] + x_i^2 [conj(G_k) g + F_k conj(g)],  g = gy_{i+k}
// Each bracket is widely linear in g, so it is evaluated like the forward
// filter: four real Horner polynomials per bracket, run as two packed f32x2
// Horner chains whose results multiply the window sample {c, d} and its swap
// {d, c} (table built by wl_table_kernel, one float4 per power).
//
// The coefficient gradient is the correlation
//   gh_{(p,k)} = sum_j r_j^b conj(x_j) gy_{j+k},  gh_{(q,k)} = sum_j r_j^b x_j gy_{j+k},
//   gh_c = sum_n gy_n,
// i.e. conj(Psi)^T gy with the basis matrix Psi of Eq. 2.  Both branches come
// from two packed real correlations per (power, tap) (gh_accumulate), taken
// per thread over groups of up to five taps, reduced per CTA in a fixed order
// into a partials workspace and summed over CTAs in FP64 by
// adj_finalize_kernel.  The basis is recomputed from x: nothing from the
// forward pass is stored.
//
// Data movement.  For 16-byte aligned x and gy both gradients run as persistent
// kernels fed like the forward filter: one producer thread streams tiles of x
// and of gy (plus kHalo samples of look-ahead) into a ring of shared-memory
// slots with bulk copies completed on mbarriers, and the consumer warps read
// their windows from shared memory.  Other alignments (and callers without an
// error word) use the plain-load kernels, which read through L1.
#pragma once

#include "dpd_device.cuh"
#include "dpd_internal.h"

namespace dpd {

constexpr int kAdjV = 4;          // samples per thread (plain-load kernels, staged gx)
constexpr int kAdjGhV = 4;        // samples per thread of the staged gh kernel
constexpr int kAdjWarps = 8;      // consumer warps of the staged gx kernel
constexpr int kAdjGhWarps = 12;   // warps of the staged gh kernel (warp 0 also issues the copies)
constexpr int kAdjStages = 4;     // ring slots of the staged gx kernel
// Staged gh tile: 4 sub-blocks of V samples per thread (6144 samples), 2 ring
// slots (197 KB).  Measured on GB300 (2^24 samples, us): 2 x 4 slots 84.8 /
// 67.6 / 147.5, 3 x 3 83.9 / 62.7 / 142.8, 4 x 2 83.0 / 63.5 / 138.2 at
// P = Q = 9, M = 4 / P = Q = 7, M = 3 / P = Q = 11, M = 7: a longer tile spreads
// warp 0's wait for the slot release over more accumulation.
constexpr int kAdjGhStages = 2;   // ring slots of the staged gh kernel
constexpr int kAdjGhSub = 4;      // sub-blocks of V samples per thread and staged gh tile

// NS consecutive complex samples p[base .. base+NS-1] (zero past n).  When the
// buffer is 16-byte aligned, base is even and the rounded-up window lies inside
// the buffer, they are fetched as float4 pairs; otherwise sample by sample.
template <int NS>
__device__ __forceinline__ void adj_load_window(const float2 *__restrict__ p, int64_t base, int64_t n,
                                                bool vec, float2 (&out)[NS])
{
    constexpr int NV = (NS + 1) / 2;
    if (vec && (base & 1) == 0 && base + 2 * NV <= n) {
        const float4 *q = reinterpret_cast<const float4 *>(p + base);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float4 t = __ldg(q + j);
            out[2 * j] = make_float2(t.x, t.y);
            if (2 * j + 1 < NS) out[2 * j + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NS; ++j) out[j] = base + j < n ? __ldg(p + base + j) : make_float2(0.f, 0.f);
    }
}

// NS samples of a shared-memory slot from element `off`: float4 pairs when off
// is even (the slot holds the rounded-up window), else one by one.
template <int NS>
__device__ __forceinline__ void adj_slot_window(const float2 *slot, int off, float2 (&out)[NS])
{
    if ((off & 1) == 0) {
        const float4 *q = reinterpret_cast<const float4 *>(slot + off);
#pragma unroll
        for (int j = 0; j < (NS + 1) / 2; ++j) {
            const float4 t = q[j];
            out[2 * j] = make_float2(t.x, t.y);
            if (2 * j + 1 < NS) out[2 * j + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NS; ++j) out[j] = slot[off + j];
    }
}

// ---------------------------------------------------------------- staged tiles
// A slot holds x[s0, s0 + S) and, from element S on, gy[s0, s0 + S + halo);
// near the end of the signal only the even-length prefix that exists is copied.
// The look-ahead `halo` (even) covers the furthest gy sample a consumer reads
// for tile s0: kHalo for gx (T - 1 taps past its last sample, plus one for the
// float4 rounding of the window), kAdjGhHalo for the tap-grouped gh kernels.
__host__ __device__ constexpr int adj_slot_elems(int S, int halo = kHalo) { return 2 * S + halo; }

// The gh kernels read the window of taps k0 .. k0 + TG - 1 with k0 <= T - 1, so
// their look-ahead reaches T + TG - 2 samples (+1 for the float4 rounding).
constexpr int kAdjGhMaxTG = 5;
constexpr int kAdjGhHalo = kMaxT + kAdjGhMaxTG - 1;
static_assert(kAdjGhHalo % 2 == 0 && kHalo % 2 == 0, "slot parts must stay 16-byte aligned");

__device__ __forceinline__ void adj_slot_counts(int64_t s0, int S, int64_t n, int &xc, int &gc, int halo = kHalo)
{
    const int64_t rem = n - s0;
    xc = (int)((rem < S ? rem : (int64_t)S) & ~int64_t(1));
    gc = (int)((rem < S + halo ? rem : (int64_t)(S + halo)) & ~int64_t(1));
}

// NS samples of `src` from global index `g` whose slot copy starts at element
// `base` of the slot and holds `cnt` samples from global index s0.
template <int NS>
__device__ __forceinline__ void adj_slot_window_tail(const float2 *slot_part, int64_t s0, int cnt,
                                                     const float2 *__restrict__ src, int64_t g, int64_t n,
                                                     float2 (&out)[NS])
{
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int64_t gj = g + j;
        float2 v = make_float2(0.f, 0.f);
        if (gj - s0 < cnt)
            v = slot_part[gj - s0];
        else if (gj < n)
            v = __ldg(src + gj);
        out[j] = v;
    }
}

// The producer thread: stream every tile of this CTA into the ring.  Waits are
// bounded; after a failed wait the copies already issued are allowed to land
// before returning.
__device__ __forceinline__ void adj_produce(const AdjArgs &a, float2 *ring, uint64_t *bars, int stages, int S,
                                            int64_t ntiles, int halo = kHalo)
{
    const int slot_elems = adj_slot_elems(S, halo);
    int64_t it = 0;
    bool ok = true;
    int s = 0;          // slot and parity of tile `it`, kept incrementally (no division per tile)
    uint32_t ph = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        if (it > 0 && ++s == stages) {
            s = 0;
            ph ^= 1u;
        }
        if (it >= stages && !mbar_wait(smem_addr(&bars[stages + s]), ph ^ 1u, a.status)) {
            ok = false;
            break;
        }
        if (it == 1 && !mbar_wait(smem_addr(&bars[0]), 0u, a.status)) {   // start-up: first tile first
            ok = false;
            break;
        }
        const int64_t s0 = tile * S;
        int xc, gc;
        adj_slot_counts(s0, S, a.n, xc, gc, halo);
        const uint32_t fb = smem_addr(&bars[s]);
        mbar_arrive_expect_tx(fb, (uint32_t)(xc + gc) * (uint32_t)sizeof(float2));
        float2 *slot = ring + (size_t)s * slot_elems;
        if (xc) bulk_copy_g2s(smem_addr(slot), a.x + s0, (uint32_t)xc * sizeof(float2), fb);
        if (gc) bulk_copy_g2s(smem_addr(slot + S), a.gy + s0, (uint32_t)gc * sizeof(float2), fb);
    }
    if (!ok) {
        const int64_t first = it > stages ? it - stages : 0;
        for (int64_t j = first; j < it; ++j)
            mbar_wait(smem_addr(&bars[j % stages]), (uint32_t)((j / stages) & 1), a.status);
    }
}

// Shared-memory bytes of a staged kernel: barriers, reduction scratch, ring.
__host__ __device__ constexpr size_t adj_staged_smem(int S, int stages, int scratch_floats, int halo = kHalo)
{
    return 128 + (((size_t)scratch_floats * 4 + 127) / 128) * 128 +
           (size_t)stages * (size_t)adj_slot_elems(S, halo) * sizeof(float2);
}

// ---------------------------------------------------------------- input gradient
// Adjoint table passed by value (kernel parameter bank), 16-byte aligned so
// that its packed pairs can be 64-bit constant operands.
template <int B, int T>
struct alignas(8) AdjParamTab {
    float v[adj_table_floats(B, T)];
};

// gx for the V samples i0.. from their x (xs) and the gy window g (samples
// i0 .. i0 + V + T - 2).  The adjoint table of the model comes from shared
// memory (tab) or, with PARAM, from the parameter bank (ptab), whose entries
// the packed FMAs take as operands directly.
template <int B, int T, int V, bool PARAM = false>
__device__ __forceinline__ void gx_compute(const float *tab, const AdjParamTab<B, T> &ptab,
                                           const float2 (&xs)[V], const float2 (&g)[V + T - 1], float2 (&acc)[V])
{
    constexpr int QB = B, RB = B - 1;       // coefficients per Q / S polynomial
    constexpr int PER_TAP = 4 * QB + 4 * RB;
    constexpr int W = V + T - 1;
    float2 gs[W];   // window samples swapped: {d, c}
#pragma unroll
    for (int j = 0; j < W; ++j) gs[j] = make_float2(g[j].y, g[j].x);
    float ur[V], ui[V], rr[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float2 q = xs[v];
        rr[v] = fmaf(q.x, q.x, q.y * q.y);
        ur[v] = fmaf(q.x, q.x, -q.y * q.y);   // x^2
        ui[v] = 2.f * q.x * q.y;
    }
    // {Re, Im} of the gradient of each sample, and of the tap sum of the second
    // bracket (its factor x^2 does not depend on the tap, so it is applied once
    // after the tap loop).  Every tap advances all V samples together with
    // packed f32x2 FMAs (coefficient pairs adjacent in the table).
    float2 ws[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        acc[v] = make_float2(0.f, 0.f);
        ws[v] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < T; ++k) {
        // quadruple j of tap k's block: the Q quadruples, then the S ones
        auto coef = [&](int j) -> float4 {
            if constexpr (PARAM) {
                const int o = PER_TAP * k + 4 * j;
                return make_float4(ptab.v[o], ptab.v[o + 1], ptab.v[o + 2], ptab.v[o + 3]);
            } else {
                return reinterpret_cast<const float4 *>(tab + PER_TAP * k)[j];
            }
        };
        float2 pa[V], pb[V];
        {
            const float4 c4 = coef(QB - 1);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                pa[v] = make_float2(c4.x, c4.y);
                pb[v] = make_float2(c4.z, c4.w);
            }
        }
#pragma unroll
        for (int m = QB - 2; m >= 0; --m) {
            const float4 c4 = coef(m);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 rr2 = make_float2(rr[v], rr[v]);
                pa[v] = __ffma2_rn(pa[v], rr2, make_float2(c4.x, c4.y));
                pb[v] = __ffma2_rn(pb[v], rr2, make_float2(c4.z, c4.w));
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc[v] = __ffma2_rn(pa[v], g[v + k], acc[v]);    // {Q0 c, Q3 d}
            acc[v] = __ffma2_rn(pb[v], gs[v + k], acc[v]);   // {Q1 d, Q2 c}
        }
        if constexpr (RB > 0) {
            float2 sa[V], sb[V];
            {
                const float4 c4 = coef(QB + RB - 1);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    sa[v] = make_float2(c4.x, c4.y);
                    sb[v] = make_float2(c4.z, c4.w);
                }
            }
#pragma unroll
            for (int m = RB - 2; m >= 0; --m) {
                const float4 c4 = coef(QB + m);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float2 rr2 = make_float2(rr[v], rr[v]);
                    sa[v] = __ffma2_rn(sa[v], rr2, make_float2(c4.x, c4.y));
                    sb[v] = __ffma2_rn(sb[v], rr2, make_float2(c4.z, c4.w));
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                // conj(G) g + F conj(g) = {S0 c + S1 d, S2 c + S3 d}
                ws[v] = __ffma2_rn(sa[v], g[v + k], ws[v]);    // {S0 c, S3 d}
                ws[v] = __ffma2_rn(sb[v], gs[v + k], ws[v]);   // {S1 d, S2 c}
            }
        }
    }
    if constexpr (RB > 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // acc += x^2 ws (complex):  {ur wr - ui wi, ur wi + ui wr}
            acc[v] = __ffma2_rn(make_float2(ur[v], ur[v]), ws[v], acc[v]);
            acc[v] = __ffma2_rn(make_float2(-ui[v], ui[v]), make_float2(ws[v].y, ws[v].x), acc[v]);
        }
    }
}

template <int V>
__device__ __forceinline__ void gx_store(float2 *__restrict__ gx, int64_t i0, int64_t n, bool vec,
                                         const float2 (&acc)[V], bool streaming)
{
    if (vec && i0 + V <= n) {
        float4 *o = reinterpret_cast<float4 *>(gx + i0);
#pragma unroll
        for (int j = 0; j < V / 2; ++j) {
            const float4 q = make_float4(acc[2 * j].x, acc[2 * j].y, acc[2 * j + 1].x, acc[2 * j + 1].y);
            if (streaming)
                st_stream_f4(o + j, q);
            else
                o[j] = q;
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (i0 + v < n) gx[i0 + v] = acc[v];
    }
}

template <int B, int T>
__host__ __device__ constexpr int adj_tab_padded() { return ((adj_table_floats(B, T) + 3) / 4) * 4; }

// Plain-load variant (any 8-byte alignment): grid-stride over V-sample runs.
template <int B, int T, int V>
__global__ void __launch_bounds__(256) adj_gx_kernel(AdjArgs a)
{
    constexpr int W = V + T - 1;            // gy window: samples i0 .. i0 + V + T - 2
    constexpr int TABF = adj_table_floats(B, T);
    __shared__ __align__(16) float tab[adj_tab_padded<B, T>()];
    for (int i = threadIdx.x; i < TABF; i += blockDim.x) tab[i] = a.adj_tab[i];
    __syncthreads();

    static_assert(V % 2 == 0, "V samples are stored as float4 pairs");
    const bool vec_in = ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.gy)) & 15) == 0;
    const bool vec_out = (reinterpret_cast<uintptr_t>(a.gx) & 15) == 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; i0 < a.n; i0 += stride) {
        float2 xs[V], g[W], acc[V];
        adj_load_window<V>(a.x, i0, a.n, vec_in, xs);
        adj_load_window<W>(a.gy, i0, a.n, vec_in, g);
        gx_compute<B, T, V>(tab, *reinterpret_cast<const AdjParamTab<B, T> *>(tab), xs, g, acc);
        gx_store<V>(a.gx, i0, a.n, vec_out, acc, false);
    }
}

// Staged variant: persistent CTAs of kAdjWarps consumer warps + 1 producer warp
// walk tiles of S = kAdjWarps * 32 * V samples.  x and gy 16-byte aligned.
template <int B, int T, int V, bool PARAM>
__global__ void __launch_bounds__(32 * (kAdjWarps + 1))
    adj_gx_tma_kernel(AdjArgs a, int stages, int64_t ntiles, const __grid_constant__ AdjParamTab<B, T> ptab)
{
    constexpr int W = V + T - 1;
    constexpr int TABF = adj_table_floats(B, T);
    constexpr int S = kAdjWarps * 32 * V;
    static_assert(T - 1 <= kHalo, "look-ahead must fit the slot");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);   // full[s], empty[s]
    float *tab = reinterpret_cast<float *>(smem + 128);
    float2 *ring = reinterpret_cast<float2 *>(smem + adj_staged_smem(S, 0, adj_tab_padded<B, T>()));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_addr(&bars[s]), 1);
            mbar_init(smem_addr(&bars[stages + s]), kAdjWarps);
        }
        fence_barrier_init();
    }
    if constexpr (!PARAM)
        for (int i = tid; i < TABF; i += blockDim.x) tab[i] = a.adj_tab[i];
    __syncthreads();
    if (warp == kAdjWarps) {
        if (lane == 0) adj_produce(a, ring, bars, stages, S, ntiles);
        return;
    }
    const bool vec_out = (reinterpret_cast<uintptr_t>(a.gx) & 15) == 0;
    const int slot_elems = adj_slot_elems(S);
    int s = 0;          // slot and parity of the current tile, kept incrementally
    uint32_t ph = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (!mbar_wait(smem_addr(&bars[s]), ph, a.status)) return;
        const float2 *slot = ring + (size_t)s * slot_elems;
        const int64_t s0 = tile * S;
        const int off = tid * V;
        const bool full = s0 + S + kHalo <= a.n;
        float2 xs[V], g[W];
        if (full) {
            adj_slot_window<V>(slot, off, xs);
            adj_slot_window<W>(slot + S, off, g);
        } else {
            int xc, gc;
            adj_slot_counts(s0, S, a.n, xc, gc);
            adj_slot_window_tail<V>(slot, s0, xc, a.x, s0 + off, a.n, xs);
            adj_slot_window_tail<W>(slot + S, s0, gc, a.gy, s0 + off, a.n, g);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bars[stages + s]));
        if (++s == stages) {
            s = 0;
            ph ^= 1u;
        }
        float2 acc[V];
        gx_compute<B, T, V, PARAM>(tab, ptab, xs, g, acc);
        gx_store<V>(a.gx, s0 + off, a.n, vec_out, acc, true);
    }
}

// ---------------------------------------------------------------- coefficient gradient
// Tap groups: group y owns taps [y*TG, y*TG + TG) of every branch; group 0 also
// owns the LO-leakage term.  Each CTA writes one row of partials (K complex),
// only at the indices of its group.
//
// With a_b = r^b Re x, c_b = r^b Im x and g = gy_{j+k} = c + j d, both branches
// follow from two packed correlations per (b, k):
//   X_{b,k} = sum_j {a_b, c_b}_j * {c, d},   Y_{b,k} = sum_j {a_b, c_b}_j * {d, c},
//   main  sum r^b conj(x) g = {X.x + X.y, Y.x - Y.y},
//   conj  sum r^b x g       = {X.x - X.y, Y.x + Y.y},
// so every (sample, b, tap) costs two packed f32x2 FMAs whose operands are the
// packed power {a_b, c_b} and the window sample as stored or swapped (once per
// window sample): no per-product broadcasts.  Accumulators per thread:
// [b*TG + kk] X, [B*TG + b*TG + kk] Y, last sum g (for c).
template <int B, int TG, int V>
__device__ __forceinline__ void gh_accumulate(const float2 (&xs)[V], const float2 (&g)[V + TG - 1], bool group0,
                                              float2 (&acc2)[2 * B * TG + 1])
{
    constexpr int NP = 2 * B * TG + 1;
    constexpr int NG = V + TG - 1;
    if (group0) {
#pragma unroll
        for (int v = 0; v < V; ++v)   // the gy window starts at the sample itself for group 0
            acc2[NP - 1] = __fadd2_rn(acc2[NP - 1], g[v]);
    }
    float2 gs[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) gs[j] = make_float2(g[j].y, g[j].x);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float r = fmaf(xs[v].x, xs[v].x, xs[v].y * xs[v].y);
        float2 p = xs[v];   // {a_b, c_b}
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (b > 0) p = __fmul2_rn(p, make_float2(r, r));
#pragma unroll
            for (int kk = 0; kk < TG; ++kk) {
                acc2[b * TG + kk] = __ffma2_rn(p, g[v + kk], acc2[b * TG + kk]);
                acc2[B * TG + b * TG + kk] = __ffma2_rn(p, gs[v + kk], acc2[B * TG + b * TG + kk]);
            }
        }
    }
}

// Fixed-order reduction of the accumulators of `nw` warps (threads tid < 32*nw
// take part; `red` holds nw * NA floats), then one row of partials.  NAMED:
// synchronise on named barrier 1 (the staged kernels, whose producer warp has
// left) instead of __syncthreads.
template <int B, int TG, bool NAMED>
__device__ __forceinline__ void gh_reduce_row(float2 (&acc2)[2 * B * TG + 1], float *red, int nw, int tid, int k0,
                                              bool group0, int T, int Bp, int Bq, float2 *row)
{
    constexpr int NP = 2 * B * TG + 1;
    constexpr int NA = 2 * NP;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float2 v = acc2[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        acc2[i] = v;
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            red[warp * NA + 2 * i] = acc2[i].x;
            red[warp * NA + 2 * i + 1] = acc2[i].y;
        }
    }
    if constexpr (NAMED)
        asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
    else
        __syncthreads();
    // One (b, kk) pair per thread: X and Y summed over the warps in index
    // order, then both branches.
    for (int e = tid; e <= B * TG; e += nw * 32) {
        float q[4] = {0.f, 0.f, 0.f, 0.f};
        const int i0 = e < B * TG ? 2 * e : 2 * (NP - 1), i1 = 2 * (B * TG + e);
        for (int w2 = 0; w2 < nw; ++w2) {
            const float *rw = red + w2 * NA;
            q[0] += rw[i0];
            q[1] += rw[i0 + 1];
            if (e < B * TG) {
                q[2] += rw[i1];
                q[3] += rw[i1 + 1];
            }
        }
        if (e == B * TG) {
            if (group0) row[(Bp + Bq) * T] = make_float2(q[0], q[1]);
            continue;
        }
        const int b = e / TG, kk = e % TG;
        if (k0 + kk >= T) continue;
        if (b < Bp) row[b * T + k0 + kk] = make_float2(q[0] + q[1], q[2] - q[3]);
        if (b < Bq) row[(Bp + b) * T + k0 + kk] = make_float2(q[0] - q[1], q[2] + q[3]);
    }
}

// Plain-load variant: grid (blocks, tap groups), 256 threads.
template <int B, int TG, int V>
__global__ void __launch_bounds__(256) adj_gh_kernel(AdjArgs a, int T, int Bp, int Bq, int K)
{
    constexpr int NA = 4 * B * TG + 2;
    constexpr int NP = NA / 2;
    const int k0 = blockIdx.y * TG;
    float2 acc2[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc2[i] = make_float2(0.f, 0.f);

    const bool vec_in = ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.gy)) & 15) == 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    for (int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; j0 < a.n; j0 += stride) {
        float2 xs[V], g[V + TG - 1];
        adj_load_window<V>(a.x, j0, a.n, vec_in, xs);
        adj_load_window<V + TG - 1>(a.gy, j0 + k0, a.n, vec_in, g);
        gh_accumulate<B, TG, V>(xs, g, blockIdx.y == 0, acc2);
    }
    __shared__ float red[8 * NA];
    gh_reduce_row<B, TG, false>(acc2, red, blockDim.x >> 5, threadIdx.x, k0, blockIdx.y == 0, T, Bp, Bq,
                                a.partials + (size_t)blockIdx.x * K);
}

// Staged variant: grid (blocks, tap groups) of persistent CTAs of kAdjGhWarps
// warps, every CTA streaming the tiles of its blockIdx.x share.  x and gy
// 16-byte aligned.  With 2 B TG + 1 packed accumulators a thread takes about
// 170 registers, so one CTA fits an SM; the bulk copies are issued by lane 0
// of warp 0 between its own tiles instead of by a separate producer warp, so
// that all twelve warps (three per SM sub-partition) accumulate.  At the start
// of its tile i warp 0 refills the slot of tile i - 1 (once every warp has
// released it) with tile i - 1 + stages; the whole warp waits, so that its
// lanes stay converged.
template <int B, int TG, int V>
__device__ __forceinline__ void adj_gh_tma_body(const AdjArgs &a, int stages, int64_t ntiles, int T, int Bp, int Bq,
                                                int K)
{
    constexpr int NA = 4 * B * TG + 2;
    constexpr int NP = NA / 2;
    constexpr int S = kAdjGhWarps * 32 * V * kAdjGhSub;
    constexpr int NG = V + TG - 1;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);   // full[s], empty[s]
    float *red = reinterpret_cast<float *>(smem + 128);
    static_assert(TG <= kAdjGhMaxTG, "tap group exceeds the staged look-ahead");
    float2 *ring = reinterpret_cast<float2 *>(smem + adj_staged_smem(S, 0, kAdjGhWarps * NA, kAdjGhHalo));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = blockIdx.y * TG;
    const bool group0 = blockIdx.y == 0;
    const bool producer = tid == 0;
    const int slot_elems = adj_slot_elems(S, kAdjGhHalo);
    // Local tile i of this CTA is global tile blockIdx.x + i * gridDim.x.
    const int64_t nlocal = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto issue = [&](int64_t i) {   // producer: tile i into slot i % stages (its empty phase passed)
        const int sl = (int)(i % stages);
        const int64_t s0 = ((int64_t)blockIdx.x + i * gridDim.x) * S;
        int xc, gc;
        adj_slot_counts(s0, S, a.n, xc, gc, kAdjGhHalo);
        const uint32_t fb = smem_addr(&bars[sl]);
        float2 *slot = ring + (size_t)sl * slot_elems;
        mbar_arrive_expect_tx(fb, (uint32_t)(xc + gc) * (uint32_t)sizeof(float2));
        if (xc) bulk_copy_g2s(smem_addr(slot), a.x + s0, (uint32_t)xc * sizeof(float2), fb);
        if (gc) bulk_copy_g2s(smem_addr(slot + S), a.gy + s0, (uint32_t)gc * sizeof(float2), fb);
    };
    if (producer) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_addr(&bars[s]), 1);
            mbar_init(smem_addr(&bars[stages + s]), kAdjGhWarps);
        }
        fence_barrier_init();
    }
    __syncthreads();
    int64_t issued = 0;   // tiles issued so far (kept by every lane of warp 0)
    if (warp == 0)
        for (; issued < stages && issued < nlocal; ++issued)
            if (producer) issue(issued);
    float2 acc2[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc2[i] = make_float2(0.f, 0.f);
    int s = 0;          // slot and parity of the current tile, kept incrementally
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t i = 0; i < nlocal; ++i) {
        // A failed wait (error word set) ends this warp's tiles; it still joins
        // the reduction so that no warp waits for it.
        if (!mbar_wait(smem_addr(&bars[s]), ph, a.status)) {
            ok = false;
            break;
        }
        // Refill: tile i - 1 + stages into the slot of tile i - 1, once all
        // warps have released that tile (empty phase (i - 1) / stages).
        if (warp == 0 && i >= 1 && issued < nlocal) {
            const int64_t done = i - 1;
            bool w = mbar_wait(smem_addr(&bars[stages + (int)(done % stages)]), (uint32_t)((done / stages) & 1),
                               a.status);
            w = __shfl_sync(0xffffffffu, w, 0);   // lane 0's outcome for the whole warp
            if (!w) {
                ok = false;
                break;
            }
            if (producer) issue(issued);
            ++issued;
            __syncwarp();
        }
        const float2 *slot = ring + (size_t)s * slot_elems;
        const int64_t s0 = ((int64_t)blockIdx.x + i * gridDim.x) * S;
        const bool fast = s0 + S + kAdjGhHalo <= a.n;
        int xc = S, gc = S + kAdjGhHalo;
        if (!fast) adj_slot_counts(s0, S, a.n, xc, gc, kAdjGhHalo);
        // Sub-block j of the tile: samples (j * threads + tid) * V ..; the slot
        // is released once the last sub-block's windows are in registers.
#pragma unroll 1
        for (int j = 0; j < kAdjGhSub; ++j) {
            const int off = (j * kAdjGhWarps * 32 + tid) * V;
            float2 xs[V], g[NG];
            if (fast) {
                adj_slot_window<V>(slot, off, xs);
                adj_slot_window<NG>(slot + S, off + k0, g);
            } else {
                adj_slot_window_tail<V>(slot, s0, xc, a.x, s0 + off, a.n, xs);
                adj_slot_window_tail<NG>(slot + S, s0, gc, a.gy, s0 + off + k0, a.n, g);
            }
            if (j == kAdjGhSub - 1) {
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&bars[stages + s]));
            }
            gh_accumulate<B, TG, V>(xs, g, group0, acc2);
        }
        if (++s == stages) {
            s = 0;
            ph ^= 1u;
        }
    }
    if (producer && !ok) {
        // Let the copies already issued land before the CTA exits.
        const int64_t first = issued > stages ? issued - stages : 0;
        for (int64_t q = first; q < issued; ++q)
            mbar_wait(smem_addr(&bars[q % stages]), (uint32_t)((q / stages) & 1), a.status);
    }
    gh_reduce_row<B, TG, false>(acc2, red, kAdjGhWarps, tid, k0, group0, T, Bp, Bq,
                                a.partials + (size_t)blockIdx.x * K);
}

template <int B, int TG, int V>
__global__ void __launch_bounds__(32 * kAdjGhWarps, 1)
    adj_gh_tma_kernel(AdjArgs a, int stages, int64_t ntiles, int T, int Bp, int Bq, int K)
{
    adj_gh_tma_body<B, TG, V>(a, stages, ntiles, T, Bp, Bq, K);
}

// Many independent problems in one launch (the least-squares refinement of a
// batch): grid (CTAs per problem, tap groups, problems); problem z's
// arguments (x, gy, n, its own partials rows, 16-byte aligned buffers) come
// from args[z].
template <int B, int TG, int V>
__global__ void __launch_bounds__(32 * kAdjGhWarps, 1)
    adj_gh_tma_batched_kernel(const AdjArgs *__restrict__ args, int stages, int T, int Bp, int Bq, int K)
{
    constexpr int S = kAdjGhWarps * 32 * V * kAdjGhSub;
    const AdjArgs a = args[blockIdx.z];
    adj_gh_tma_body<B, TG, V>(a, stages, (a.n + S - 1) / S, T, Bp, Bq, K);
}

// ---------------------------------------------------------------- launches
inline bool adj_staged_ok(const AdjArgs &a)
{
    return a.status != nullptr &&
           ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.gy)) & 15) == 0;
}

template <int B, int T, int V, bool PARAM>
cudaError_t launch_adj_gx_tma(const AdjArgs &a, const AdjParamTab<B, T> &ptab, int sm_count, cudaStream_t s)
{
    constexpr int S = kAdjWarps * 32 * V;
    // The shared-memory table area is kept in both forms (it is small).
    const size_t smem = adj_staged_smem(S, kAdjStages, adj_tab_padded<B, T>());
    auto kern = adj_gx_tma_kernel<B, T, V, PARAM>;
    static SmemAttr smem_rec;
    cudaError_t attr = ensure_smem(smem_rec, (const void *)kern, smem);
    if (attr != cudaSuccess) return attr;
    static OccCache occ_rec;
    int occ = 0;
    attr = occupancy(occ_rec, (const void *)kern, 32 * (kAdjWarps + 1), smem, &occ);
    if (attr != cudaSuccess) return attr;
    if (occ < 1) occ = 1;
    const int64_t ntiles = (a.n + S - 1) / S;
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > ntiles) grid = ntiles;
    kern<<<(unsigned)grid, 32 * (kAdjWarps + 1), smem, s>>>(a, kAdjStages, ntiles, ptab);
    count_launch();
    return cudaGetLastError();
}

template <int B, int T>
cudaError_t launch_adj_gx_t(const AdjArgs &a, int sm_count, cudaStream_t s)
{
    constexpr int V = kAdjV;
    if (adj_staged_ok(a)) {
        if (a.host_adj_tab) {
            AdjParamTab<B, T> ptab;
            for (int i = 0; i < adj_table_floats(B, T); ++i) ptab.v[i] = a.host_adj_tab[i];
            return launch_adj_gx_tma<B, T, V, true>(a, ptab, sm_count, s);
        }
        return launch_adj_gx_tma<B, T, V, false>(a, AdjParamTab<B, T>{}, sm_count, s);
    }
    static OccCache occ_rec;
    int occ = 0;
    const cudaError_t oe = occupancy(occ_rec, (const void *)adj_gx_kernel<B, T, V>, 256, 0, &occ);
    if (oe != cudaSuccess) return oe;
    if (occ < 1) occ = 1;
    const int64_t need = (a.n + 256 * V - 1) / (256 * V);
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > need) grid = need;
    adj_gx_kernel<B, T, V><<<(unsigned)grid, 256, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int B, int TG>
cudaError_t launch_adj_gh_tg(const AdjArgs &a, int blocks, int T, int Bp, int Bq, int K, cudaStream_t s)
{
    const int groups = (T + TG - 1) / TG;
    dim3 grid((unsigned)blocks, (unsigned)groups);
    if (adj_staged_ok(a)) {
        constexpr int V = kAdjGhV;
        constexpr int S = kAdjGhWarps * 32 * V * kAdjGhSub;
        constexpr int NA = 4 * B * TG + 2;
        const size_t smem = adj_staged_smem(S, kAdjGhStages, kAdjGhWarps * NA, kAdjGhHalo);
        static SmemAttr smem_rec;
        const cudaError_t attr = ensure_smem(smem_rec, (const void *)adj_gh_tma_kernel<B, TG, V>, smem);
        if (attr != cudaSuccess) return attr;
        const int64_t ntiles = (a.n + S - 1) / S;
        adj_gh_tma_kernel<B, TG, V><<<grid, 32 * kAdjGhWarps, smem, s>>>(a, kAdjGhStages, ntiles, T, Bp, Bq, K);
        count_launch();
        return cudaGetLastError();
    }
    adj_gh_kernel<B, TG, kAdjV><<<grid, 256, 0, s>>>(a, T, Bp, Bq, K);
    count_launch();
    return cudaGetLastError();
}

// gh: the tap-group size (1, 2 or 4 taps per group) and the CTAs per group
// (= rows of partials, already clamped by the caller).
template <int B>
cudaError_t launch_adj_gh(const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K, cudaStream_t s)
{
    switch (L.tap_group) {
    case 1: return launch_adj_gh_tg<B, 1>(a, L.gh_blocks, T, Bp, Bq, K, s);
    case 2: return launch_adj_gh_tg<B, 2>(a, L.gh_blocks, T, Bp, Bq, K, s);
    case 3: return launch_adj_gh_tg<B, 3>(a, L.gh_blocks, T, Bp, Bq, K, s);
    case 4: return launch_adj_gh_tg<B, 4>(a, L.gh_blocks, T, Bp, Bq, K, s);
    case 5: return launch_adj_gh_tg<B, 5>(a, L.gh_blocks, T, Bp, Bq, K, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int B, int TG>
cudaError_t launch_adj_gh_batched_tg(const AdjArgs *args, int count, int blocks, int T, int Bp, int Bq, int K,
                                     cudaStream_t s)
{
    constexpr int V = kAdjGhV;
    constexpr int S = kAdjGhWarps * 32 * V * kAdjGhSub;
    constexpr int NA = 4 * B * TG + 2;
    const size_t smem = adj_staged_smem(S, kAdjGhStages, kAdjGhWarps * NA, kAdjGhHalo);
    static SmemAttr smem_rec;
    const cudaError_t attr = ensure_smem(smem_rec, (const void *)adj_gh_tma_batched_kernel<B, TG, V>, smem);
    if (attr != cudaSuccess) return attr;
    dim3 grid((unsigned)blocks, (unsigned)((T + TG - 1) / TG), (unsigned)count);
    adj_gh_tma_batched_kernel<B, TG, V><<<grid, 32 * kAdjGhWarps, smem, s>>>(args, kAdjGhStages, T, Bp, Bq, K);
    count_launch();
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_adj_gh_batched(const AdjArgs *args, int count, int blocks, int tap_group, int T, int Bp, int Bq,
                                  int K, cudaStream_t s)
{
    switch (tap_group) {
    case 1: return launch_adj_gh_batched_tg<B, 1>(args, count, blocks, T, Bp, Bq, K, s);
    case 2: return launch_adj_gh_batched_tg<B, 2>(args, count, blocks, T, Bp, Bq, K, s);
    case 3: return launch_adj_gh_batched_tg<B, 3>(args, count, blocks, T, Bp, Bq, K, s);
    case 4: return launch_adj_gh_batched_tg<B, 4>(args, count, blocks, T, Bp, Bq, K, s);
    case 5: return launch_adj_gh_batched_tg<B, 5>(args, count, blocks, T, Bp, Bq, K, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int B>
cudaError_t launch_adj_gx(const AdjArgs &a, int T, int sm_count, cudaStream_t s)
{
    switch (T) {
    case 1: return launch_adj_gx_t<B, 1>(a, sm_count, s);
    case 2: return launch_adj_gx_t<B, 2>(a, sm_count, s);
    case 3: return launch_adj_gx_t<B, 3>(a, sm_count, s);
    case 4: return launch_adj_gx_t<B, 4>(a, sm_count, s);
    case 5: return launch_adj_gx_t<B, 5>(a, sm_count, s);
    case 6: return launch_adj_gx_t<B, 6>(a, sm_count, s);
    case 7: return launch_adj_gx_t<B, 7>(a, sm_count, s);
    case 8: return launch_adj_gx_t<B, 8>(a, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

#define DPD_DEFINE_LAUNCH_ADJ(BB)                                                                  \
    template <>                                                                                    \
    cudaError_t launch_adj<BB>(const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K, \
                               int sm_count, cudaStream_t s)                                       \
    {                                                                                              \
        if (a.gx) {                                                                                \
            cudaError_t e = launch_adj_gx<BB>(a, T, sm_count, s);                                  \
            if (e != cudaSuccess) return e;                                                        \
        }                                                                                          \
        if (a.partials) return launch_adj_gh<BB>(a, L, T, Bp, Bq, K, s);                           \
        return cudaSuccess;                                                                        \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t launch_adj_gh_many<BB>(const AdjArgs *args, int count, int blocks, int tap_group,  \
                                       int T, int Bp, int Bq, int K, cudaStream_t s)               \
    {                                                                                              \
        return launch_adj_gh_batched<BB>(args, count, blocks, tap_group, T, Bp, Bq, K, s);          \
    }

}  // namespace dpd
