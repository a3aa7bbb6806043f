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
// filter: four real Horner polynomials per bracket (table built by
// adj_table_kernel).  The coefficient gradient is the correlation
//   gh_{(p,k)} = sum_j r_j^b conj(x_j) gy_{j+k},  gh_{(q,k)} = sum_j r_j^b x_j gy_{j+k},
//   gh_c = sum_n gy_n,
// i.e. conj(Psi)^T gy with the basis matrix Psi of Eq. 2, accumulated per
// thread, reduced per CTA in a fixed order into a partials workspace and summed
// over CTAs in FP64 by adj_finalize_kernel.  The basis is recomputed from x:
// nothing from the forward pass is stored.
#pragma once

#include "dpd_device.cuh"
#include "dpd_internal.h"

namespace dpd {

// ---------------------------------------------------------------- input gradient
template <int B, int T, int V>
__global__ void __launch_bounds__(256) adj_gx_kernel(AdjArgs a)
{
    constexpr int W = V + T - 1;            // gy window: samples i0 .. i0 + V + T - 2
    constexpr int QB = B, RB = B - 1;       // coefficients per Q / R polynomial
    constexpr int PER_TAP = 4 * QB + 4 * RB;
    constexpr int TABF = PER_TAP * T;
    __shared__ __align__(16) float tab[((TABF + 3) / 4) * 4 + 4];
    for (int i = threadIdx.x; i < TABF; i += blockDim.x) tab[i] = a.adj_tab[i];
    __syncthreads();

    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; i0 < a.n; i0 += stride) {
        float xr[V], xi[V], ur[V], ui[V], rr[V];
        float gr[W], gi[W];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float2 q = make_float2(0.f, 0.f);
            if (i0 + v < a.n) q = __ldg(a.x + i0 + v);
            xr[v] = q.x;
            xi[v] = q.y;
            rr[v] = fmaf(q.x, q.x, q.y * q.y);
            ur[v] = fmaf(q.x, q.x, -q.y * q.y);   // x^2
            ui[v] = 2.f * q.x * q.y;
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            float2 q = make_float2(0.f, 0.f);
            if (i0 + j < a.n) q = __ldg(a.gy + i0 + j);
            gr[j] = q.x;
            gi[j] = q.y;
        }
        float oR[V], oI[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            oR[v] = 0.f;
            oI[v] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const float *tk = tab + PER_TAP * k;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float c = gr[v + k], d = gi[v + k], r = rr[v];
                float q0 = tk[0 * QB + QB - 1], q1 = tk[1 * QB + QB - 1];
                float q2 = tk[2 * QB + QB - 1], q3 = tk[3 * QB + QB - 1];
#pragma unroll
                for (int m = QB - 2; m >= 0; --m) {
                    q0 = fmaf(q0, r, tk[0 * QB + m]);
                    q1 = fmaf(q1, r, tk[1 * QB + m]);
                    q2 = fmaf(q2, r, tk[2 * QB + m]);
                    q3 = fmaf(q3, r, tk[3 * QB + m]);
                }
                oR[v] = fmaf(q0, c, oR[v]);
                oR[v] = fmaf(q1, d, oR[v]);
                oI[v] = fmaf(q2, c, oI[v]);
                oI[v] = fmaf(q3, d, oI[v]);
                if constexpr (RB > 0) {
                    const float *rk = tk + 4 * QB;
                    float s0 = rk[0 * RB + RB - 1], s1 = rk[1 * RB + RB - 1];
                    float s2 = rk[2 * RB + RB - 1], s3 = rk[3 * RB + RB - 1];
#pragma unroll
                    for (int m = RB - 2; m >= 0; --m) {
                        s0 = fmaf(s0, r, rk[0 * RB + m]);
                        s1 = fmaf(s1, r, rk[1 * RB + m]);
                        s2 = fmaf(s2, r, rk[2 * RB + m]);
                        s3 = fmaf(s3, r, rk[3 * RB + m]);
                    }
                    const float wr = fmaf(s0, c, s1 * d);   // conj(G) g + F conj(g)
                    const float wi = fmaf(s2, c, s3 * d);
                    oR[v] = fmaf(ur[v], wr, oR[v]);
                    oR[v] = fmaf(-ui[v], wi, oR[v]);
                    oI[v] = fmaf(ur[v], wi, oI[v]);
                    oI[v] = fmaf(ui[v], wr, oI[v]);
                }
            }
        }
        (void)xr;
        (void)xi;
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (i0 + v < a.n) a.gx[i0 + v] = make_float2(oR[v], oI[v]);
    }
}

// ---------------------------------------------------------------- coefficient gradient
// Grid (blocks, tap groups): group g owns taps [g*TG, g*TG + TG) of every branch;
// group 0 also owns the LO-leakage term.  Each CTA writes one row of partials
// (K complex), only at the indices of its group.
template <int B, int TG, int V>
__global__ void __launch_bounds__(256) adj_gh_kernel(AdjArgs a, int T, int Bp, int Bq, int K)
{
    constexpr int NA = 4 * B * TG + 2;   // main + conj accumulators (complex) + c
    const int k0 = blockIdx.y * TG;
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.f;

    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    for (int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; j0 < a.n; j0 += stride) {
        float xr[V], xi[V], gr[V + TG - 1], gi[V + TG - 1];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float2 q = make_float2(0.f, 0.f);
            if (j0 + v < a.n) q = __ldg(a.x + j0 + v);
            xr[v] = q.x;
            xi[v] = q.y;
        }
#pragma unroll
        for (int j = 0; j < V + TG - 1; ++j) {
            float2 q = make_float2(0.f, 0.f);
            const int64_t g = j0 + k0 + j;
            if (g < a.n) q = __ldg(a.gy + g);
            gr[j] = q.x;
            gi[j] = q.y;
        }
        if (blockIdx.y == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) {   // gy window starts at j0 for group 0
                acc[NA - 2] += gr[v];
                acc[NA - 1] += gi[v];
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float r = fmaf(xr[v], xr[v], xi[v] * xi[v]);
#pragma unroll
            for (int kk = 0; kk < TG; ++kk) {
                const float c = gr[v + kk], d = gi[v + kk];
                const float ac_ = xr[v] * c, bd = xi[v] * d, ad = xr[v] * d, bc = xi[v] * c;
                const float m_re = ac_ + bd, m_im = ad - bc;   // conj(x) g
                const float c_re = ac_ - bd, c_im = ad + bc;   // x g
                float w = 1.f;
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    float *am = acc + 2 * (b * TG + kk);
                    float *aq = acc + 2 * B * TG + 2 * (b * TG + kk);
                    am[0] = fmaf(w, m_re, am[0]);
                    am[1] = fmaf(w, m_im, am[1]);
                    aq[0] = fmaf(w, c_re, aq[0]);
                    aq[1] = fmaf(w, c_im, aq[1]);
                    w *= r;
                }
            }
        }
    }

    // Fixed-order reduction: warp butterfly, then warps in index order.
    __shared__ float red[8][NA];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        float v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[i] = v;
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NA; ++i) red[warp][i] = acc[i];
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    float2 *row = a.partials + (size_t)blockIdx.x * K;
    for (int i = threadIdx.x; i < NA; i += blockDim.x) {
        float s = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) s += red[w2][i];
        int idx = -1;
        if (i < 2 * B * TG) {
            const int b = (i >> 1) / TG, kk = (i >> 1) % TG;
            if (b < Bp && k0 + kk < T) idx = b * T + k0 + kk;
        } else if (i < 4 * B * TG) {
            const int e = (i - 2 * B * TG) >> 1;
            const int b = e / TG, kk = e % TG;
            if (b < Bq && k0 + kk < T) idx = (Bp + b) * T + k0 + kk;
        } else if (blockIdx.y == 0) {
            idx = (Bp + Bq) * T;
        }
        if (idx >= 0) {
            if (i & 1)
                row[idx].y = s;
            else
                row[idx].x = s;
        }
    }
}

#define DPD_ADJ_GX_CASE(BB, TT)                                                                    \
    case TT: {                                                                                     \
        int occ = 0;                                                                               \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adj_gx_kernel<BB, TT, 4>, 256, 0);     \
        if (occ < 1) occ = 1;                                                                      \
        const int64_t need = (a.n + 1023) / 1024;                                                  \
        int64_t grid = (int64_t)sm_count * occ;                                                    \
        if (grid > need) grid = need;                                                              \
        adj_gx_kernel<BB, TT, 4><<<(unsigned)grid, 256, 0, s>>>(a);                                \
        count_launch();                                                                            \
        return cudaGetLastError();                                                                 \
    }

template <int B, int TG>
cudaError_t launch_adj_gh_tg(const AdjArgs &a, int gx_blocks, int T, int Bp, int Bq, int K,
                             cudaStream_t s)
{
    const int groups = (T + TG - 1) / TG;
    dim3 grid((unsigned)gx_blocks, (unsigned)groups);
    adj_gh_kernel<B, TG, 4><<<grid, 256, 0, s>>>(a, T, Bp, Bq, K);
    count_launch();
    return cudaGetLastError();
}

// gh: choose the tap-group size (1, 2 or 4 taps per group) and the CTA count.
template <int B>
cudaError_t launch_adj_gh(const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K,
                          cudaStream_t s)
{
    const int blocks = L.gh_blocks;   // already clamped by the caller; = rows of partials
    switch (L.tap_group) {
    case 1: return launch_adj_gh_tg<B, 1>(a, blocks, T, Bp, Bq, K, s);
    case 2: return launch_adj_gh_tg<B, 2>(a, blocks, T, Bp, Bq, K, s);
    case 4: return launch_adj_gh_tg<B, 4>(a, blocks, T, Bp, Bq, K, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int B>
cudaError_t launch_adj_gx(const AdjArgs &a, int T, int sm_count, cudaStream_t s)
{
    switch (T) {
        DPD_ADJ_GX_CASE(B, 1)
        DPD_ADJ_GX_CASE(B, 2)
        DPD_ADJ_GX_CASE(B, 3)
        DPD_ADJ_GX_CASE(B, 4)
        DPD_ADJ_GX_CASE(B, 5)
        DPD_ADJ_GX_CASE(B, 6)
        DPD_ADJ_GX_CASE(B, 7)
        DPD_ADJ_GX_CASE(B, 8)
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
    }

}  // namespace dpd
