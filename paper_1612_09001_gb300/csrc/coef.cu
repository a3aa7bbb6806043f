// Coefficient preparation: the stacked vector of Sec. 2.2 -> the per-tap
// polynomial tables read by the forward kernels (widely-linear form, see
// dpd_internal.h) and by the adjoint input-gradient kernel (see dpd_adj.cuh).
// Also the FP64 finalisation of the coefficient gradient.
#include "dpd_internal.h"

namespace dpd {

// Coefficient k of the stacked vector as FP32 (FP64 sources are rounded to
// nearest, as the FP32 copy of an FP64 estimate is).
__device__ __forceinline__ float2 coef_f32(const float2 *h, int i) { return h[i]; }
__device__ __forceinline__ float2 coef_f32(const double2 *h, int i)
{
    return make_float2((float)h[i].x, (float)h[i].y);
}

// blockIdx.x selects a problem of a batch: coefficients hin + x * hstride,
// table tab + x * tstride (0 for a single table).
template <typename H>
__global__ void wl_table_kernel(const H *__restrict__ hin, int Bp, int Bq, int T, int B, float *__restrict__ tab,
                                float *__restrict__ adj, int hstride = 0, int tstride = 0)
{
    hin += (size_t)blockIdx.x * hstride;
    tab += (size_t)blockIdx.x * tstride;
    auto h = [hin](int i) { return coef_f32(hin, i); };
    const int i = threadIdx.x;   // one thread per (tap k, order index m)
    if (i < T * B) {
        const int k = i / B, m = i % B;
        const float2 A = (m < Bp) ? h(m * T + k) : make_float2(0.f, 0.f);          // h_{2m+1,k}
        const float2 C = (m < Bq) ? h((Bp + m) * T + k) : make_float2(0.f, 0.f);   // hbar_{2m+1,k}
        tab[wl_index(B, k, m, 0)] = A.x + C.x;      // P0 = Re(A+C)
        tab[wl_index(B, k, m, 1)] = -(A.y - C.y);   // P1 = -Im(A-C)
        tab[wl_index(B, k, m, 2)] = A.y + C.y;      // P2 = Im(A+C)
        tab[wl_index(B, k, m, 3)] = A.x - C.x;      // P3 = Re(A-C)
        if (adj) {
            // Per tap: for each power m the quadruple {Q0, Q3, Q1, Q2} of the
            // bracket conj(E) g + H conj(g) = {Q0 c + Q1 d, Q2 c + Q3 d}
            // (g = c + j d), then for each m < B-1 the quadruple {S0, S3, S1, S2}
            // of conj(G) g + F conj(g): the pairs {Q0, Q3}, {Q1, Q2} multiply
            // {c, d} and {d, c} in packed f32x2 FMAs.
            const int per_tap = 4 * B + 4 * (B - 1);
            float *q = adj + per_tap * k;
            // E_m = (m+1) h_m, H_m = (m+1) hbar_m  (coefficients of r^m)
            const float s = (float)(m + 1);
            const float Er = s * A.x, Ei = s * A.y, Hr = s * C.x, Hi = s * C.y;
            q[4 * m + 0] = Er + Hr;   // Q0
            q[4 * m + 1] = Er - Hr;   // Q3
            q[4 * m + 2] = Ei + Hi;   // Q1
            q[4 * m + 3] = Hi - Ei;   // Q2
            if (m < B - 1) {
                // F_m = (m+1) h_{m+1}, G_m = (m+1) hbar_{m+1}
                const float2 A1 = (m + 1 < Bp) ? h((m + 1) * T + k) : make_float2(0.f, 0.f);
                const float2 C1 = (m + 1 < Bq) ? h((Bp + m + 1) * T + k) : make_float2(0.f, 0.f);
                const float Fr = s * A1.x, Fi = s * A1.y, Gr = s * C1.x, Gi = s * C1.y;
                float *r = q + 4 * B;
                r[4 * m + 0] = Gr + Fr;   // S0
                r[4 * m + 1] = Gr - Fr;   // S3
                r[4 * m + 2] = Gi + Fi;   // S1
                r[4 * m + 3] = Fi - Gi;   // S2
            }
        }
    }
    if (i == 0) {
        const float2 c = h((Bp + Bq) * T);
        tab[4 * B * T] = c.x;
        tab[4 * B * T + 1] = c.y;
    }
}

cudaError_t launch_wl_table(const float2 *h, int Bp, int Bq, int T, float *tab, float *adj_tab,
                            cudaStream_t s)
{
    const int B = Bp > Bq ? Bp : Bq;
    wl_table_kernel<float2><<<1, 64, 0, s>>>(h, Bp, Bq, T, B, tab, adj_tab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_wl_table_f64(const double2 *h, int Bp, int Bq, int T, float *tab, cudaStream_t s)
{
    const int B = Bp > Bq ? Bp : Bq;
    wl_table_kernel<double2><<<1, 64, 0, s>>>(h, Bp, Bq, T, B, tab, nullptr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_wl_table_f64_many(const double2 *h, int count, int hstride, int Bp, int Bq, int T, float *tab,
                                     int tstride, cudaStream_t s)
{
    const int B = Bp > Bq ? Bp : Bq;
    wl_table_kernel<double2><<<count, 64, 0, s>>>(h, Bp, Bq, T, B, tab, nullptr, hstride, tstride);
    count_launch();
    return cudaGetLastError();
}

// One block per coefficient: thread t sums rows t, t + 256, ... in order, then a
// fixed shared-memory tree combines the 256 sums (deterministic, FP64).
// blockIdx.y selects a problem of a batch (its rows and outputs follow the
// previous problem's).
__global__ void adj_finalize_kernel(const float2 *__restrict__ partials, int rows, int K,
                                    float2 *__restrict__ gh, double2 *__restrict__ gh64)
{
    const int i = blockIdx.x, t = threadIdx.x;
    partials += (size_t)blockIdx.y * rows * K;
    if (gh) gh += (size_t)blockIdx.y * K;
    if (gh64) gh64 += (size_t)blockIdx.y * K;
    double re = 0.0, im = 0.0;
    for (int r = t; r < rows; r += 256) {
        const float2 v = partials[(size_t)r * K + i];
        re += v.x;
        im += v.y;
    }
    __shared__ double sre[256], sim[256];
    sre[t] = re;
    sim[t] = im;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            sre[t] += sre[t + w];
            sim[t] += sim[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (gh) gh[i] = make_float2((float)sre[0], (float)sim[0]);
        if (gh64) gh64[i] = make_double2(sre[0], sim[0]);
    }
}

cudaError_t launch_adj_finalize(const float2 *partials, int rows, int K, float2 *gh, cudaStream_t s)
{
    adj_finalize_kernel<<<K, 256, 0, s>>>(partials, rows, K, gh, nullptr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adj_finalize64(const float2 *partials, int rows, int K, double2 *out, cudaStream_t s)
{
    adj_finalize_kernel<<<K, 256, 0, s>>>(partials, rows, K, nullptr, out);
    count_launch();
    return cudaGetLastError();
}

// One partial row per problem (the batched refinement): the FP64 sum is the
// row itself, widened; one thread per coefficient instead of a 256-thread
// reduction per coefficient.
__global__ void adj_widen_kernel(const float2 *__restrict__ partials, int64_t n, double2 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 v = partials[i];
        out[i] = make_double2(v.x, v.y);
    }
}

cudaError_t launch_adj_finalize64_many(const float2 *partials, int rows, int K, int count, double2 *out,
                                       cudaStream_t s)
{
    if (rows == 1) {
        const int64_t n = (int64_t)K * count;
        adj_widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partials, n, out);
        count_launch();
        return cudaGetLastError();
    }
    adj_finalize_kernel<<<dim3((unsigned)K, (unsigned)count), 256, 0, s>>>(partials, rows, K, nullptr, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
