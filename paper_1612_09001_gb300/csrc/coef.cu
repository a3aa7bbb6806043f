// Coefficient preparation: the stacked vector of Sec. 2.2 -> the widely-linear
// per-tap polynomial table the forward kernels read (see dpd_internal.h).
#include "dpd_internal.h"

namespace dpd {

__global__ void wl_table_kernel(const float2 *__restrict__ h, int Bp, int Bq, int T, int B,
                                float *__restrict__ tab)
{
    const int i = threadIdx.x;   // one thread per (tap k, order index m)
    if (i < T * B) {
        const int k = i / B, m = i % B;
        const float2 A = (m < Bp) ? h[m * T + k] : make_float2(0.f, 0.f);          // h_{2m+1,k}
        const float2 C = (m < Bq) ? h[(Bp + m) * T + k] : make_float2(0.f, 0.f);   // hbar_{2m+1,k}
        float *row = tab + 4 * B * k;
        row[0 * B + m] = A.x + C.x;      // Re(A+C)
        row[1 * B + m] = -(A.y - C.y);   // -Im(A-C)
        row[2 * B + m] = A.y + C.y;      // Im(A+C)
        row[3 * B + m] = A.x - C.x;      // Re(A-C)
    }
    if (i == 0) {
        const float2 c = h[(Bp + Bq) * T];
        tab[4 * B * T] = c.x;
        tab[4 * B * T + 1] = c.y;
    }
}

cudaError_t launch_wl_table(const float2 *h, int Bp, int Bq, int T, float *tab, cudaStream_t s)
{
    const int B = Bp > Bq ? Bp : Bq;
    wl_table_kernel<<<1, 64, 0, s>>>(h, Bp, Bq, T, B, tab);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
