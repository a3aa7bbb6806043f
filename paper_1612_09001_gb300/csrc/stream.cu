// Stream continuation for dpd_apply_stream.  A block of a continuous stream
// differs from an isolated block only in its first M outputs: the taps of
// Eq. 1 reach back into the previous block.  The forward kernels run on the
// block with zero history; this kernel then recomputes those outputs with the
// saved history and saves the new one.
#include "dpd_handle.h"

namespace dpd {

__global__ void stream_head_kernel(const float *__restrict__ tab, int B, int T, const float2 *__restrict__ x,
                                   int64_t n, float2 *__restrict__ hist, float2 *__restrict__ y)
{
    const int j = threadIdx.x;   // output index; T - 1 <= kHalo - 1 < 32
    const int64_t heads = n < (int64_t)(T - 1) ? n : (int64_t)(T - 1);
    float2 out = make_float2(tab[4 * B * T], tab[4 * B * T + 1]);   // c
    if (j < heads) {
        for (int k = 0; k < T; ++k) {
            const int g = j - k;   // sample n - k, negative = previous block
            const float2 v = g >= 0 ? x[g] : hist[kHalo + g];
            const float r = v.x * v.x + v.y * v.y;
            const float4 *cf = reinterpret_cast<const float4 *>(tab) + k * B;   // {P0, P2, P1, P3} per order
            float4 p = cf[B - 1];
            for (int m = B - 2; m >= 0; --m) {
                const float4 c = cf[m];
                p.x = fmaf(p.x, r, c.x);
                p.y = fmaf(p.y, r, c.y);
                p.z = fmaf(p.z, r, c.z);
                p.w = fmaf(p.w, r, c.w);
            }
            out.x = fmaf(p.x, v.x, out.x);
            out.x = fmaf(p.z, v.y, out.x);
            out.y = fmaf(p.y, v.x, out.y);
            out.y = fmaf(p.w, v.y, out.y);
        }
    }
    // new history: position n + i of (hist ++ x), i < kHalo
    float2 nh = make_float2(0.f, 0.f);
    if (j < kHalo) {
        const int64_t src = (int64_t)j + n;
        nh = src < kHalo ? hist[src] : x[src - kHalo];
    }
    __syncwarp();   // every read of the old history precedes the writes
    if (j < heads) y[j] = out;
    if (j < kHalo) hist[j] = nh;
}

cudaError_t launch_stream_head(const float *tab, int B, int T, const float2 *x, int64_t n, float2 *hist,
                               float2 *y, cudaStream_t s)
{
    stream_head_kernel<<<1, 32, 0, s>>>(tab, B, T, x, n, hist, y);
    count_launch();
    return cudaGetLastError();
}

// Squared-error loss of direct learning and its gradient in one pass: each
// block sums |e|^2 (FP32 products, FP64 sums) over a grid-stride range and
// combines its threads with a fixed shared-memory tree; one more block adds the
// block sums in order.
__global__ void sq_error_kernel(const float2 *__restrict__ y, const float2 *__restrict__ x, int64_t n, float2 g,
                                double scale, double *__restrict__ part, float2 *__restrict__ gy)
{
    const float s2 = (float)(2.0 * scale);
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = x[i], b = y[i];
        const float er = b.x - (g.x * a.x - g.y * a.y), ei = b.y - (g.x * a.y + g.y * a.x);
        acc += (double)(er * er + ei * ei);
        if (gy) gy[i] = make_float2(s2 * er, s2 * ei);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sq_error_sum_kernel(const double *__restrict__ part, int blocks, double scale, float *loss)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < blocks; b += 256) acc += part[b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = (float)(scale * red[0]);
}

cudaError_t launch_sq_error(const float2 *y, const float2 *x, int64_t n, float2 g, double scale, double *part,
                            float *loss, float2 *gy, cudaStream_t s)
{
    sq_error_kernel<<<kLossBlocks, 256, 0, s>>>(y, x, n, g, scale, part, gy);
    count_launch();
    sq_error_sum_kernel<<<1, 256, 0, s>>>(part, kLossBlocks, scale, loss);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
