// Internal declarations of libdpd shared by the host API and the kernel
// translation units.  Not part of the public C ABI (include/dpd.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

// Bits of the per-handle device error word.
enum : int {
    kFlagTimeout = 1,   // a barrier wait inside a kernel exceeded its time limit
    kFlagBadWork = 2,   // a work descriptor failed a device-side range check
};

constexpr int kMaxB = 6;       // (P+1)/2 for P <= 11
constexpr int kMaxT = 8;       // M + 1 <= 8
constexpr int kHalo = 8;       // samples of history staged in front of a tile (>= kMaxT - 1, 16-byte multiple)

// Size in floats of the widely-linear coefficient table consumed by the
// forward kernels: for each tap k, four real polynomials in r = |x|^2
// (B coefficients each, lowest order first), then Re c, Im c.
//   P0 = Re(A+C), P1 = -Im(A-C), P2 = Im(A+C), P3 = Re(A-C)
// where A_k(r) = sum_b h_{2b+1,k} r^b and C_k(r) = sum_b hbar_{2b+1,k} r^b, so that
// A_k(r) x + C_k(r) conj(x) = (P0 a + P1 b) + j (P2 a + P3 b) for x = a + j b.
__host__ __device__ constexpr int wl_table_floats(int B, int T) { return 4 * B * T + 2; }

// Forward launch shape.
struct FwdLaunch {
    int V = 4;            // samples per consumer thread (2 or 4)
    int warps = 8;        // consumer warps per CTA (tile = warps * 32 * V samples)
    int stages = 4;       // shared-memory ring depth (bulk-copy pipeline)
    int ctas_per_sm = 0;  // 0: as many as fit
    int use_tma = 1;      // 0: plain global loads (also used for 8-byte aligned buffers)
};

struct FwdArgs {
    const float2 *x;
    float2 *y;
    int64_t n;
    const float *tab;     // device widely-linear table, wl_table_floats(B, T) floats
    int *status;          // device error word
    int vec_store;        // y is 16-byte aligned
};

// Launch the forward filter for max branch count B and T taps (host side;
// defined per B in fwd_b<B>.cu).  Returns the launch error.
template <int B>
cudaError_t launch_fwd(int T, const FwdArgs &a, const FwdLaunch &L, int sm_count, cudaStream_t s);

cudaError_t launch_fwd_any(int B, int T, const FwdArgs &a, const FwdLaunch &L, int sm_count,
                           cudaStream_t s);

// Build the widely-linear table from the stacked coefficient vector h (K complex).
cudaError_t launch_wl_table(const float2 *h, int Bp, int Bq, int T, float *tab, cudaStream_t s);

void count_launch(int n = 1);

}  // namespace dpd
