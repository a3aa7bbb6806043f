// Batched forward kernel for streams with orders up to 9 (B <= 5) and up to 7 taps.
#include "dpd_batched.cuh"

namespace dpd {
cudaError_t launch_batched_57(const BatchArgs &a, int V, int warps, int stages, int cps, int sm_count,
                              cudaStream_t s)
{
    if (V == 4) return launch_batched_impl<5, 7, 4>(a, warps, stages, cps, sm_count, s);
    if (V == 6) return launch_batched_impl<5, 7, 6>(a, warps, stages, cps, sm_count, s);
    if (V == 8) return launch_batched_impl<5, 7, 8>(a, warps, stages, cps, sm_count, s);
    return cudaErrorInvalidValue;
}
}  // namespace dpd
