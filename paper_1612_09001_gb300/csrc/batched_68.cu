// Batched forward kernel for every supported model (orders up to 11, up to 8 taps).
#include "dpd_batched.cuh"

namespace dpd {
cudaError_t launch_batched_68(const BatchArgs &a, int V, int warps, int stages, int cps, int sm_count,
                              cudaStream_t s)
{
    if (V == 4) return launch_batched_impl<6, 8, 4>(a, warps, stages, cps, sm_count, s);
    if (V == 6) return launch_batched_impl<6, 8, 6>(a, warps, stages, cps, sm_count, s);
    if (V == 8) return launch_batched_impl<6, 8, 8>(a, warps, stages, cps, sm_count, s);
    return cudaErrorInvalidValue;
}
}  // namespace dpd
