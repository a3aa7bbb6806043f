// Host-side entry of the zero-copy forward filter (dpd_zc.cuh).
#pragma once

#include "dpd_internal.h"

namespace dpd {

// y = filter(x) for x, y device-visible addresses of mapped host memory, both
// 16-byte aligned.  param_coef: coefficients from a.host_tab (parameter bank),
// else from a.tab.  Defined per B in fwd_b<B>.cu.
template <int B>
cudaError_t launch_zc(int T, const FwdArgs &a, bool param_coef, cudaStream_t s);

cudaError_t launch_zc_any(int B, int T, const FwdArgs &a, bool param_coef, cudaStream_t s);

}  // namespace dpd
