// Forward-filter instantiations for B = 1 branch pairs (orders up to 1).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(1)
DPD_DEFINE_LAUNCH_ZC(1)
}  // namespace dpd
