// Forward-filter instantiations for B = 2 branch pairs (orders up to 3).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(2)
DPD_DEFINE_LAUNCH_ZC(2)
}  // namespace dpd
