// Forward-filter instantiations for B = 3 branch pairs (orders up to 5).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(3)
DPD_DEFINE_LAUNCH_ZC(3)
}  // namespace dpd
