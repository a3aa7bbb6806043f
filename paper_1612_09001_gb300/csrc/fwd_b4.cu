// Forward-filter instantiations for B = 4 branch pairs (orders up to 7).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(4)
DPD_DEFINE_LAUNCH_ZC(4)
}  // namespace dpd
