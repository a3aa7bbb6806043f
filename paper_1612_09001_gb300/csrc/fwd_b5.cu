// Forward-filter instantiations for B = 5 branch pairs (orders up to 9).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(5)
DPD_DEFINE_LAUNCH_ZC(5)
}  // namespace dpd
