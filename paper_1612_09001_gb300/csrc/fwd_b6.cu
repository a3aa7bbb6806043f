// Forward-filter instantiations for B = 6 branch pairs (orders up to 11).
#include "dpd_fwd.cuh"
#include "dpd_zc.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(6)
DPD_DEFINE_LAUNCH_ZC(6)
}  // namespace dpd
