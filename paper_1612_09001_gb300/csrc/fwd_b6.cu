// Forward-filter instantiations for B = 6 branch pairs (orders up to 11).
#include "dpd_fwd.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(6)
}  // namespace dpd
