// Forward-filter instantiations for B = 4 branch pairs (orders up to 7).
#include "dpd_fwd.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(4)
}  // namespace dpd
