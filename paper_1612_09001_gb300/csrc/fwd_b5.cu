// Forward-filter instantiations for B = 5 branch pairs (orders up to 9).
#include "dpd_fwd.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_FWD(5)
}  // namespace dpd
