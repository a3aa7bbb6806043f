// Adjoint instantiations for B = 3 branch pairs (orders up to 5).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(3)
}  // namespace dpd
