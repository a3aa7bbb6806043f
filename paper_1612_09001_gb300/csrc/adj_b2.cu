// Adjoint instantiations for B = 2 branch pairs (orders up to 3).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(2)
}  // namespace dpd
