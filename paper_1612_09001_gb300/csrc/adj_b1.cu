// Adjoint instantiations for B = 1 branch pairs (orders up to 1).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(1)
}  // namespace dpd
