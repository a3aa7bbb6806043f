// Adjoint instantiations for B = 4 branch pairs (orders up to 7).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(4)
}  // namespace dpd
