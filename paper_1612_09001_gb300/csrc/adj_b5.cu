// Adjoint instantiations for B = 5 branch pairs (orders up to 9).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(5)
}  // namespace dpd
