// Adjoint instantiations for B = 6 branch pairs (orders up to 11).
#include "dpd_adj.cuh"

namespace dpd {
DPD_DEFINE_LAUNCH_ADJ(6)
}  // namespace dpd
