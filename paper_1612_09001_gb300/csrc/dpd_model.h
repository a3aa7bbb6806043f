// Validation of a model (P, Q, M) shared by the C entry points.  The paper's
// order sets hold odd orders only (Sec. 2.1), so an even order is a model this
// library does not build (DPD_ERR_UNSUPPORTED), as are orders above 11 and
// more than 8 taps; negative values, and a model with neither branch, are
// invalid arguments.  Host code only; depends on nothing but the public header.
#pragma once

#include "../../include/dpd.h"

namespace dpd {

constexpr int kModelMaxOrder = 11;   // B = (P + 1) / 2 <= 6
constexpr int kModelMaxTaps = 8;     // T = M + 1 <= 8

inline dpd_status order_status(int o)
{
    if (o < 0) return DPD_ERR_INVALID_ARGUMENT;
    if (o == 0) return DPD_OK;
    if (o % 2 == 0 || o > kModelMaxOrder) return DPD_ERR_UNSUPPORTED;
    return DPD_OK;
}

inline dpd_status model_status(int P, int Q, int M)
{
    if (P < 0 || Q < 0 || M < 0 || (P == 0 && Q == 0)) return DPD_ERR_INVALID_ARGUMENT;
    dpd_status st = order_status(P);
    if (st == DPD_OK) st = order_status(Q);
    if (st == DPD_OK && M + 1 > kModelMaxTaps) st = DPD_ERR_UNSUPPORTED;
    return st;
}

}  // namespace dpd
