// Dispatch table of the templated hot-path drivers (one entry per compute
// type and rank; defined in the bfc_inst_*.cu translation units).
#pragma once

#include "bfc_internal.h"

namespace bfc {

struct Ops {
    bfc_status (*configure)(Ctx*);
    bfc_status (*sweep)(Ctx*);
    bfc_status (*grad)(Ctx*, double2*, double*);
    bfc_status (*eval)(Ctx*, const int32_t*, const int32_t*, int64_t, double2*, const double2*, double*, int);
    size_t (*record_bytes)(int64_t n, int64_t S);
    size_t (*fallback_bytes)(int64_t S);
};

constexpr int MAX_RANK = 12;

const Ops* ops_float_lo(int r);   // r = 1..5
const Ops* ops_float_hi(int r);   // r = 6..10
const Ops* ops_float_xl(int r);   // r = 11..12
const Ops* ops_double_lo(int r);
const Ops* ops_double_hi(int r);
const Ops* ops_double_xl(int r);

inline const Ops* get_ops(bool fp32, int r)
{
    if (r < 1 || r > MAX_RANK) return nullptr;
    if (fp32) return r <= 5 ? ops_float_lo(r) : (r <= 10 ? ops_float_hi(r) : ops_float_xl(r));
    return r <= 5 ? ops_double_lo(r) : (r <= 10 ? ops_double_hi(r) : ops_double_xl(r));
}

}  // namespace bfc
