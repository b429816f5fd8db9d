// Dispatch interface of the first-order methods (ADAM, Alg. 3/4; ADF,
// Alg. 5) and the butterfly matrix-vector product (Eq. (butterfly-mat-vec));
// the kernels and drivers are in bfc_first_order.cuh, instantiated per
// compute type in bfc_fo_float.cu / bfc_fo_double.cu.
#pragma once

#include "bfc_internal.h"
#include "bfc_ops.h"

namespace bfc {

// Alg. 3 constants of one outer iteration t: inv1 = 1 / (1 - beta1^t),
// inv2 = 1 / (1 - beta2^t).
struct AdamHyper {
    double alpha, beta1, beta2, sigma, inv1, inv2;
};

struct FoOps {
    // u = X(S) V for nvec vectors: Vd, Ud device n x nvec complex128; y0, y1
    // scratch of 2^{L+1} nvec r compute-type complex values each
    bfc_status (*matvec)(Ctx*, int nvec, const double2* Vd, double2* Ud, void* y0, void* y1);
    // one outer iteration of Alg. 4 with moments M, V (packed like the factors)
    bfc_status (*adam_iter)(Ctx*, const AdamHyper&, double2* M, double2* V);
    // one iteration of Alg. 5
    bfc_status (*adf_iter)(Ctx*);
};

const FoOps* fo_ops_float(int r);
const FoOps* fo_ops_double(int r);

inline const FoOps* get_fo_ops(bool fp32, int r)
{
    if (r < 1 || r > MAX_RANK) return nullptr;
    return fp32 ? fo_ops_float(r) : fo_ops_double(r);
}

}  // namespace bfc
