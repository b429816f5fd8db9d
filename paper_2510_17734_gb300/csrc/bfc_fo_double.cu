// Dispatch table of the first-order methods and the matrix-vector product
// for compute type double, ranks 1..12.
#include "bfc_first_order.cuh"

namespace bfc {

const FoOps* fo_ops_double(int r)
{
    switch (r) {
    case 1: return &FoEntry<double, 1>::ops;
    case 2: return &FoEntry<double, 2>::ops;
    case 3: return &FoEntry<double, 3>::ops;
    case 4: return &FoEntry<double, 4>::ops;
    case 5: return &FoEntry<double, 5>::ops;
    case 6: return &FoEntry<double, 6>::ops;
    case 7: return &FoEntry<double, 7>::ops;
    case 8: return &FoEntry<double, 8>::ops;
    case 9: return &FoEntry<double, 9>::ops;
    case 10: return &FoEntry<double, 10>::ops;
    case 11: return &FoEntry<double, 11>::ops;
    case 12: return &FoEntry<double, 12>::ops;
    default: return nullptr;
    }
}

}  // namespace bfc
