// Dispatch table of the first-order methods and the matrix-vector product
// for compute type float, ranks 1..12.
#include "bfc_first_order.cuh"

namespace bfc {

const FoOps* fo_ops_float(int r)
{
    switch (r) {
    case 1: return &FoEntry<float, 1>::ops;
    case 2: return &FoEntry<float, 2>::ops;
    case 3: return &FoEntry<float, 3>::ops;
    case 4: return &FoEntry<float, 4>::ops;
    case 5: return &FoEntry<float, 5>::ops;
    case 6: return &FoEntry<float, 6>::ops;
    case 7: return &FoEntry<float, 7>::ops;
    case 8: return &FoEntry<float, 8>::ops;
    case 9: return &FoEntry<float, 9>::ops;
    case 10: return &FoEntry<float, 10>::ops;
    case 11: return &FoEntry<float, 11>::ops;
    case 12: return &FoEntry<float, 12>::ops;
    default: return nullptr;
    }
}

}  // namespace bfc
