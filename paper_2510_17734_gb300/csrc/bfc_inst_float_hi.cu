// Instantiation of the hot-path drivers for compute type float, ranks 6..10.
#include "bfc_ops.h"
#include "bfc_path.cuh"

namespace bfc {

template <typename T, int R> static Ops make_ops()
{
    return Ops{&Path<T, R>::configure, &Path<T, R>::sweep, &Path<T, R>::grad, &Path<T, R>::eval,
               &Path<T, R>::record_bytes, &Path<T, R>::fallback_bytes};
}

const Ops* ops_float_hi(int r)
{
    static const Ops tab[] = {make_ops<float, 6>(), make_ops<float, 7>(), make_ops<float, 8>(), make_ops<float, 9>(), make_ops<float, 10>(), };
    return (r >= 6 && r <= 10) ? &tab[r - 6] : nullptr;
}

}  // namespace bfc
