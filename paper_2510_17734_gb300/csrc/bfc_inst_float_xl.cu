// Instantiation of the hot-path drivers for compute type float, ranks 11..12.
#include "bfc_ops.h"
#include "bfc_path.cuh"

namespace bfc {

template <typename T, int R> static Ops make_ops()
{
    return Ops{&Path<T, R>::configure, &Path<T, R>::sweep, &Path<T, R>::grad, &Path<T, R>::eval,
               &Path<T, R>::record_bytes, &Path<T, R>::fallback_bytes};
}

const Ops* ops_float_xl(int r)
{
    static const Ops tab[] = {make_ops<float, 11>(), make_ops<float, 12>()};
    return (r >= 11 && r <= 12) ? &tab[r - 11] : nullptr;
}

}  // namespace bfc
