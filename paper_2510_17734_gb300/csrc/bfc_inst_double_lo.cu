// Instantiation of the hot-path drivers for compute type double, ranks 1..5.
#include "bfc_ops.h"
#include "bfc_path.cuh"

namespace bfc {

template <typename T, int R> static Ops make_ops()
{
    return Ops{&Path<T, R>::configure, &Path<T, R>::sweep, &Path<T, R>::grad, &Path<T, R>::eval,
               &Path<T, R>::record_bytes, &Path<T, R>::fallback_bytes};
}

const Ops* ops_double_lo(int r)
{
    static const Ops tab[] = {make_ops<double, 1>(), make_ops<double, 2>(), make_ops<double, 3>(), make_ops<double, 4>(), make_ops<double, 5>(), };
    return (r >= 1 && r <= 5) ? &tab[r - 1] : nullptr;
}

}  // namespace bfc
