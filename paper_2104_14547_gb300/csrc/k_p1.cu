// Tile kernels with u degree 1 (0: curves), every v degree and variant.
#include "nurbs_kernel.cuh"

namespace nurbs {

template <int Q>
static KernelVariant pick(int v)
{
    if (v == 0) return VariantOf<1, Q, false, false>::get();
    if (v == 1) return VariantOf<1, Q, true, false>::get();
    return VariantOf<1, Q, true, true>::get();
}

KernelVariant variant_p1(int v, int q)
{
    switch (q) {
        case 1: return pick<1>(v);
        case 2: return pick<2>(v);
        case 3: return pick<3>(v);
        case 4: return pick<4>(v);
        default: return pick<5>(v);
    }
}

}  // namespace nurbs
