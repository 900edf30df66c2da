// Tile kernels with u degree 2 (0: curves), every v degree and variant.
#include "nurbs_kernel.cuh"

namespace nurbs {

template <int Q>
static KernelVariant pick(int v)
{
    switch (v) {
        case 0: return VariantOf<2, Q, false, false, false>::get();
        case 1: return VariantOf<2, Q, true, false, false>::get();
        case 2: return VariantOf<2, Q, true, true, false>::get();
        case 3: return VariantOf<2, Q, true, false, true>::get();
        case 4: return VariantOf<2, Q, true, true, true>::get();
        default: return VariantOf<2, Q, false, false, false, true>::get();
    }
}

KernelVariant variant_p2(int v, int q)
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
