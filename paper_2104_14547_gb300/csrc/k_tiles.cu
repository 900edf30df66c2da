// Tile kernels of one u degree and one variant, for every v degree.  The build
// compiles this file once per (NURBS_P, NURBS_V) pair, 0 <= P <= 5 (0: curves too
// long for the curve kernels) and 0 <= V <= 5, so the 180 instantiations spread
// over 36 translation units that compile in parallel.  Without both macros the
// file defines nothing.
#include "nurbs_kernel.cuh"

#if defined(NURBS_P) && defined(NURBS_V)
namespace nurbs {

template <int Q>
static KernelVariant pick()
{
    constexpr int P = NURBS_P, V = NURBS_V;
    if constexpr (V == 0) return VariantOf<P, Q, false, false, false>::get();
    else if constexpr (V == 1) return VariantOf<P, Q, true, false, false>::get();
    else if constexpr (V == 2) return VariantOf<P, Q, true, true, false>::get();
    else if constexpr (V == 3) return VariantOf<P, Q, true, false, true>::get();
    else if constexpr (V == 4) return VariantOf<P, Q, true, true, true>::get();
    else return VariantOf<P, Q, false, false, false, true>::get();
}

#define NURBS_TILE_FN_(p, v) tile_variant_p##p##_v##v
#define NURBS_TILE_FN(p, v) NURBS_TILE_FN_(p, v)

KernelVariant NURBS_TILE_FN(NURBS_P, NURBS_V)(int q)
{
    switch (q) {
        case 1: return pick<1>();
        case 2: return pick<2>();
        case 3: return pick<3>();
        case 4: return pick<4>();
        default: return pick<5>();
    }
}

}  // namespace nurbs
#endif
