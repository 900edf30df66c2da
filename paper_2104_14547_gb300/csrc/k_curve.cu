// Curve kernels (one warp per curve), every degree and variant.
#include "nurbs_curve.cuh"
#include "nurbs_kernel.cuh"

namespace nurbs {

template <int P, bool G, bool K, bool M, bool D = false>
struct CurveVariantOf {
    static cudaError_t launch(const KParams& kp, int grid, int block, int smem, cudaStream_t s)
    {
        curves_kernel<P, G, K, M, D><<<grid, block, smem, s>>>(kp);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(int* n, int block, int smem)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, curves_kernel<P, G, K, M, D>, block, smem);
    }
    static cudaError_t set_smem(int* limit)
    {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, curves_kernel<P, G, K, M, D>);
        if (e != cudaSuccess) return e;
        *limit = optin - (int)fa.sharedSizeBytes;
        return cudaFuncSetAttribute(curves_kernel<P, G, K, M, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, *limit);
    }
    static KernelVariant get() { return KernelVariant{launch, occupancy, set_smem}; }
};

template <int P>
static KernelVariant pick(int v)
{
    switch (v) {
        case 0: return CurveVariantOf<P, false, false, false>::get();
        case 1: return CurveVariantOf<P, true, false, false>::get();
        case 2: return CurveVariantOf<P, true, true, false>::get();
        case 3: return CurveVariantOf<P, true, false, true>::get();
        case 4: return CurveVariantOf<P, true, true, true>::get();
        default: return CurveVariantOf<P, false, false, false, true>::get();
    }
}

KernelVariant curve_variant(int v, int p)
{
    switch (p) {
        case 1: return pick<1>(v);
        case 2: return pick<2>(v);
        case 3: return pick<3>(v);
        case 4: return pick<4>(v);
        default: return pick<5>(v);
    }
}

}  // namespace nurbs
