// Persistent tile kernel, one instantiation per (u degree, v degree, variant):
// CTAs pull tiles of their degree group from a queue in the workspace.
#pragma once
#include "nurbs_tile.cuh"

namespace nurbs {

template <int P, int Q, bool GRAD, bool KNOTS, bool MSE, bool DER = false>
__global__ void __launch_bounds__(256, 2) tiles_kernel(const __grid_constant__ KParams kp)
{
    // the first tile of each CTA is its own index; later ones come from the queue
    __shared__ int s_t;
    int t = kp.t0 + (int)blockIdx.x;
    while (t < kp.t1) {
        tile_body<P, Q, GRAD, KNOTS, MSE, DER>(kp, t);
        if (threadIdx.x == 0) s_t = kp.t0 + (int)gridDim.x + (int)atomicAdd(kp.queue, 1u);
        __syncthreads();
        t = s_t;
        __syncthreads();
    }
    // the last CTA out rearms the queue for the next launch on this workspace
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned e = atomicAdd(kp.queue + 1, 1u);
        if (e + 1 == gridDim.x) {
            kp.queue[0] = 0u;
            kp.queue[1] = 0u;
            __threadfence();
        }
    }
}

// Host-side hooks of one compiled kernel.
struct KernelVariant {
    cudaError_t (*launch)(const KParams&, int grid, int block, int smem, cudaStream_t);
    cudaError_t (*occupancy)(int* ctas_per_sm, int block, int smem);
    cudaError_t (*set_smem)(int* limit);
};

template <int P, int Q, bool G, bool K, bool M, bool D = false>
struct VariantOf {
    static cudaError_t launch(const KParams& kp, int grid, int block, int smem, cudaStream_t s)
    {
        tiles_kernel<P, Q, G, K, M, D><<<grid, block, smem, s>>>(kp);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(int* n, int block, int smem)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, tiles_kernel<P, Q, G, K, M, D>, block, smem);
    }
    // Raise the kernel's dynamic shared-memory limit to what the device allows next to
    // its static shared memory (the attribute is per function, so it is never lowered).
    static cudaError_t set_smem(int* limit)
    {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tiles_kernel<P, Q, G, K, M, D>);
        if (e != cudaSuccess) return e;
        *limit = optin - (int)fa.sharedSizeBytes;
        return cudaFuncSetAttribute(tiles_kernel<P, Q, G, K, M, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, *limit);
    }
    static KernelVariant get() { return KernelVariant{launch, occupancy, set_smem}; }
};

// variant: 0 forward; 1 / 2 backward from dL/dS without / with knot gradients;
// 3 / 4 the same from an MSE target; 5 forward with tangents and normals.
// tile_variant_p<P>_v<V>(q) is defined in k_tiles.cu compiled with NURBS_P = P,
// NURBS_V = V; tile_variant(p, v, q) (nurbs_api.cu) dispatches over them.
#define NURBS_DECLARE_TILE_P(p)                                                         \
    KernelVariant tile_variant_p##p##_v0(int q); KernelVariant tile_variant_p##p##_v1(int q); \
    KernelVariant tile_variant_p##p##_v2(int q); KernelVariant tile_variant_p##p##_v3(int q); \
    KernelVariant tile_variant_p##p##_v4(int q); KernelVariant tile_variant_p##p##_v5(int q);
NURBS_DECLARE_TILE_P(0)
NURBS_DECLARE_TILE_P(1)
NURBS_DECLARE_TILE_P(2)
NURBS_DECLARE_TILE_P(3)
NURBS_DECLARE_TILE_P(4)
NURBS_DECLARE_TILE_P(5)
#undef NURBS_DECLARE_TILE_P
// Curve kernels (one warp per curve) of degree p, defined in k_curve.cu.
KernelVariant curve_variant(int v, int p);

}  // namespace nurbs
