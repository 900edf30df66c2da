// Chamfer and Hausdorff distances between batched point sets (the paper's
// point-cloud losses of Sec. 4), with their gradients with respect to the first
// set:
//   L_CD = sum_i min_j |P_i - Q_j| + sum_j min_i |P_i - Q_j|
//   L_HD = max_i min_j |P_i - Q_j| + max_j min_i |P_i - Q_j|
//
// Three kernels per call:
//   nn_kernel      both directions: each thread keeps the nearest point of the
//                  other set for two of its points, scanning the other set
//                  through shared-memory tiles.  Squared distances are rounded
//                  operation by operation, ((dx dx + dy dy) + dz dz), and the
//                  first index wins a tie, so the argmin is a fixed function of
//                  the float32 inputs.
//   reduce_kernel  one CTA per pair: sums and maxima in a fixed order, and the
//                  Hausdorff gradient at the two arg-max points.
//   grad_kernel    the Chamfer gradient of every P_i: its own term, then the
//                  terms of the Q_j whose nearest point it is, in j order.
//                  With scratch, the Q points are first bucketed by their
//                  nearest P point: integer counts, a per-pair prefix sum, and
//                  placement, then each bucket is sorted by j, so the sums keep a
//                  fixed order.  Without scratch, each P_i scans the pair's whole
//                  nearest-point map instead.
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nurbs.h"

namespace {

constexpr int kThreads = 256;   // threads per CTA
constexpr int kTile = 1024;     // points of the other set staged per pass

__device__ __forceinline__ float dist2_rn(float4 a, float4 b)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float4 load3(const float* X, long long i)
{
    return make_float4(X[3 * i], X[3 * i + 1], X[3 * i + 2], 0.f);
}

// For the points of A in pair blockIdx.y: index (pair-local) of the nearest point
// of B and the distance to it.  Each thread owns points i and i + kThreads of the
// CTA's 2*kThreads block.
__global__ void __launch_bounds__(kThreads) nn_kernel(const float* __restrict__ A, const int64_t* __restrict__ a_off,
                                                      const float* __restrict__ B, const int64_t* __restrict__ b_off,
                                                      int32_t* __restrict__ nn, float* __restrict__ dist)
{
    __shared__ float4 s_b[kTile];
    const int k = blockIdx.y;
    const long long a0 = a_off[k], na = a_off[k + 1] - a0;
    const long long b0 = b_off[k], nb = b_off[k + 1] - b0;
    const long long base = (long long)blockIdx.x * 2 * kThreads;
    if (base >= na) return;                                   // the whole CTA leaves
    const long long i0 = base + threadIdx.x, i1 = i0 + kThreads;
    const bool v0 = i0 < na, v1 = i1 < na;
    const float4 p0 = v0 ? load3(A, a0 + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 p1 = v1 ? load3(A, a0 + i1) : make_float4(0.f, 0.f, 0.f, 0.f);
    float best0 = __int_as_float(0x7f800000), best1 = best0;
    int arg0 = -1, arg1 = -1;
    for (long long t0 = 0; t0 < nb; t0 += kTile) {
        const int nt = (int)min((long long)kTile, nb - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt; e += kThreads) s_b[e] = load3(B, b0 + t0 + e);
        __syncthreads();
        for (int e = 0; e < nt; ++e) {
            const float4 q = s_b[e];
            const float d0 = dist2_rn(p0, q), d1 = dist2_rn(p1, q);
            if (d0 < best0) { best0 = d0; arg0 = (int)(t0 + e); }
            if (d1 < best1) { best1 = d1; arg1 = (int)(t0 + e); }
        }
    }
    if (v0) { nn[a0 + i0] = arg0; dist[a0 + i0] = arg0 >= 0 ? sqrtf(best0) : 0.f; }
    if (v1) { nn[a0 + i1] = arg1; dist[a0 + i1] = arg1 >= 0 ? sqrtf(best1) : 0.f; }
}

// Fixed-order CTA reductions of one pair: sums, and maxima with the first index.
__device__ void block_sum_max(const float* __restrict__ d, long long n, float& sum, float& mx, long long& arg)
{
    __shared__ float s_sum[kThreads], s_max[kThreads];
    __shared__ long long s_arg[kThreads];
    float ls = 0.f, lm = -1.f;
    long long la = -1;
    for (long long i = threadIdx.x; i < n; i += kThreads) {
        const float v = d[i];
        ls += v;
        if (v > lm) { lm = v; la = i; }
    }
    s_sum[threadIdx.x] = ls;
    s_max[threadIdx.x] = lm;
    s_arg[threadIdx.x] = la;
    __syncthreads();
    for (int w = kThreads / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w) {
            const int o = threadIdx.x + w;
            s_sum[threadIdx.x] += s_sum[o];
            const bool take = s_max[o] > s_max[threadIdx.x] ||
                              (s_max[o] == s_max[threadIdx.x] && s_arg[o] >= 0 &&
                               (s_arg[threadIdx.x] < 0 || s_arg[o] < s_arg[threadIdx.x]));
            if (take) { s_max[threadIdx.x] = s_max[o]; s_arg[threadIdx.x] = s_arg[o]; }
        }
        __syncthreads();
    }
    sum = s_sum[0];
    mx = s_max[0];
    arg = s_arg[0];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) reduce_kernel(const float* __restrict__ P, const int64_t* __restrict__ p_off,
                                                          const float* __restrict__ Q, const int64_t* __restrict__ q_off,
                                                          const int32_t* __restrict__ nn_p, const float* __restrict__ d_p,
                                                          const int32_t* __restrict__ nn_q, const float* __restrict__ d_q,
                                                          float* cd, float* hd, float* grad_hd)
{
    const int k = blockIdx.x;
    const long long p0 = p_off[k], np = p_off[k + 1] - p0, q0 = q_off[k], nq = q_off[k + 1] - q0;
    const bool empty = np == 0 || nq == 0;
    float sp = 0.f, mp = 0.f, sq = 0.f, mq = 0.f;
    long long ip = -1, jq = -1;
    if (!empty) {
        block_sum_max(d_p + p0, np, sp, mp, ip);
        block_sum_max(d_q + q0, nq, sq, mq, jq);
    }
    if (threadIdx.x == 0) {
        if (cd != nullptr) cd[k] = empty ? 0.f : sp + sq;
        if (hd != nullptr) hd[k] = empty ? 0.f : mp + mq;
    }
    if (grad_hd == nullptr) return;
    for (long long i = threadIdx.x; i < 3 * np; i += kThreads) grad_hd[3 * p0 + i] = 0.f;
    __syncthreads();
    if (threadIdx.x == 0 && !empty) {
        // the point farthest from Q, then the point nearest to the Q point farthest from P
        if (ip >= 0 && mp > 0.f) {
            const long long j = q0 + nn_p[p0 + ip];
            for (int c = 0; c < 3; ++c) grad_hd[3 * (p0 + ip) + c] += (P[3 * (p0 + ip) + c] - Q[3 * j + c]) / mp;
        }
        if (jq >= 0 && mq > 0.f) {
            const long long i = p0 + nn_q[q0 + jq];
            for (int c = 0; c < 3; ++c) grad_hd[3 * i + c] += (P[3 * i + c] - Q[3 * (q0 + jq) + c]) / mq;
        }
    }
}

__global__ void __launch_bounds__(kThreads) grad_kernel(const float* __restrict__ P, const int64_t* __restrict__ p_off,
                                                        const float* __restrict__ Q, const int64_t* __restrict__ q_off,
                                                        const int32_t* __restrict__ nn_p, const float* __restrict__ d_p,
                                                        const int32_t* __restrict__ nn_q, const float* __restrict__ d_q,
                                                        float* __restrict__ grad_cd)
{
    __shared__ int32_t s_nn[kTile];
    const int k = blockIdx.y;
    const long long p0 = p_off[k], np = p_off[k + 1] - p0, q0 = q_off[k], nq = q_off[k + 1] - q0;
    const long long base = (long long)blockIdx.x * kThreads;
    if (base >= np) return;
    const long long i = base + threadIdx.x;
    const bool act = i < np;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act && nq > 0) {
        pi = load3(P, p0 + i);
        const float d = d_p[p0 + i];
        if (d > 0.f) {
            const float4 q = load3(Q, q0 + nn_p[p0 + i]);
            gx = (pi.x - q.x) / d; gy = (pi.y - q.y) / d; gz = (pi.z - q.z) / d;
        }
    }
    for (long long t0 = 0; t0 < nq; t0 += kTile) {
        const int nt = (int)min((long long)kTile, nq - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt; e += kThreads) s_nn[e] = nn_q[q0 + t0 + e];
        __syncthreads();
        if (act) {
            for (int e = 0; e < nt; ++e) {
                if (s_nn[e] == (int)i) {
                    const long long j = q0 + t0 + e;
                    const float d = d_q[j];
                    if (d > 0.f) {
                        const float4 q = load3(Q, j);
                        gx += (pi.x - q.x) / d; gy += (pi.y - q.y) / d; gz += (pi.z - q.z) / d;
                    }
                }
            }
        }
    }
    if (act) {
        grad_cd[3 * (p0 + i)] = gx;
        grad_cd[3 * (p0 + i) + 1] = gy;
        grad_cd[3 * (p0 + i) + 2] = gz;
    }
}


// ---- bucketing of the Q points by their nearest P point (scratch path)
__global__ void __launch_bounds__(kThreads) count_kernel(const int64_t* __restrict__ p_off,
                                                         const int64_t* __restrict__ q_off,
                                                         const int32_t* __restrict__ nn_q, int32_t* __restrict__ cnt)
{
    const int k = blockIdx.y;
    const long long p0 = p_off[k], q0 = q_off[k], nq = q_off[k + 1] - q0;
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < nq; j += (long long)gridDim.x * kThreads) {
        const int i = nn_q[q0 + j];
        if (i >= 0) atomicAdd(cnt + p0 + i, 1);   // integer counts: the result does not depend on order
    }
}

// Per pair: start[i] = q0 + exclusive prefix of the counts; cursor[i] = start[i].
__global__ void __launch_bounds__(kThreads) scan_kernel(const int64_t* __restrict__ p_off,
                                                        const int64_t* __restrict__ q_off,
                                                        int32_t* __restrict__ start, int32_t* __restrict__ cursor)
{
    __shared__ int32_t s_v[kThreads];
    const int k = blockIdx.x;
    const long long p0 = p_off[k], np = p_off[k + 1] - p0;
    int32_t carry = (int32_t)q_off[k];
    for (long long c0 = 0; c0 < np; c0 += kThreads) {
        const long long i = c0 + threadIdx.x;
        const int32_t v = i < np ? cursor[p0 + i] : 0;   // the counts
        s_v[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kThreads; o <<= 1) {          // inclusive Hillis-Steele scan
            const int32_t add = threadIdx.x >= o ? s_v[threadIdx.x - o] : 0;
            __syncthreads();
            s_v[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < np) {
            const int32_t st = carry + s_v[threadIdx.x] - v;
            start[p0 + i] = st;
            cursor[p0 + i] = st;
        }
        carry += s_v[kThreads - 1];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) place_kernel(const int64_t* __restrict__ p_off,
                                                         const int64_t* __restrict__ q_off,
                                                         const int32_t* __restrict__ nn_q, int32_t* __restrict__ cursor,
                                                         int32_t* __restrict__ list)
{
    const int k = blockIdx.y;
    const long long p0 = p_off[k], q0 = q_off[k], nq = q_off[k + 1] - q0;
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < nq; j += (long long)gridDim.x * kThreads) {
        const int i = nn_q[q0 + j];
        if (i >= 0) list[atomicAdd(cursor + p0 + i, 1)] = (int32_t)j;   // order fixed later by sorting
    }
}

// Chamfer gradient from the buckets: P_i's own term, then its bucket in j order.
__global__ void __launch_bounds__(kThreads) grad_bucket_kernel(const float* __restrict__ P,
                                                               const int64_t* __restrict__ p_off,
                                                               const float* __restrict__ Q,
                                                               const int64_t* __restrict__ q_off,
                                                               const int32_t* __restrict__ nn_p,
                                                               const float* __restrict__ d_p,
                                                               const float* __restrict__ d_q,
                                                               const int32_t* __restrict__ start,
                                                               const int32_t* __restrict__ end, int32_t* list,
                                                               float* __restrict__ grad_cd)
{
    const int k = blockIdx.y;
    const long long p0 = p_off[k], np = p_off[k + 1] - p0, q0 = q_off[k], nq = q_off[k + 1] - q0;
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (i >= np) return;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (nq > 0) {
        const float4 pi = load3(P, p0 + i);
        const float d = d_p[p0 + i];
        if (d > 0.f) {
            const float4 q = load3(Q, q0 + nn_p[p0 + i]);
            gx = (pi.x - q.x) / d; gy = (pi.y - q.y) / d; gz = (pi.z - q.z) / d;
        }
        const int a = start[p0 + i], b = end[p0 + i];
        for (int x = a + 1; x < b; ++x) {                 // insertion sort of the bucket by j
            const int v = list[x];
            int y = x - 1;
            while (y >= a && list[y] > v) { list[y + 1] = list[y]; --y; }
            list[y + 1] = v;
        }
        for (int x = a; x < b; ++x) {
            const long long j = q0 + list[x];
            const float dj = d_q[j];
            if (dj > 0.f) {
                const float4 q = load3(Q, j);
                gx += (pi.x - q.x) / dj; gy += (pi.y - q.y) / dj; gz += (pi.z - q.z) / dj;
            }
        }
    }
    grad_cd[3 * (p0 + i)] = gx;
    grad_cd[3 * (p0 + i) + 1] = gy;
    grad_cd[3 * (p0 + i) + 2] = gz;
}

}  // namespace

extern "C" nurbs_status nurbs_chamfer(int32_t count, const int64_t* p_off, const int64_t* q_off, int32_t max_p,
                                      int32_t max_q, const float* P, const float* Q, int32_t* nn_p, float* dist_p,
                                      int32_t* nn_q, float* dist_q, float* cd, float* hd, float* grad_cd,
                                      float* grad_hd, int32_t* scratch, int64_t total_p, int64_t total_q,
                                      nurbs_stream_t stream)
{
    nvtxRangePushA("nurbs_chamfer");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop_;
    if (count < 0 || max_p < 0 || max_q < 0) return NURBS_ERR_ARG;
    if (count == 0) return NURBS_OK;
    if (count > 65535) return NURBS_ERR_SIZE;
    if (p_off == nullptr || q_off == nullptr || nn_p == nullptr || dist_p == nullptr || nn_q == nullptr ||
        dist_q == nullptr)
        return NURBS_ERR_ARG;
    if ((max_p > 0 && P == nullptr) || (max_q > 0 && Q == nullptr)) return NURBS_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const unsigned bp = (unsigned)((max_p + 2 * kThreads - 1) / (2 * kThreads));
    const unsigned bq = (unsigned)((max_q + 2 * kThreads - 1) / (2 * kThreads));
    if (bp > 0) nn_kernel<<<dim3(bp, count), kThreads, 0, s>>>(P, p_off, Q, q_off, nn_p, dist_p);
    if (bq > 0) nn_kernel<<<dim3(bq, count), kThreads, 0, s>>>(Q, q_off, P, p_off, nn_q, dist_q);
    if (cd != nullptr || hd != nullptr || grad_hd != nullptr)
        reduce_kernel<<<count, kThreads, 0, s>>>(P, p_off, Q, q_off, nn_p, dist_p, nn_q, dist_q, cd, hd, grad_hd);
    const unsigned gp = (unsigned)((max_p + kThreads - 1) / kThreads);
    if (grad_cd != nullptr && gp > 0) {
        if (scratch != nullptr && total_p > 0) {
            int32_t* start = scratch;
            int32_t* cursor = scratch + total_p;
            int32_t* list = scratch + 2 * total_p;
            const cudaError_t e0 = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)total_p, s);
            if (e0 != cudaSuccess) return NURBS_ERR_CUDA;
            const unsigned gq = (unsigned)min((max_q + kThreads - 1) / kThreads, 64);
            if (gq > 0) count_kernel<<<dim3(gq, count), kThreads, 0, s>>>(p_off, q_off, nn_q, cursor);
            scan_kernel<<<count, kThreads, 0, s>>>(p_off, q_off, start, cursor);
            if (gq > 0) place_kernel<<<dim3(gq, count), kThreads, 0, s>>>(p_off, q_off, nn_q, cursor, list);
            grad_bucket_kernel<<<dim3(gp, count), kThreads, 0, s>>>(P, p_off, Q, q_off, nn_p, dist_p, dist_q, start,
                                                                    cursor, list, grad_cd);
        } else {
            grad_kernel<<<dim3(gp, count), kThreads, 0, s>>>(P, p_off, Q, q_off, nn_p, dist_p, nn_q, dist_q, grad_cd);
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NURBS_OK : NURBS_ERR_CUDA;
}
