// The libnurbs tile kernels.
//
// Work decomposition.  A surface item is cut into tiles of consecutive sample
// rows (u) and up to 32*warps sample columns (v).  A curve too long for the curve
// kernels (nurbs_curve.cuh) is mapped onto the v direction (degree-0 u direction
// with a single row), so one code path serves both.  The warps of a tile form
// `nwr` units (row groups) of `nwc`
// column warps; lane b of a warp keeps its column's span and v-basis in
// registers and walks the rows of its unit in order.  Because the samples are
// non-decreasing, the u-span never decreases along that walk, so the lane holds
// a sliding window of P+1 v-contracted homogeneous control rows
//     Qw[r](b) = sum_h Nv_h(b) Pw[s_u - P + r][s_v(b) - Q + h]
// and each point costs (P+1) 4-wide FMAs (the separable form of Eq. 3).
//
// Backward (Eq. 7, Eq. 8, Eq. 9, knot derivative of Sec. 3.2, Alg. 2) with the
// homogeneous adjoint lambda = (g / W, -S.g / W):
//   tau[r](b)   = sum_a Nu_r(a) lambda_ab         (same sliding window, registers)
//   A[i][j]     = sum_b Nv_{j-s_v(b)+Q}(b) tau[i](b)
//                 (rows leaving the window are staged in shared memory, kBatch at a
//                  time, and contracted over all tile columns by the whole unit in
//                  a fixed order: a segmented reduction with no atomics)
//   beta_r(a)   = sum_b Qw[r](b) . lambda_ab       (warp shuffle reduction)
//   Gamma_h(b)  = sum_i tau[i](b) . Pw[i][s_v(b)-Q+h]
// dL/dU and dL/dV follow from beta and Gamma by the reverse-mode knot derivative
// of the basis.  An item that is a single tile keeps its adjoint in shared
// memory and the CTA finishes it alone; otherwise unit partials go to the
// workspace and the last CTA to finish a tile of the item adds them in unit
// order.  Every result is independent of scheduling (bit-identical run to run,
// alone or in any batch with the same tile shape).
#pragma once
#include "nurbs_basis.cuh"
#include "nurbs_tables.h"

namespace nurbs {

enum : unsigned {
    kErrKnots = 1u << 2,
    kErrDomain = 1u << 4,
    kErrOrder = 1u << 5,
};

constexpr int kBatch = 4;       // retired control rows contracted together
constexpr int kJbCap = 256;     // column ranges cached per tile
constexpr int kWinCap = 1024;   // control points staged in shared memory (whole net, else the tile's window)
constexpr int kSmemACap = 40 * 1024;   // bytes of shared adjoint per single-tile item
constexpr int kSmemPerSM = 228 * 1024; // shared memory of one SM (sm_103)

struct KParams {
    const ItemDev* items;
    const TileDev* tiles;
    int t0, t1;              // tile range of this launch (one degree group)
    unsigned int* queue;     // the group's queue pair: next tile, CTAs finished
    WsHeader* hdr;
    unsigned int* counts;
    float* part;
    const float* knots;
    const float4* ctrl;      // (x, y, z, w) per control point
    float4* ctrl_w;          // same memory, written by the fit step (else null)
    const float* params;
    float* pts;              // S output, or null
    const float* gin;        // dL/dS (gsrc 0) or MSE target (gsrc 1)
    float4* grad_ctrl;
    float* grad_knots;
    float* loss_items;
    float4* adam_m;
    float4* adam_v;
    float grad_scale, lr_t, inv_sqrt_bc2, b1, b2, eps, lr;
    int gsrc;
    int fit;
    int step;                // Adam step of the launch (items may override)
    // shared-memory carve-up in bytes (host-computed for the plan's largest tile)
    int R, C;
    int off_misc, off_su, off_u, off_nu, off_sv, off_v, off_nv, off_stage, off_beta, off_duc, off_dvc,
        off_jb, off_win, off_run, off_knots, off_w, off_acc, off_sa, off_dnu;

    int acc_cap;             // bytes available to the final reduction from off_acc
    float* d_du;             // forward with tangents: S_u, S_v, unit normals (each may be null)
    float* d_dv;
    float* d_nrm;
    int c_mc, c_wbytes;      // curve kernels: control-point capacity, shared bytes per warp
    float knot_sigma;        // > 0: knot derivative with the Gaussian-smoothed indicator term
    int grad_homog;          // grad_ctrl receives dL/dPw (homogeneous) instead of dL/d(P, w)
    int win_cap;             // control points staged in shared memory at most (0: none)
};

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// float4 arithmetic on packed FP32 pairs (FFMA2 / FMUL2, sm_100 and later): one
// instruction per two components, each component rounded as the scalar operation.
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c)
{
    const float2 s2 = make_float2(s, s);
    const float2 l = __ffma2_rn(s2, lo2(a), lo2(c));
    const float2 h = __ffma2_rn(s2, hi2(a), hi2(c));
    return make_float4(l.x, l.y, h.x, h.y);
}

// a.b as (a.x b.x + a.z b.z) + (a.y b.y + a.w b.w)
__device__ __forceinline__ float dot4(float4 a, float4 b)
{
    const float2 p = __ffma2_rn(lo2(a), lo2(b), __fmul2_rn(hi2(a), hi2(b)));
    return p.x + p.y;
}

// Homogeneous control point (w x, w y, w z, w) of Sec. 3.1 step 3.
__device__ __forceinline__ float4 homog(float4 c)
{
    return make_float4(c.x * c.w, c.y * c.w, c.z * c.w, c.w);
}

// Approximate reciprocal (one MUFU op; relative error below 2^-22 for normal inputs).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The N basis values of one row / column from its 16-byte aligned table entry.
template <int N>
__device__ __forceinline__ void load_basis(const float* p, float (&v)[N])
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    if constexpr (N > 1) v[1] = a.y;
    if constexpr (N > 2) v[2] = a.z;
    if constexpr (N > 3) v[3] = a.w;
    if constexpr (N > 4) {
        const float4 b = *reinterpret_cast<const float4*>(p + 4);
        v[4] = b.x;
        if constexpr (N > 5) v[5] = b.y;
    }
}

template <bool B> struct BoolTag { static constexpr bool value = B; };
template <int N> struct IntTag { static constexpr int value = N; };

// Barrier over the `nthreads` threads (a multiple of 32) of one unit.
__device__ __forceinline__ void unit_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gmem_src)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Sum of V values across the warp with a halving transpose: after the call,
// v[0] in lane l holds the full sum of value index `reduce_index<V>(l)`.
template <int V>
__device__ __forceinline__ void warp_reduce_multi(float (&v)[V], int lane)
{
    int offset = 16;
#pragma unroll
    for (int width = V; width > 1; width >>= 1) {
        const int half = width >> 1;
        const bool up = (lane & offset) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            float keep = up ? v[k + half] : v[k];
            float send = up ? v[k] : v[k + half];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, offset);
        }
        offset >>= 1;
    }
#pragma unroll
    for (int o = 32 / V / 2; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

template <int V>
__device__ __forceinline__ int reduce_index(int lane)
{
    int idx = 0, offset = 16;
#pragma unroll
    for (int width = V; width > 1; width >>= 1) {
        if (lane & offset) idx += width >> 1;
        offset >>= 1;
    }
    return idx;
}

template <int N> struct Pow2 { static constexpr int v = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32; };

__device__ __forceinline__ int lower_bound_i(const int* a, int n, int key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float* tile_slot(const KParams& kp, const TileDev& tl) { return kp.part + tl.part; }

// Adam bias corrections: the launch's, or this item's own step.
__device__ __forceinline__ void adam_corrections(const KParams& kp, const ItemDev& it, float& lr_t, float& isb2)
{
    lr_t = kp.lr_t;
    isb2 = kp.inv_sqrt_bc2;
    if (kp.fit && it.adam_step > 0 && it.adam_step != kp.step) {
        const float t = (float)it.adam_step;
        lr_t = kp.lr / (1.f - powf(kp.b1, t));
        isb2 = rsqrtf(1.f - powf(kp.b2, t));
    }
}

// Control point idx (Cartesian c) from its homogeneous adjoint a = dL/dPw: the
// gradient (Cartesian, or a itself when grad_homog is set) and, in a fit step, the
// Adam update of the point and its weight from the Cartesian gradient, with the
// moments mm, vv (loaded by the caller).
__device__ __forceinline__ void finish_point(const KParams& kp, long long idx, float4 c, float4 a, float4 mm,
                                             float4 vv, float lr_t, float isb2)
{
    // Pw = (w x, w y, w z, w): dL/dx = w A.x, ..., dL/dw = x A.x + y A.y + z A.z + A.w
    const float4 g = make_float4(c.w * a.x, c.w * a.y, c.w * a.z, fmaf(c.x, a.x, fmaf(c.y, a.y, fmaf(c.z, a.z, a.w))));
    if (kp.grad_ctrl != nullptr) kp.grad_ctrl[idx] = kp.grad_homog ? a : g;
    if (kp.fit) {
        const float ob1 = 1.f - kp.b1, ob2 = 1.f - kp.b2;
        mm.x = fmaf(kp.b1, mm.x, ob1 * g.x); vv.x = fmaf(kp.b2, vv.x, ob2 * g.x * g.x);
        mm.y = fmaf(kp.b1, mm.y, ob1 * g.y); vv.y = fmaf(kp.b2, vv.y, ob2 * g.y * g.y);
        mm.z = fmaf(kp.b1, mm.z, ob1 * g.z); vv.z = fmaf(kp.b2, vv.z, ob2 * g.z * g.z);
        mm.w = fmaf(kp.b1, mm.w, ob1 * g.w); vv.w = fmaf(kp.b2, vv.w, ob2 * g.w * g.w);
        float4 cn;
        cn.x = c.x - lr_t * mm.x / fmaf(sqrtf(vv.x), isb2, kp.eps);
        cn.y = c.y - lr_t * mm.y / fmaf(sqrtf(vv.y), isb2, kp.eps);
        cn.z = c.z - lr_t * mm.z / fmaf(sqrtf(vv.z), isb2, kp.eps);
        cn.w = c.w - lr_t * mm.w / fmaf(sqrtf(vv.w), isb2, kp.eps);
        kp.adam_m[idx] = mm;
        kp.adam_v[idx] = vv;
        kp.ctrl_w[idx] = cn;
    }
}

__device__ __forceinline__ void finish_ctrl(const KParams& kp, const ItemDev& it, int e, float4 a, float lr_t,
                                            float isb2)
{
    const long long idx = it.ctrl + e;
    const float4 c = kp.ctrl[idx];
    float4 mm = f4zero(), vv = f4zero();
    if (kp.fit) { mm = kp.adam_m[idx]; vv = kp.adam_v[idx]; }
    finish_point(kp, idx, c, a, mm, vv, lr_t, isb2);
}

// The only tile of its item, with A kept in shared memory.  The net block (zeroed
// before the tile's rows) holds, for each control row, what its first covering
// unit wrote; the overflow block of unit u (pb rows from its first row) holds its
// share of rows an earlier unit also covers.  s_units[3u..3u+2] = first control
// row, row count and the last control row of the earlier units; columns
// [jlo, jlo+cw) were written.  The overflow rows are added into the net block in
// unit order, then every control point is finished (its Cartesian point read from
// global memory), four per thread per pass with their loads issued first.
// Adds unit u's overflow block into the net block.
__device__ __forceinline__ void merge_overflow_smem(const KParams& kp, const ItemDev& it, int u, int pb,
                                                    const int* s_units, int jlo, int cw)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    const int m1 = it.m1, ncp = it.n1 * m1, bs = blockDim.x;
    float4* sB = reinterpret_cast<float4*>(smem + kp.off_sa);
    const float4* sO = sB + ncp;
    const int ilo = s_units[3 * u], nr = s_units[3 * u + 1], pm = s_units[3 * u + 2];
    const int nov = nr > 0 ? max(0, min(ilo + nr - 1, pm) - ilo + 1) : 0;
    for (int x = threadIdx.x; x < nov * cw; x += bs) {
        const int ii = x / cw, jj = x - ii * cw;
        float4& d = sB[(ilo + ii) * m1 + jlo + jj];
        const float4 v = sO[(u * pb + ii) * m1 + jlo + jj];
        d.x += v.x; d.y += v.y; d.z += v.z; d.w += v.w;
    }
}

// Finishes every control point of the item from the (merged) net block.
__device__ __forceinline__ void finish_ctrl_smem(const KParams& kp, const ItemDev& it)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    if (kp.grad_ctrl == nullptr && !kp.fit) return;
    const int ncp = it.n1 * it.m1, bs = blockDim.x;
    const float4* sB = reinterpret_cast<const float4*>(smem + kp.off_sa);
    float lr_t, isb2;
    adam_corrections(kp, it, lr_t, isb2);
    constexpr int EB = 4;
    for (int e0 = threadIdx.x; e0 < ncp; e0 += EB * bs) {
        float4 a[EB], c[EB], mm[EB], vv[EB];
#pragma unroll
        for (int k = 0; k < EB; ++k) {
            const int e = e0 + k * bs;
            a[k] = c[k] = mm[k] = vv[k] = f4zero();
            if (e >= ncp) continue;
            const long long idx = it.ctrl + e;
            c[k] = kp.ctrl[idx];
            a[k] = sB[e];
            if (kp.fit) { mm[k] = kp.adam_m[idx]; vv[k] = kp.adam_v[idx]; }
        }
#pragma unroll
        for (int k = 0; k < EB; ++k) {
            const int e = e0 + k * bs;
            if (e < ncp) finish_point(kp, it.ctrl + e, c[k], a[k], mm[k], vv[k], lr_t, isb2);
        }
    }
}

__device__ __forceinline__ void final_ctrl_smem(const KParams& kp, const ItemDev& it, int nwr, int pb,
                                                const int* s_units, int jlo, int cw)
{
    if (kp.grad_ctrl == nullptr && !kp.fit) return;
    for (int u = 1; u < nwr; ++u) {
        merge_overflow_smem(kp, it, u, pb, s_units, jlo, cw);
        __syncthreads();
    }
    finish_ctrl_smem(kp, it);
}

// ---------------------------------------------------------------------------
// Final, fixed-order reduction of one item's partials (run by the last CTA to
// finish a tile of the item): loss, knot gradients, control-point gradients
// (homogeneous adjoint -> Cartesian P and w), and the optional Adam update.
// ---------------------------------------------------------------------------
static __device__ __noinline__ void final_reduce(const KParams& kp, int item, bool ctrl_only)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    const ItemDev it = kp.items[item];
    const int tid = threadIdx.x, bs = blockDim.x;
    const TileDev* T = kp.tiles + it.first_tile;

    if (!ctrl_only && kp.loss_items != nullptr && tid == 0) {
        float L = 0.f;
        for (int t = 0; t < it.ntiles; ++t) L += __ldcg(tile_slot(kp, T[t]) + 8);
        kp.loss_items[item] = L;
    }
    if (!ctrl_only && kp.grad_knots != nullptr) {
        if (!it.curve) {
            const int nU = it.n1 + it.p + 1;
            for (int K = tid; K < nU; K += bs) {
                float acc = 0.f;
                for (int t = 0; t < it.ntiles; ++t) {
                    const float* sl = tile_slot(kp, T[t]);
                    const int lo = __ldcg(reinterpret_cast<const int*>(sl) + 0);
                    const int nk = __ldcg(reinterpret_cast<const int*>(sl) + 1);
                    if (K >= lo && K < lo + nk) acc += __ldcg(sl + 12 + (K - lo));
                }
                if (K < it.p + 1 || K > it.n1 - 1) acc = 0.f;
                kp.grad_knots[it.knot_u + K] = acc;
            }
        }
        const int nV = it.m1 + it.q + 1;
        for (int K = tid; K < nV; K += bs) {
            float acc = 0.f;
            for (int t = 0; t < it.ntiles; ++t) {
                const float* sl = tile_slot(kp, T[t]);
                const int lo = __ldcg(reinterpret_cast<const int*>(sl) + 2);
                const int nk = __ldcg(reinterpret_cast<const int*>(sl) + 3);
                if (K >= lo && K < lo + nk) acc += __ldcg(sl + 12 + it.ku_cap + (K - lo));
            }
            if (K < it.q + 1 || K > it.m1 - 1) acc = 0.f;
            kp.grad_knots[it.knot_v + K] = acc;
        }
    }
    if (kp.grad_ctrl == nullptr && !kp.fit) return;

    // Stage every unit's header and partial offset in shared memory (units in
    // tile order, then row-group order; the planner sizes the buffer).
    int* s_units = reinterpret_cast<int*>(smem + kp.off_acc);
    int nunits = 0;
    {
        int u0 = 0;
        for (int t = 0; t < it.ntiles; ++t) {
            const long long base = T[t].part + it.wbase;
            const int nwr = T[t].nwr;
            for (int e = tid; e < nwr * 5; e += bs) {
                const int u = e / 5, k = e - u * 5;
                s_units[(u0 + u) * 8 + k] = __ldcg(reinterpret_cast<const int*>(kp.part + base + (long long)u * it.unit_slot) + k);
            }
            for (int u = tid; u < nwr; u += bs) {
                const long long off = base + (long long)u * it.unit_slot + it.abase;
                s_units[(u0 + u) * 8 + 6] = (int)(off & 0xffffffffLL);
                s_units[(u0 + u) * 8 + 7] = (int)(off >> 32);
            }
            u0 += nwr;
        }
        nunits = u0;
    }
    __syncthreads();
    const int m1 = it.m1, ncp = it.n1 * m1;
    float lr_t, isb2;
    adam_corrections(kp, it, lr_t, isb2);
    auto finish = [&](int e, float4 a) { finish_ctrl(kp, it, e, a, lr_t, isb2); };
    // two control points per pass; the loads of four units for both are issued
    // before any is summed, and the sums run in unit order
    constexpr int UB = 4;
    for (int e0 = tid; e0 < ncp; e0 += 2 * bs) {
        const int e1 = e0 + bs;
        const bool has1 = e1 < ncp;
        const int i0 = e0 / m1, j0 = e0 - i0 * m1;
        const int i1 = e1 / m1, j1 = e1 - i1 * m1;
        float4 a0 = f4zero(), a1 = f4zero();
        for (int ub = 0; ub < nunits; ub += UB) {
            float4 v0[UB], v1[UB];
#pragma unroll
            for (int k = 0; k < UB; ++k) {
                v0[k] = f4zero();
                v1[k] = f4zero();
                const int u = ub + k;
                if (u < nunits) {
                    const int* h = s_units + u * 8;
                    const int ilo = h[0], nr = h[1], jlo = h[2], cw = h[3];
                    const long long off = (long long)(unsigned)h[6] | ((long long)h[7] << 32);
                    const float4* A = reinterpret_cast<const float4*>(kp.part + off);
                    if (h[4] && i0 >= ilo && i0 < ilo + nr && j0 >= jlo && j0 < jlo + cw)
                        v0[k] = __ldcg(A + (i0 - ilo) * m1 + (j0 - jlo));
                    if (h[4] && has1 && i1 >= ilo && i1 < ilo + nr && j1 >= jlo && j1 < jlo + cw)
                        v1[k] = __ldcg(A + (i1 - ilo) * m1 + (j1 - jlo));
                }
            }
#pragma unroll
            for (int k = 0; k < UB; ++k) {
                a0.x += v0[k].x; a0.y += v0[k].y; a0.z += v0[k].z; a0.w += v0[k].w;
                a1.x += v1[k].x; a1.y += v1[k].y; a1.z += v1[k].z; a1.w += v1[k].w;
            }
        }
        finish(e0, a0);
        if (has1) finish(e1, a1);
    }
}

// ---------------------------------------------------------------------------
// One tile.  GRAD = false: forward only (S -> pts).  GRAD = true: recompute the
// forward, form dL/dS (given, or from the target when MSE), and write this tile's
// partials; the last CTA of the item reduces them.  KNOTS adds beta / Gamma and
// the knot partials.
// ---------------------------------------------------------------------------
template <int P, int Q, bool GRAD, bool KNOTS, bool MSE, bool DER = false>
__device__ __forceinline__ void tile_body(const KParams& kp, int t)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    constexpr int PB = P + 1, QB = Q + 1;
    // shared-table strides: basis rows padded to float4 loads, knot windows exact
    constexpr int SU = (PB + 3) & ~3, SV = (QB + 3) & ~3;
    constexpr int KU = 2 * P > 0 ? 2 * P : 1, KV = 2 * Q;
    const TileDev tl = kp.tiles[t];
    const ItemDev it = kp.items[tl.item];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, bs = blockDim.x;

    int* s_flag = reinterpret_cast<int*>(smem + kp.off_misc);          // [0] bad, [1] last
    float* s_red = reinterpret_cast<float*>(smem + kp.off_misc) + 16;  // per-warp loss
    int* s_su = reinterpret_cast<int*>(smem + kp.off_su);
    float* s_u = reinterpret_cast<float*>(smem + kp.off_u);
    float* s_nu = reinterpret_cast<float*>(smem + kp.off_nu);
    int* s_sv = reinterpret_cast<int*>(smem + kp.off_sv);
    float* s_v = reinterpret_cast<float*>(smem + kp.off_v);
    float* s_nv = reinterpret_cast<float*>(smem + kp.off_nv);

    const int n = it.n1 - 1, m = it.m1 - 1;
    const float* __restrict__ U = kp.knots + it.knot_u;
    const float* __restrict__ V = kp.knots + it.knot_v;
    const int nrows = tl.nrows, ncols = tl.ncols;
    const bool empty = nrows <= 0 || ncols <= 0;   // an item without samples: zero gradients

    if (tid == 0) { s_flag[0] = empty ? 1 : 0; s_flag[1] = 0; }

    // tile geometry: units of nwc column warps, each over a group of rows
    const int nwc = tl.nwc, nwr = tl.nwr, rpg = tl.rpg;
    const int wc = warp % nwc, wr = warp / nwc;
    const int ra = wr * rpg, rb = min(nrows, ra + rpg);
    const int wcol0 = wc * 32;
    const int nvw = max(0, min(32, ncols - wcol0));     // valid columns of this warp
    const int uthreads = nwc * 32, ut = wc * 32 + lane; // threads of the unit, index in it
    const int bl = wcol0 + lane;
    const int blc = min(bl, max(ncols - 1, 0));

    const long long prow0 = it.pts + (long long)tl.row0 * it.nv + tl.col0 + wcol0;  // point (row 0, lane 0)
    const float* grow0 = GRAD ? kp.gin + 3 * prow0 : nullptr;
    const bool wrows = !empty && wr < nwr && ra < rb;
    // ---- staging, in two cp.async groups: the knot vectors and this tile's samples (the
    // tables below need only these), then the control net.  The tables are built while
    // the net and the first dL/dS (or target) rows land.
    float* s_knU = reinterpret_cast<float*>(smem + kp.off_knots);
    float* s_knV = s_knU + ((P > 0) ? ((it.n1 + P + 1 + 3) & ~3) : 0);
    const int nU = (P > 0) ? it.n1 + P + 1 : 0, nV = it.m1 + Q + 1;
    if (!empty) {
        for (int k = tid; k < nU; k += bs) cp_async4(s_knU + k, U + k);
        for (int k = tid; k < nV; k += bs) cp_async4(s_knV + k, V + k);
        if constexpr (P > 0)
            for (int r = tid; r < nrows; r += bs) cp_async4(s_u + r, kp.params + it.param_u + tl.row0 + r);
        for (int c = tid; c < ncols; c += bs) cp_async4(s_v + c, kp.params + it.param_v + tl.col0 + c);
    }
    cp_async_commit();
    // the whole control net rides along when it fits (else the tile's window follows
    // later); once landed it is kept as homogeneous points Pw = (w x, w y, w z, w)
    float4* s_win = reinterpret_cast<float4*>(smem + kp.off_win);
    const int ncp = it.n1 * it.m1;
    const bool net_staged = !empty && ncp <= kp.win_cap;
    if (net_staged) {
        const float4* src = kp.ctrl + it.ctrl;
        for (int e = tid; e < ncp; e += bs)
            cp_async16(reinterpret_cast<float*>(s_win + e), reinterpret_cast<const float*>(src + e));
    }
    cp_async_commit();
    // dL/dS (or target) rows come straight from global memory into registers: each step
    // loads the two rows after its own and prefetches the two after those into L2 (a
    // shared-memory ring cost more instructions per row than the loads)
    const bool pf_on = GRAD && wrows && lane < nvw;
    const float* psrc = pf_on ? grow0 + 3 * lane : nullptr;   // tile row 0, this lane's point
    auto load_row = [&](int x, float (&v)[3]) {
        if (pf_on && x < rb) {
            const float* p = psrc + (long long)x * (3 * it.nv);
            v[0] = __ldcs(p); v[1] = __ldcs(p + 1); v[2] = __ldcs(p + 2);
        } else {
            v[0] = v[1] = v[2] = 0.f;
        }
    };
    auto prefetch_row = [&](int x) {
        if (pf_on && x < rb) {
            const float* p = psrc + (long long)x * (3 * it.nv);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        }
    };
    float pf0[3], pf1[3];
    if constexpr (GRAD) {
        load_row(ra, pf0);
        load_row(ra + 1, pf1);
        prefetch_row(ra + 2);
        prefetch_row(ra + 3);
    }
    cp_async_wait<1>();
    __syncthreads();

    // ---- one pass over rows and columns: device checks (knot vectors once per item,
    // samples in the domain and in order) and each sample row's and column's span and
    // basis (Sec. 3.1 steps 1-2); samples outside the domain are clamped to it (and
    // reported), and the clamped values are recomputed where needed
    const float ulo = (P > 0) ? s_knU[P] : 0.f, uhi = (P > 0) ? s_knU[n + 1] : 0.f;
    const float vlo = s_knV[Q], vhi = s_knV[m + 1];
    const int npro_r = empty ? 0 : nrows, npro_c = empty ? 0 : ncols;   // empty tiles skip the tables
    if (GRAD && it.smemA) {   // the shared adjoint block of a single-tile item starts at zero
        float4* sB = reinterpret_cast<float4*>(smem + kp.off_sa);
        for (int e = tid; e < ncp; e += bs) sB[e] = f4zero();
    }
    if (!empty) {
        unsigned e = 0;
        if (tl.tidx == 0) {
            if constexpr (P > 0) {
                for (int k = tid; k < nU - 1; k += bs)
                    if (s_knU[k] > s_knU[k + 1]) e |= kErrKnots;
                if (tid == 0 && !(s_knU[n] < s_knU[n + 1])) e |= kErrKnots;
            }
            for (int k = tid; k < nV - 1; k += bs)
                if (s_knV[k] > s_knV[k + 1]) e |= kErrKnots;
            if (tid == 0 && !(s_knV[m] < s_knV[m + 1])) e |= kErrKnots;
        }
        for (int x = tid; x < npro_r + npro_c; x += bs) {
            if (x < npro_r) {
                const int r = x;
                float N[PB];
                int s = 0;
                float uc = 0.f;
                if constexpr (P > 0) {
                    const float u0 = s_u[r];
                    if (!(u0 >= ulo && u0 <= uhi)) e |= kErrDomain;
                    if (r > 0 && s_u[r - 1] > u0) e |= kErrOrder;
                    uc = fminf(fmaxf(u0, ulo), uhi);
                    s = find_span(n, P, uc, s_knU);
                }
                if constexpr (DER) {
                    float dN[PB];
                    basis_funs_d<P>(s, uc, s_knU, N, dN);
                    float* s_dnu = reinterpret_cast<float*>(smem + kp.off_dnu);
#pragma unroll
                    for (int k = 0; k < PB; ++k) s_dnu[r * SU + k] = dN[k];
                } else {
                    basis_funs<P>(s, uc, s_knU, N);
                }
                s_su[r] = s;
#pragma unroll
                for (int k = 0; k < PB; ++k) s_nu[r * SU + k] = N[k];
            } else {
                const int c = x - npro_r;
                const float v0 = s_v[c];
                if (!(v0 >= vlo && v0 <= vhi)) e |= kErrDomain;
                if (c > 0 && s_v[c - 1] > v0) e |= kErrOrder;
                const float vc = fminf(fmaxf(v0, vlo), vhi);
                float N[QB];
                const int s = find_span(m, Q, vc, s_knV);
                basis_funs<Q>(s, vc, s_knV, N);
                s_sv[c] = s;
#pragma unroll
                for (int k = 0; k < QB; ++k) s_nv[c * SV + k] = N[k];
            }
        }
        if (e) atomicOr(&kp.hdr->error, e);
    }
    __syncthreads();

    // ---- the sliding windows need non-decreasing spans; anything else is refused.
    // Same pass: rows with equal u-span form runs (s_run[r] = end of the run holding
    // r), and for control column jlo_t + jj of the A contraction the sample columns
    // [lo, lo+len) feeding it.  The contraction A[i][j] = sum_b Nv_{j-s_v(b)+Q}(b)
    // tau[i](b) is a fixed sparse matrix: its weights for column jj sit at
    // s_w[s_joff[jj] ...] (every sample feeds Q+1 columns, so ncols*(Q+1) weights).
    int* s_run = reinterpret_cast<int*>(smem + kp.off_run);
    int2* s_jb = reinterpret_cast<int2*>(smem + kp.off_jb);
    int* s_joff = reinterpret_cast<int*>(smem + kp.off_w);
    float* s_w = reinterpret_cast<float*>(smem + kp.off_w) + kJbCap;
    const int jlo_0 = empty ? 0 : s_sv[0] - Q;
    const int cw_0 = empty ? 0 : max(0, s_sv[ncols - 1] - jlo_0 + 1);
    const int njb = GRAD ? min(cw_0, kJbCap) : 0;
    {
        bool badl = false;
        for (int x = tid; x < npro_r + npro_c + njb; x += bs) {
            if (x < npro_r) {
                const int r = x;
                if (r > 0) badl |= s_su[r] < s_su[r - 1];
                int re = r + 1;
                while (re < nrows && s_su[re] == s_su[r]) ++re;
                s_run[r] = re;
            } else if (x < npro_r + npro_c) {
                const int c = x - npro_r;
                if (c > 0) badl |= s_sv[c] < s_sv[c - 1];
            } else {
                const int jj = x - npro_r - npro_c;
                const int lo = lower_bound_i(s_sv, ncols, jlo_0 + jj);
                s_jb[jj] = make_int2(lo, lower_bound_i(s_sv, ncols, jlo_0 + jj + Q + 1) - lo);
            }
        }
        if (badl) { s_flag[0] = 1; atomicOr(&kp.hdr->error, kErrOrder); }
    }
    __syncthreads();
    const bool bad = s_flag[0] != 0;

    const bool uactive = !bad && wr < nwr && ra < rb;   // the warp's unit has work
    const bool cvalid = uactive && lane < nvw;

    float* slot = GRAD ? tile_slot(kp, tl) : nullptr;
    float* uslot = GRAD ? slot + it.wbase + (long long)wr * it.unit_slot : nullptr;

    float lossacc = 0.f;
    const float gsc = it.gscale > 0.f ? it.gscale : kp.grad_scale;   // the item's own dL/dS scale, if set
    float Gam[QB];
#pragma unroll
    for (int h = 0; h < QB; ++h) Gam[h] = 0.f;

    // column range of the A contraction (all units of a tile span the same columns)
    const int jlo_t = bad ? 0 : jlo_0;
    const int cw_t = bad ? 0 : cw_0;
    if constexpr (GRAD) {
        // exclusive prefix of the columns' sample counts (one warp, shuffle scan)
        if (warp == 0 && !bad) {
            int carry = 0;
            for (int base = 0; base < njb; base += 32) {
                const int jj = base + lane;
                const int len = jj < njb ? s_jb[jj].y : 0;
                int incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (jj < njb) s_joff[jj] = carry + incl - len;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
    }
    // otherwise the tile's window of control points, rows [iwl, iwl+rw) x columns
    // [jlo_t, jlo_t+cw_t), when it fits
    const int iwl = (bad || net_staged) ? 0 : s_su[0] - P;
    const int rw_t = bad ? 0 : s_su[nrows - 1] - (s_su[0] - P) + 1;
    const bool win_only = !bad && !net_staged && rw_t * cw_t <= kp.win_cap;
    const bool win = net_staged || win_only;
    const int w_j0 = net_staged ? 0 : jlo_t;        // window column of element 0
    const int w_stride = net_staged ? it.m1 : cw_t;  // window row stride
    if (win_only) {
        const float4* src = kp.ctrl + it.ctrl + (long long)iwl * it.m1 + jlo_t;
        for (int e = tid; e < rw_t * cw_t; e += bs) {
            const int ii = e / cw_t, jj = e - ii * cw_t;
            cp_async16(reinterpret_cast<float*>(s_win + e), reinterpret_cast<const float*>(src + (long long)ii * it.m1 + jj));
        }
        cp_async_commit();
    }
    __syncthreads();
    if constexpr (GRAD) {
        // sample b's basis value h is the weight of column s_v(b) - Q + h
        if (!bad) {
            for (int x = tid; x < ncols * QB; x += bs) {
                const int b = x / QB, h = x - b * QB;
                const int jj = s_sv[b] - Q + h - jlo_t;
                if (jj < njb) s_w[s_joff[jj] + (b - s_jb[jj].x)] = s_nv[b * SV + h];
            }
        }
    }
    if (win_only) {
        cp_async_wait<0>();
    } else if (net_staged) {   // the net's group
        cp_async_wait<0>();
    }
    __syncthreads();
    if (win) {
        const int nwin = net_staged ? ncp : rw_t * cw_t;
        for (int e = tid; e < nwin; e += bs) s_win[e] = homog(s_win[e]);
        __syncthreads();
    }

    if (uactive) {
        const int svb = s_sv[blc];
        const float vb = fminf(fmaxf(s_v[blc], vlo), vhi);
        float Nv[QB];
#pragma unroll
        for (int h = 0; h < QB; ++h) Nv[h] = s_nv[blc * SV + h];
        float dNv[DER ? QB : 1];   // tangents: the column's v-derivatives of its basis
        if constexpr (DER) {
            float nv_[QB];
            basis_funs_d<Q>(svb, vb, s_knV, nv_, dNv);
        }
        const float4* __restrict__ cbase = kp.ctrl + it.ctrl + (svb - Q);  // column of h = 0
        const int m1 = it.m1;

        const float4* wbase = s_win + (svb - Q - w_j0) - iwl * w_stride;   // window element (i, column of h = 0)
        // sum_h c_h Pw[i][column of h] over row i's Q+1 homogeneous control points: the
        // staged window, else global memory (one branch per row, not per point: a
        // per-point select costs the row loop its registers)
        auto contract_row = [&](int i, const float (&c)[QB]) -> float4 {
            float4 acc = f4zero();
            if (win) {
                const float4* wr_ = wbase + i * w_stride;
#pragma unroll
                for (int h = 0; h < QB; ++h) acc = fma4(c[h], wr_[h], acc);
            } else {
                const float4* cr = cbase + i * m1;
#pragma unroll
                for (int h = 0; h < QB; ++h) acc = fma4(c[h], homog(__ldg(cr + h)), acc);
            }
            return acc;
        };
        // Qw = sum_h Nv_h Pw of row i's Q+1 control points
        auto computeQ = [&](int i) -> float4 { return contract_row(i, Nv); };
        // tangents: Qv = sum_h dNv_h Pw of row i's Q+1 control points
        auto computeQv = [&](int i) -> float4 {
            if constexpr (DER) return contract_row(i, dNv);
            return f4zero();
        };

        // Retired control rows (consecutive, from ilo) wait in tbuf until kBatch of
        // them are contracted together over the tile columns by the whole unit.
        float4* tbuf = reinterpret_cast<float4*>(smem + kp.off_stage) + wr * (kBatch * uthreads);
        // single-tile items whose A fits keep it in shared memory (dense rows by control
        // index, one block per unit); others write dense rows from ilo to the unit slot
        // Rows a unit shares with an earlier unit (at most P+1, those up to pm, the last
        // control row of the sample rows before the unit's) go to the unit's overflow
        // block; every other row has a single first writer in the shared net block.
        const bool sa = GRAD && it.smemA;
        const int pm = wr > 0 ? s_su[ra - 1] : -1;
        float4* sA = reinterpret_cast<float4*>(smem + kp.off_sa) + jlo_t;
        float4* sOv = sA + (it.n1 + wr * PB) * it.m1;
        float4* uA = GRAD ? reinterpret_cast<float4*>(uslot + it.abase) : nullptr;
        int nb = 0, nst = 0, ilo = -1;
        // One contraction task: batched row k, control column jj (sample range r2, weights w).
        // Even and odd terms go to two accumulators, added at the end.
        auto contract = [&](int k, int2 r2, const float* w) -> float4 {
            const float4* tb = tbuf + k * uthreads + r2.x;
            float4 a0 = f4zero(), a1 = f4zero();
            int q = 0;
            for (; q + 3 < r2.y; q += 4) {
                a0 = fma4(w[q], tb[q], a0);
                a1 = fma4(w[q + 1], tb[q + 1], a1);
                a0 = fma4(w[q + 2], tb[q + 2], a0);
                a1 = fma4(w[q + 3], tb[q + 3], a1);
            }
            if (q + 1 < r2.y) {
                a0 = fma4(w[q], tb[q], a0);
                a1 = fma4(w[q + 1], tb[q + 1], a1);
                q += 2;
            }
            if (q < r2.y) a0 = fma4(w[q], tb[q], a0);
            return make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
        };
        auto put = [&](int k, int jj, float4 acc) {
            const int gi = ilo + nst + k;
            if (!sa) uA[(nst + k) * m1 + jj] = acc;
            else if (gi <= pm) sOv[(gi - ilo) * m1 + jj] = acc;
            else sA[gi * m1 + jj] = acc;
        };
        // When a full batch has a thread per task (cw_t * kBatch <= uthreads), thread ut
        // takes task (ut / cw_t, ut % cw_t), without the general loop.
        auto flush = [&]() {
            unit_barrier(1 + wr, uthreads);
            if (cw_t * kBatch <= uthreads && cw_t <= kJbCap) {
                const int k = ut / cw_t, jj = ut - k * cw_t;
                if (k < nb) put(k, jj, contract(k, s_jb[jj], s_w + s_joff[jj]));
            } else {
                const int tasks = nb * cw_t;
                for (int task = ut; task < tasks; task += uthreads) {
                    const int k = task / cw_t, jj = task - k * cw_t;
                    float4 acc;
                    if (jj < kJbCap) {
                        acc = contract(k, s_jb[jj], s_w + s_joff[jj]);
                    } else {
                        const int j = jlo_t + jj;
                        const int lo = lower_bound_i(s_sv, ncols, j), hi = lower_bound_i(s_sv, ncols, j + Q + 1);
                        const float4* tb = tbuf + k * uthreads;
                        acc = f4zero();
                        for (int b = lo; b < hi; ++b) acc = fma4(s_nv[b * SV + (j - s_sv[b] + Q)], tb[b], acc);
                    }
                    put(k, jj, acc);
                }
            }
            nst += nb;
            nb = 0;
            unit_barrier(1 + wr, uthreads);
        };
        // Row i of the window is complete for this unit (rows retire in increasing,
        // consecutive order; rows skipped by a jump retire with tau = 0).
        auto retire = [&](int i, float4 tv) {
            if constexpr (KNOTS) {
                if (win) {
                    const float4* wr_ = wbase + i * w_stride;
#pragma unroll
                    for (int h = 0; h < QB; ++h) Gam[h] += dot4(tv, wr_[h]);
                } else {
                    const float4* cr = cbase + i * m1;
#pragma unroll
                    for (int h = 0; h < QB; ++h) Gam[h] += dot4(tv, homog(__ldg(cr + h)));
                }
            }
            if (ilo < 0) ilo = i;
            tbuf[nb * uthreads + ut] = tv;
            if (++nb == kBatch) flush();
        };


        float4 Qw[PB];
        float4 tau[PB];
        float4 Qv[DER ? PB : 1];
        int cur = -1;
        // Move the window to u-span s: rows leave in increasing order (GRAD: retire them).
        auto advance = [&](int s) {
            if (cur < 0 || s - cur > P) {
                if constexpr (GRAD) {
                    if (cur >= 0) {
#pragma unroll
                        for (int k = 0; k < PB; ++k) retire(cur - P + k, tau[k]);
                        for (int i = cur + 1; i < s - P; ++i) retire(i, f4zero());
                    }
                }
#pragma unroll
                for (int k = 0; k < PB; ++k) { Qw[k] = computeQ(s - P + k); tau[k] = f4zero(); }
                if constexpr (DER) {
#pragma unroll
                    for (int k = 0; k < PB; ++k) Qv[k] = computeQv(s - P + k);
                }
                cur = s;
            } else {
                while (cur < s) {
                    if constexpr (GRAD) retire(cur - P, tau[0]);
#pragma unroll
                    for (int k = 0; k < P; ++k) { Qw[k] = Qw[k + 1]; tau[k] = tau[k + 1]; }
                    ++cur;
                    Qw[P] = computeQ(cur);
                    tau[P] = f4zero();
                    if constexpr (DER) {
#pragma unroll
                        for (int k = 0; k < P; ++k) Qv[k] = Qv[k + 1];
                        Qv[P] = computeQv(cur);
                    }
                }
            }
        };

        const int rstride = 3 * it.nv;                        // floats between sample rows
        const bool store = cvalid && kp.pts != nullptr;
        const bool full = nvw == 32;   // every lane of the warp holds a valid column
        float* orow = kp.pts != nullptr ? kp.pts + 3 * (prow0 + lane) : nullptr;   // row 0 of this lane
        // derivative outputs share the points' layout: element offset of row 0 of this lane
        const long long doff = 3 * (prow0 + lane);
        float* s_beta_w = reinterpret_cast<float*>(smem + kp.off_beta) + (wc * kp.R) * SU;

        // One or two rows (same u-span) per step: S, dL/dS, lambda, tau and beta.
        // NR = rows in the step; its dL/dS (or target) rows are in pf0 / pf1 on entry.
        auto step = [&](auto nr_tag, int r) {
            constexpr int NR = decltype(nr_tag)::value;
            float Nu[NR][PB];
#pragma unroll
            for (int q = 0; q < NR; ++q) load_basis<PB>(s_nu + (r + q) * SU, Nu[q]);
            // homogeneous point and perspective divide (Sec. 3.1 step 3)
            float Sx[NR], Sy[NR], Sz[NR], inv[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                float4 Sw = f4zero();
#pragma unroll
                for (int k = 0; k < PB; ++k) Sw = fma4(Nu[q][k], Qw[k], Sw);
                inv[q] = rcp_approx(Sw.w);
                Sx[q] = Sw.x * inv[q]; Sy[q] = Sw.y * inv[q]; Sz[q] = Sw.z * inv[q];
            }
            if constexpr (!GRAD) {
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    float* o = orow + (r + q) * rstride;
                    if (store) { o[0] = Sx[q]; o[1] = Sy[q]; o[2] = Sz[q]; }
                }
                if constexpr (DER) {
                    // S_u = (A_u - W_u S) / W with (A_u, W_u) = sum_r dNu_r Qw_r; S_v alike
                    // with the dNv-contracted window; unit normal S_u x S_v / |S_u x S_v|
                    const float* s_dnu = reinterpret_cast<const float*>(smem + kp.off_dnu);
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        float dNu[PB];
                        load_basis<PB>(s_dnu + (r + q) * SU, dNu);
                        float4 Au = f4zero(), Av = f4zero();
#pragma unroll
                        for (int k = 0; k < PB; ++k) {
                            Au = fma4(dNu[k], Qw[k], Au);
                            Av = fma4(Nu[q][k], Qv[k], Av);
                        }
                        const float ux = (Au.x - Au.w * Sx[q]) * inv[q], uy = (Au.y - Au.w * Sy[q]) * inv[q],
                                    uz = (Au.z - Au.w * Sz[q]) * inv[q];
                        const float vx = (Av.x - Av.w * Sx[q]) * inv[q], vy = (Av.y - Av.w * Sy[q]) * inv[q],
                                    vz = (Av.z - Av.w * Sz[q]) * inv[q];
                        if (cvalid) {
                            const long long off = doff + (long long)(r + q) * rstride;
                            if (kp.d_du != nullptr) {
                                float* o = kp.d_du + off;
                                o[0] = ux; o[1] = uy; o[2] = uz;
                            }
                            if (kp.d_dv != nullptr) {
                                float* o = kp.d_dv + off;
                                o[0] = vx; o[1] = vy; o[2] = vz;
                            }
                            if (kp.d_nrm != nullptr) {
                                const float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
                                const float l2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
                                const float il = l2 > 0.f ? rsqrtf(l2) : 0.f;
                                float* o = kp.d_nrm + off;
                                o[0] = nx * il; o[1] = ny * il; o[2] = nz * il;
                            }
                        }
                    }
                }
            } else {
                float gv[NR][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) gv[0][c] = pf0[c];
                if constexpr (NR == 2) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) gv[1][c] = pf1[c];
                    load_row(r + 2, pf0);
                    load_row(r + 3, pf1);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) pf0[c] = pf1[c];
                    load_row(r + 2, pf1);
                }
                prefetch_row(r + 4);
                prefetch_row(r + 5);
                float4 lam[NR];
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    const float* gp = gv[q];
                    float gx, gy, gz;
                    float ginv = inv[q];   // dL/dS = ginv * W * (gx, gy, gz)
                    if constexpr (MSE) {
                        float dx = Sx[q] - gp[0], dy = Sy[q] - gp[1], dz = Sz[q] - gp[2];
                        if (!full) { dx = cvalid ? dx : 0.f; dy = cvalid ? dy : 0.f; dz = cvalid ? dz : 0.f; }
                        lossacc = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, lossacc)));
                        gx = dx; gy = dy; gz = dz;
                        ginv *= gsc;
                    } else if (full) {
                        gx = gp[0]; gy = gp[1]; gz = gp[2];
                    } else {
                        gx = cvalid ? gp[0] : 0.f; gy = cvalid ? gp[1] : 0.f; gz = cvalid ? gp[2] : 0.f;
                    }
                    float* o = orow + (r + q) * rstride;
                    if (store) { o[0] = Sx[q]; o[1] = Sy[q]; o[2] = Sz[q]; }
                    // lambda = dL/dS' for S' = (NR, W): (g / W, -S.g / W)
                    const float gbx = gx * ginv, gby = gy * ginv, gbz = gz * ginv;
                    lam[q] = make_float4(gbx, gby, gbz, -fmaf(Sx[q], gbx, fmaf(Sy[q], gby, Sz[q] * gbz)));
                }
#pragma unroll
                for (int q = 0; q < NR; ++q)
#pragma unroll
                    for (int k = 0; k < PB; ++k) tau[k] = fma4(Nu[q][k], lam[q], tau[k]);
                if constexpr (KNOTS && P > 0) {
                    constexpr int VB = Pow2<NR * PB>::v;
                    static_assert(VB >= NR * PB && VB <= 32, "beta reduction width");
                    float beta[VB];
#pragma unroll
                    for (int v = 0; v < VB; ++v) {
                        const int q = v / PB, k = v - (v / PB) * PB;
                        beta[v] = v < NR * PB ? dot4(Qw[k < PB ? k : 0], lam[q < NR ? q : 0]) : 0.f;
                    }
                    warp_reduce_multi<VB>(beta, lane);
                    const int idx = reduce_index<VB>(lane);
                    if ((lane & (32 / VB - 1)) == 0 && idx < NR * PB) {
                        const int q = idx / PB;
                        s_beta_w[(r + q) * SU + (idx - q * PB)] = beta[0];
                    }
                }
            }
        };
        {
            int r = ra;
            while (r < rb) {
                const int re = min(s_run[r], rb);
                advance(s_su[r]);
                // two-row steps, except where the knot cotangents of two rows (2 (P+1) > 8
                // values) would push the step past its registers
                if constexpr (!(KNOTS && P > 3)) {
                    for (; r + 1 < re; r += 2) step(IntTag<2>{}, r);
                    if (r < re) { step(IntTag<1>{}, r); ++r; }
                } else {
                    for (; r < re; ++r) step(IntTag<1>{}, r);
                }
            }
        }
        if constexpr (GRAD) {
            cp_async_wait<0>();
#pragma unroll
            for (int k = 0; k < PB; ++k) retire(cur - P + k, tau[k]);
            if (nb > 0) flush();
            if (ut == 0) {
                if (sa) {
                    s_flag[32 + 3 * wr] = ilo;
                    s_flag[33 + 3 * wr] = nst;
                    s_flag[34 + 3 * wr] = pm;
                } else {
                    int* uh = reinterpret_cast<int*>(uslot);
                    uh[0] = ilo; uh[1] = nst; uh[2] = jlo_t; uh[3] = cw_t; uh[4] = 1;
                }
            }
            if constexpr (KNOTS) {
                // the column's Gamma of this unit; the knot derivative is linear in it, so
                // the epilogue sums the units first and differentiates once per column
                if (cvalid) {
                    float* gv = reinterpret_cast<float*>(smem + kp.off_dvc) + (wr * (nwc * 32) + bl) * KV;
#pragma unroll
                    for (int h = 0; h < QB; ++h) gv[h] = Gam[h];
                }
            }
        }
    } else if (GRAD && wr < nwr && wc == 0 && lane == 0) {
        if (it.smemA) {
            s_flag[32 + 3 * wr] = 0;
            s_flag[33 + 3 * wr] = 0;
            s_flag[34 + 3 * wr] = -1;
        } else {
            int* uh = reinterpret_cast<int*>(uslot);
            uh[0] = 0; uh[1] = 0; uh[2] = 0; uh[3] = 0; uh[4] = 0;
        }
    }

    if constexpr (GRAD) {
        // tile loss: warp tree, then warps in order
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) lossacc += __shfl_xor_sync(0xffffffffu, lossacc, o);
        if (lane == 0) s_red[warp] = lossacc;
        __syncthreads();
        int* sh = reinterpret_cast<int*>(slot);
        const bool single = it.ntiles == 1;   // this CTA finishes the item itself
        if (tid == 0) {
            float L = 0.f;
            for (int w = 0; w < (bs >> 5); ++w) L += s_red[w];
            slot[8] = L;
            sh[4] = bad ? 0 : 1;
            if (single && kp.loss_items != nullptr) kp.loss_items[tl.item] = L;
        }
        // single-tile items: final knot gradients straight from the gathers below
        // (knots outside the tile's windows and the p+1 end knots get 0)
        if (single && kp.grad_knots != nullptr && (!KNOTS || bad)) {
            if constexpr (P > 0)
                for (int K = tid; K < it.n1 + P + 1; K += bs) kp.grad_knots[it.knot_u + K] = 0.f;
            for (int K = tid; K < it.m1 + Q + 1; K += bs) kp.grad_knots[it.knot_v + K] = 0.f;
        }
        // A single-tile item with its adjoint in shared memory and at most two units
        // merges unit 1's overflow during the knot pass and finishes its control points
        // during the knot sums (neither reads what the other writes).
        const bool ctrl_early = KNOTS && !bad && single && it.smemA && nwr <= 2 &&
                                (kp.grad_ctrl != nullptr || kp.fit);
        if constexpr (KNOTS) {
            if (!bad) {
                const int nwc_valid = (ncols + 31) / 32;
                const int ngv = min(nwr, (nrows + rpg - 1) / rpg);   // row groups that hold rows
                float* s_duc = reinterpret_cast<float*>(smem + kp.off_duc);
                float* s_dvc = reinterpret_cast<float*>(smem + kp.off_dvc);
                const float* s_beta = reinterpret_cast<const float*>(smem + kp.off_beta);
                // Reverse-mode knot derivative of each row's u-basis (beta summed over the
                // column warps in order) and of each column's v-basis (Gamma summed over
                // the row groups in order), in one pass
                for (int x = tid; x < nrows + ncols; x += bs) {
                    if (x < nrows) {
                        if constexpr (P > 0) {
                            const int r = x;
                            float bsum[PB];
#pragma unroll
                            for (int k = 0; k < PB; ++k) bsum[k] = 0.f;
                            for (int w = 0; w < nwc_valid; ++w) {
                                float bw[PB];
                                load_basis<PB>(s_beta + (w * kp.R + r) * SU, bw);
#pragma unroll
                                for (int k = 0; k < PB; ++k) bsum[k] += bw[k];
                            }
                            float dk[2 * P + 1];
                            const float ur = fminf(fmaxf(s_u[r], ulo), uhi);
                            basis_knot_vjp<P>(s_su[r], ur, s_knU, bsum, dk);
                            if (kp.knot_sigma > 0.f) knot_sigma_terms<P>(s_su[r], ur, s_knU, bsum, kp.knot_sigma, dk);
#pragma unroll
                            for (int k = 0; k < 2 * P; ++k) s_duc[r * KU + k] = dk[k];
                        }
                    } else {
                        const int c = x - nrows;
                        float G[QB];
#pragma unroll
                        for (int h = 0; h < QB; ++h) G[h] = 0.f;
                        for (int g = 0; g < ngv; ++g) {
#pragma unroll
                            for (int h = 0; h < QB; ++h) G[h] += s_dvc[(g * (nwc * 32) + c) * KV + h];
                        }
                        float dk[2 * Q + 1];
                        const float vc = fminf(fmaxf(s_v[c], vlo), vhi);
                        basis_knot_vjp<Q>(s_sv[c], vc, s_knV, G, dk);
                        if (kp.knot_sigma > 0.f) knot_sigma_terms<Q>(s_sv[c], vc, s_knV, G, kp.knot_sigma, dk);
#pragma unroll
                        for (int k = 0; k < 2 * Q; ++k) s_dvc[c * KV + k] = dk[k];   // group 0's slot
                    }
                }
                if (ctrl_early && nwr == 2) merge_overflow_smem(kp, it, 1, PB, s_flag + 32, jlo_t, cw_t);
                __syncthreads();
                // Each knot's derivative: the rows (columns) whose span window holds knot k
                // form a contiguous range; eight lanes sum it, lane-strided, then in a
                // fixed tree.  A single-tile item writes every knot of the item (0 at the
                // p+1 end knots and outside the tile's windows); other tiles write their
                // windows to the slot.
                const int ku_lo = (P > 0) ? s_su[0] - P + 1 : 0;
                const int nku = (P > 0) ? s_su[nrows - 1] + P - ku_lo + 1 : 0;
                const int kv_lo = s_sv[0] - Q + 1;
                const int nkv = s_sv[ncols - 1] + Q - kv_lo + 1;
                const int nkU = single ? nU : nku, nkV = single ? nV : nkv;
                const int sub = lane >> 3, sl = lane & 7;
                for (int base = warp * 4; base < nkU + nkV; base += (bs >> 5) * 4) {
                    const int kx = base + sub;
                    float acc = 0.f;
                    bool zero = true;
                    int kk = 0;
                    if (kx < nkU) {
                        kk = single ? kx : ku_lo + kx;
                        if (kk >= ku_lo && kk < ku_lo + nku && (!single || (kk >= P + 1 && kk <= it.n1 - 1))) {
                            zero = false;
                            const int r0 = lower_bound_i(s_su, nrows, kk - P), r1 = lower_bound_i(s_su, nrows, kk + P);
                            for (int r = r0 + sl; r < r1; r += 8) acc += s_duc[r * KU + (kk - (s_su[r] - P + 1))];
                        }
                    } else if (kx < nkU + nkV) {
                        kk = single ? kx - nkU : kv_lo + (kx - nkU);
                        if (kk >= kv_lo && kk < kv_lo + nkv && (!single || (kk >= Q + 1 && kk <= it.m1 - 1))) {
                            zero = false;
                            const int c0 = lower_bound_i(s_sv, ncols, kk - Q), c1 = lower_bound_i(s_sv, ncols, kk + Q);
                            for (int c = c0 + sl; c < c1; c += 8) acc += s_dvc[c * KV + (kk - (s_sv[c] - Q + 1))];
                        }
                    }
#pragma unroll
                    for (int o = 4; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (sl == 0 && kx < nkU + nkV) {
                        const float val = zero ? 0.f : acc;
                        if (kx < nkU) {
                            if (single) kp.grad_knots[it.knot_u + kk] = val;
                            else slot[12 + (kk - ku_lo)] = val;
                        } else {
                            if (single) kp.grad_knots[it.knot_v + kk] = val;
                            else slot[12 + it.ku_cap + (kk - kv_lo)] = val;
                        }
                    }
                }
                if (tid == 0) { sh[0] = ku_lo; sh[1] = nku; sh[2] = kv_lo; sh[3] = nkv; }
                if (ctrl_early) finish_ctrl_smem(kp, it);
            } else if (tid == 0) {
                sh[0] = 0; sh[1] = 0; sh[2] = 0; sh[3] = 0;
            }
        } else if (tid == 0) {
            sh[0] = 0; sh[1] = 0; sh[2] = 0; sh[3] = 0;
        }
        if (single) {
            // the only tile of its item: reduce its own units (shared memory or its slot)
            if (!ctrl_early) {
                __syncthreads();
                if (it.smemA) final_ctrl_smem(kp, it, nwr, PB, s_flag + 32, jlo_t, cw_t);
                else final_reduce(kp, tl.item, true);
            }
        } else {
            // publish the partials (the barrier orders the CTA's writes before thread 0's
            // device-scope fence); the last tile of the item reduces them
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const unsigned prev = atomicAdd(kp.counts + tl.item, 1u);
                s_flag[1] = (prev + 1 == (unsigned)it.ntiles) ? 1 : 0;
            }
            __syncthreads();
            if (s_flag[1]) {
                __threadfence();
                final_reduce(kp, tl.item, false);
                if (tid == 0) kp.counts[tl.item] = 0u;
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();
}

}  // namespace nurbs
