// The libnurbs tile kernels.
//
// Work decomposition.  A surface item is cut into tiles of consecutive sample
// rows (u) and up to 32*warps sample columns (v).  A curve item is mapped onto
// the v direction (degree-0 u direction with a single row), so one code path
// serves both.  The warps of a tile form `nwr` units (row groups) of `nwc`
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
//                 (rows leaving the window are staged in shared memory, KB at a
//                  time, and contracted over all tile columns by the whole unit in
//                  a fixed order: a segmented reduction with no atomics)
//   beta_r(a)   = sum_b Qw[r](b) . lambda_ab       (warp shuffle reduction)
//   Gamma_h(b)  = sum_i tau[i](b) . Pw[i][s_v(b)-Q+h]
// dL/dU and dL/dV follow from beta and Gamma by the reverse-mode knot derivative
// of the basis.  Unit partials go to the workspace; the last CTA to finish a
// tile of an item adds them in unit order, so every result is independent of
// scheduling (bit-identical run to run, alone or in any batch).
#pragma once
#include "nurbs_basis.cuh"
#include "nurbs_tables.h"

namespace nurbs {

enum : unsigned {
    kErrKnots = 1u << 2,
    kErrDomain = 1u << 4,
    kErrOrder = 1u << 5,
};

constexpr int kMaxBasis = 6;    // (max degree + 1)
constexpr int kMaxKnotWin = 10; // 2 * max degree
constexpr int kRing = 8;        // rows of dL/dS (or target) in flight per warp
constexpr int kBatch = 8;       // retired control rows contracted together
constexpr int kJbCap = 256;     // column ranges cached per tile

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
    float grad_scale, lr_t, inv_sqrt_bc2, b1, b2, eps;
    int gsrc;
    int fit;
    // shared-memory carve-up in bytes (host-computed for the plan's largest tile)
    int R, C;
    int off_misc, off_su, off_u, off_nu, off_sv, off_v, off_nv, off_stage, off_beta, off_duc, off_dvc, off_ring,
        off_jb, off_acc;
    int acc_cap;             // bytes available to the final reduction from off_acc
};

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c)
{
    return make_float4(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y), fmaf(s, a.z, c.z), fmaf(s, a.w, c.w));
}

__device__ __forceinline__ float dot4(float4 a, float4 b)
{
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// Homogeneous control point (w x, w y, w z, w) of Sec. 3.1 step 3.
__device__ __forceinline__ float4 homog(float4 c)
{
    return make_float4(c.x * c.w, c.y * c.w, c.z * c.w, c.w);
}

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

template <int N> struct Pow2 { static constexpr int v = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : 8; };

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

// ---------------------------------------------------------------------------
// Final, fixed-order reduction of one item's partials (run by the last CTA to
// finish a tile of the item): loss, knot gradients, control-point gradients
// (homogeneous adjoint -> Cartesian P and w), and the optional Adam update.
// ---------------------------------------------------------------------------
static __device__ __noinline__ void final_reduce(const KParams& kp, int item)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    const ItemDev it = kp.items[item];
    const int tid = threadIdx.x, bs = blockDim.x;
    const TileDev* T = kp.tiles + it.first_tile;

    if (kp.loss_items != nullptr && tid == 0) {
        float L = 0.f;
        for (int t = 0; t < it.ntiles; ++t) L += __ldcg(tile_slot(kp, T[t]) + 8);
        kp.loss_items[item] = L;
    }
    if (kp.grad_knots != nullptr) {
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

    // Stage every unit's header in shared memory (units in tile order, then row-group order).
    int* s_units = reinterpret_cast<int*>(smem + kp.off_acc);
    int nunits = 0;
    for (int t = 0; t < it.ntiles; ++t) nunits += T[t].nwr;
    const bool staged = nunits * 8 * 4 <= kp.acc_cap;
    if (staged) {
        int u0 = 0;
        for (int t = 0; t < it.ntiles; ++t) {
            const float* sl = tile_slot(kp, T[t]);
            const int nwr = T[t].nwr;
            for (int e = tid; e < nwr * 5; e += bs) {
                const int u = e / 5, k = e - u * 5;
                s_units[(u0 + u) * 8 + k] = __ldcg(reinterpret_cast<const int*>(sl + it.wbase + (long long)u * it.unit_slot) + k);
            }
            if (tid < nwr) s_units[(u0 + tid) * 8 + 5] = t;
            u0 += nwr;
        }
    }
    __syncthreads();
    const int m1 = it.m1;
    for (int e = tid; e < it.n1 * m1; e += bs) {
        const int i = e / m1, j = e - i * m1;
        float4 a = f4zero();
        int u = 0;
        for (int t = 0; t < it.ntiles; ++t) {
            const float* sl = tile_slot(kp, T[t]);
            for (int w = 0; w < T[t].nwr; ++w, ++u) {
                const float* us = sl + it.wbase + (long long)w * it.unit_slot;
                int ilo, nr, jlo, cw, valid;
                if (staged) {
                    const int* h = s_units + u * 8;
                    ilo = h[0]; nr = h[1]; jlo = h[2]; cw = h[3]; valid = h[4];
                } else {
                    const int* h = reinterpret_cast<const int*>(us);
                    ilo = __ldcg(h + 0); nr = __ldcg(h + 1); jlo = __ldcg(h + 2); cw = __ldcg(h + 3); valid = __ldcg(h + 4);
                }
                if (!valid || i < ilo || i >= ilo + nr || j < jlo || j >= jlo + cw) continue;
                const float4 v = __ldcg(reinterpret_cast<const float4*>(us + it.abase) + (long long)(i - ilo) * m1 + (j - jlo));
                a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
            }
        }
        const long long idx = it.ctrl + e;
        const float4 c = kp.ctrl[idx];
        // Pw = (w x, w y, w z, w): dL/dx = w A.x, ..., dL/dw = x A.x + y A.y + z A.z + A.w
        const float4 g = make_float4(c.w * a.x, c.w * a.y, c.w * a.z, fmaf(c.x, a.x, fmaf(c.y, a.y, fmaf(c.z, a.z, a.w))));
        if (kp.grad_ctrl != nullptr) kp.grad_ctrl[idx] = g;
        if (kp.fit) {
            float4 mm = kp.adam_m[idx], vv = kp.adam_v[idx];
            const float ob1 = 1.f - kp.b1, ob2 = 1.f - kp.b2;
            mm.x = fmaf(kp.b1, mm.x, ob1 * g.x); vv.x = fmaf(kp.b2, vv.x, ob2 * g.x * g.x);
            mm.y = fmaf(kp.b1, mm.y, ob1 * g.y); vv.y = fmaf(kp.b2, vv.y, ob2 * g.y * g.y);
            mm.z = fmaf(kp.b1, mm.z, ob1 * g.z); vv.z = fmaf(kp.b2, vv.z, ob2 * g.z * g.z);
            mm.w = fmaf(kp.b1, mm.w, ob1 * g.w); vv.w = fmaf(kp.b2, vv.w, ob2 * g.w * g.w);
            float4 cn;
            cn.x = c.x - kp.lr_t * mm.x / fmaf(sqrtf(vv.x), kp.inv_sqrt_bc2, kp.eps);
            cn.y = c.y - kp.lr_t * mm.y / fmaf(sqrtf(vv.y), kp.inv_sqrt_bc2, kp.eps);
            cn.z = c.z - kp.lr_t * mm.z / fmaf(sqrtf(vv.z), kp.inv_sqrt_bc2, kp.eps);
            cn.w = c.w - kp.lr_t * mm.w / fmaf(sqrtf(vv.w), kp.inv_sqrt_bc2, kp.eps);
            kp.adam_m[idx] = mm;
            kp.adam_v[idx] = vv;
            kp.ctrl_w[idx] = cn;
        }
    }
}

// ---------------------------------------------------------------------------
// One tile.  GRAD = false: forward only (S -> pts).  GRAD = true: recompute the
// forward, form dL/dS (given, or from the MSE target), and write this tile's
// partials; the last CTA of the item reduces them.  KNOTS adds beta / Gamma and
// the knot partials.
// ---------------------------------------------------------------------------
template <int P, int Q, bool GRAD, bool KNOTS>
__device__ __forceinline__ void tile_body(const KParams& kp, int t)
{
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    constexpr int PB = P + 1, QB = Q + 1;
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
    __syncthreads();

    // ---- knot-vector check, once per item
    if (tl.tidx == 0 && !empty) {
        unsigned e = 0;
        if constexpr (P > 0) {
            for (int k = tid; k < it.n1 + P; k += bs)
                if (__ldg(U + k) > __ldg(U + k + 1)) e |= kErrKnots;
            if (tid == 0 && !(__ldg(U + n) < __ldg(U + n + 1))) e |= kErrKnots;
        }
        for (int k = tid; k < it.m1 + Q; k += bs)
            if (__ldg(V + k) > __ldg(V + k + 1)) e |= kErrKnots;
        if (tid == 0 && !(__ldg(V + m) < __ldg(V + m + 1))) e |= kErrKnots;
        if (e) atomicOr(&kp.hdr->error, e);
    }

    // ---- row prologue: span and u-basis per sample row (Sec. 3.1 steps 1-2)
    for (int r = tid; r < nrows; r += bs) {
        float N[PB];
        int s = 0;
        float u0 = 0.f;
        if constexpr (P > 0) {
            const int a = tl.row0 + r;
            u0 = __ldg(kp.params + it.param_u + a);
            unsigned e = 0;
            const float lo = __ldg(U + P), hi = __ldg(U + n + 1);
            if (!(u0 >= lo && u0 <= hi)) { e |= kErrDomain; u0 = fminf(fmaxf(u0, lo), hi); }
            if (r > 0 && __ldg(kp.params + it.param_u + a - 1) > u0) e |= kErrOrder;
            if (e) atomicOr(&kp.hdr->error, e);
            s = find_span(n, P, u0, U);
        }
        basis_funs<P>(s, u0, U, N);
        s_su[r] = s;
        s_u[r] = u0;
#pragma unroll
        for (int k = 0; k < PB; ++k) s_nu[r * kMaxBasis + k] = N[k];
    }
    // ---- column prologue: span and v-basis per sample column
    for (int c = tid; c < ncols; c += bs) {
        float N[QB];
        const int b = tl.col0 + c;
        float v0 = __ldg(kp.params + it.param_v + b);
        unsigned e = 0;
        const float lo = __ldg(V + Q), hi = __ldg(V + m + 1);
        if (!(v0 >= lo && v0 <= hi)) { e |= kErrDomain; v0 = fminf(fmaxf(v0, lo), hi); }
        if (c > 0 && __ldg(kp.params + it.param_v + b - 1) > v0) e |= kErrOrder;
        if (e) atomicOr(&kp.hdr->error, e);
        const int s = find_span(m, Q, v0, V);
        basis_funs<Q>(s, v0, V, N);
        s_sv[c] = s;
        s_v[c] = v0;
#pragma unroll
        for (int k = 0; k < QB; ++k) s_nv[c * kMaxBasis + k] = N[k];
    }
    __syncthreads();
    // ---- the sliding windows need non-decreasing spans; anything else is refused
    {
        bool bad = false;
        for (int r = tid + 1; r < nrows; r += bs) bad |= s_su[r] < s_su[r - 1];
        for (int c = tid + 1; c < ncols; c += bs) bad |= s_sv[c] < s_sv[c - 1];
        if (bad) { s_flag[0] = 1; atomicOr(&kp.hdr->error, kErrOrder); }
    }
    __syncthreads();
    const bool bad = s_flag[0] != 0;

    const int nwc = tl.nwc, nwr = tl.nwr, rpg = tl.rpg;
    const int wc = warp % nwc, wr = warp / nwc;
    const int ra = wr * rpg, rb = min(nrows, ra + rpg);
    const int wcol0 = wc * 32;
    const int nvw = max(0, min(32, ncols - wcol0));     // valid columns of this warp
    const bool uactive = !bad && wr < nwr && ra < rb;   // the warp's unit has work
    const int uthreads = nwc * 32, ut = wc * 32 + lane; // threads of the unit, index in it
    const int bl = wcol0 + lane;
    const bool cvalid = uactive && lane < nvw;
    const int blc = min(bl, ncols - 1);

    float* slot = GRAD ? tile_slot(kp, tl) : nullptr;
    float* uslot = GRAD ? slot + it.wbase + (long long)wr * it.unit_slot : nullptr;

    float lossacc = 0.f;
    float Gam[QB];
#pragma unroll
    for (int h = 0; h < QB; ++h) Gam[h] = 0.f;

    // per-tile table of the sample-column range [lo, hi) feeding each control column
    // jlo_t + jj of the A contraction (all units of a tile span the same columns)
    const int jlo_t = bad ? 0 : s_sv[0] - Q;
    const int cw_t = bad ? 0 : s_sv[ncols - 1] - jlo_t + 1;
    int2* s_jb = reinterpret_cast<int2*>(smem + kp.off_jb);
    if constexpr (GRAD) {
        for (int jj = tid; jj < min(cw_t, kJbCap); jj += bs)
            s_jb[jj] = make_int2(lower_bound_i(s_sv, ncols, jlo_t + jj), lower_bound_i(s_sv, ncols, jlo_t + jj + Q + 1));
        __syncthreads();
    }

    if (uactive) {
        const int svb = s_sv[blc];
        const float vb = s_v[blc];
        float Nv[QB];
#pragma unroll
        for (int h = 0; h < QB; ++h) Nv[h] = s_nv[blc * kMaxBasis + h];
        const float4* __restrict__ cbase = kp.ctrl + it.ctrl + (svb - Q);  // column of h = 0
        const int m1 = it.m1;

        auto computeQ = [&](int i) -> float4 {
            const float4* cr = cbase + i * m1;
            float4 acc = f4zero();
#pragma unroll
            for (int h = 0; h < QB; ++h) {
                const float4 c = __ldg(cr + h);
                const float wn = Nv[h] * c.w;
                acc.x = fmaf(wn, c.x, acc.x);
                acc.y = fmaf(wn, c.y, acc.y);
                acc.z = fmaf(wn, c.z, acc.z);
                acc.w += wn;
            }
            return acc;
        };

        // Retired control rows (consecutive, from ilo) wait in tbuf until kBatch of
        // them are contracted together over the tile columns by the whole unit.
        float4* tbuf = reinterpret_cast<float4*>(smem + kp.off_stage) + wr * (kBatch * uthreads);
        float4* uA = GRAD ? reinterpret_cast<float4*>(uslot + it.abase) : nullptr;
        int nb = 0, nst = 0, ilo = -1;
        auto flush = [&]() {
            unit_barrier(1 + wr, uthreads);
            const int tasks = nb * cw_t;
            for (int task = ut; task < tasks; task += uthreads) {
                const int k = task / cw_t, jj = task - k * cw_t;
                const int j = jlo_t + jj;
                int lo, hi;
                if (jj < kJbCap) { const int2 r2 = s_jb[jj]; lo = r2.x; hi = r2.y; }
                else { lo = lower_bound_i(s_sv, ncols, j); hi = lower_bound_i(s_sv, ncols, j + Q + 1); }
                const float4* tb = tbuf + k * uthreads;
                float4 acc = f4zero();
                for (int b = lo; b < hi; ++b) acc = fma4(s_nv[b * kMaxBasis + (j - s_sv[b] + Q)], tb[b], acc);
                uA[(nst + k) * m1 + jj] = acc;
            }
            nst += nb;
            nb = 0;
            unit_barrier(1 + wr, uthreads);
        };
        // Row i of the window is complete for this unit (rows retire in increasing,
        // consecutive order; rows skipped by a jump retire with tau = 0).
        auto retire = [&](int i, float4 tv) {
            if constexpr (KNOTS) {
                const float4* cr = cbase + i * m1;
#pragma unroll
                for (int h = 0; h < QB; ++h) Gam[h] += dot4(tv, homog(__ldg(cr + h)));
            }
            if (ilo < 0) ilo = i;
            tbuf[nb * uthreads + ut] = tv;
            if (++nb == kBatch) flush();
        };

        // ring of incoming dL/dS (or target) rows for this warp's columns
        float* ring = reinterpret_cast<float*>(smem + kp.off_ring) + warp * (kRing * 96);
        const int nf = 3 * nvw;
        const long long prow0 = it.pts + (long long)tl.row0 * it.nv + tl.col0 + wcol0;  // point index of (ra = 0, lane 0)
        const float* grow0 = GRAD ? kp.gin + 3 * prow0 : nullptr;
        const bool al16 = ((prow0 & 3) == 0) && ((it.nv & 3) == 0) && ((nvw & 3) == 0);
        auto issue = [&](int r) {
            if (r < rb && nf > 0) {
                float* dst = ring + ((r - ra) & (kRing - 1)) * 96;
                const float* src = grow0 + 3LL * r * it.nv;
                if (al16) {
                    if (lane * 4 < nf) cp_async16(dst + lane * 4, src + lane * 4);
                } else {
                    for (int k = lane; k < nf; k += 32) cp_async4(dst + k, src + k);
                }
            }
            cp_async_commit();
        };
        if constexpr (GRAD) {
#pragma unroll
            for (int d = 0; d < kRing - 1; ++d) issue(ra + d);
        }

        float4 Qw[PB];
        float4 tau[PB];
        int cur = -1;
        for (int r = ra; r < rb; ++r) {
            if constexpr (GRAD) issue(r + kRing - 1);
            const int s = s_su[r];
            float Nu[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) Nu[k] = s_nu[r * kMaxBasis + k];
            if (s != cur) {
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
                    cur = s;
                } else {
                    while (cur < s) {
                        if constexpr (GRAD) retire(cur - P, tau[0]);
#pragma unroll
                        for (int k = 0; k < P; ++k) { Qw[k] = Qw[k + 1]; tau[k] = tau[k + 1]; }
                        ++cur;
                        Qw[P] = computeQ(cur);
                        tau[P] = f4zero();
                    }
                }
            }
            // homogeneous point and perspective divide (Sec. 3.1 step 3)
            float4 Sw = f4zero();
#pragma unroll
            for (int k = 0; k < PB; ++k) Sw = fma4(Nu[k], Qw[k], Sw);
            const float inv = __fdividef(1.f, Sw.w);
            const float Sx = Sw.x * inv, Sy = Sw.y * inv, Sz = Sw.z * inv;
            if constexpr (!GRAD) {
                if (cvalid) {
                    float* oo = kp.pts + 3 * (prow0 + lane + (long long)r * it.nv);
                    oo[0] = Sx; oo[1] = Sy; oo[2] = Sz;
                }
            } else {
                cp_async_wait<kRing - 1>();
                __syncwarp();
                const float* gp = ring + ((r - ra) & (kRing - 1)) * 96 + 3 * lane;
                float gx = 0.f, gy = 0.f, gz = 0.f;
                if (cvalid) {
                    if (kp.gsrc == 0) {
                        gx = gp[0]; gy = gp[1]; gz = gp[2];
                    } else {
                        const float dx = Sx - gp[0], dy = Sy - gp[1], dz = Sz - gp[2];
                        lossacc = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, lossacc)));
                        gx = kp.grad_scale * dx; gy = kp.grad_scale * dy; gz = kp.grad_scale * dz;
                    }
                    if (kp.pts != nullptr) {
                        float* oo = kp.pts + 3 * (prow0 + lane + (long long)r * it.nv);
                        oo[0] = Sx; oo[1] = Sy; oo[2] = Sz;
                    }
                }
                __syncwarp();   // the slot is refilled by the next iteration's issue
                // lambda = dL/dS' for S' = (NR, W): (g / W, -S.g / W)
                const float gbx = gx * inv, gby = gy * inv, gbz = gz * inv;
                const float4 lam = make_float4(gbx, gby, gbz, -fmaf(Sx, gbx, fmaf(Sy, gby, Sz * gbz)));
#pragma unroll
                for (int k = 0; k < PB; ++k) tau[k] = fma4(Nu[k], lam, tau[k]);
                if constexpr (KNOTS && P > 0) {
                    constexpr int VB = Pow2<PB>::v;
                    float beta[VB];
#pragma unroll
                    for (int k = 0; k < VB; ++k) beta[k] = k < PB ? dot4(Qw[k < PB ? k : 0], lam) : 0.f;
                    warp_reduce_multi<VB>(beta, lane);
                    const int idx = reduce_index<VB>(lane);
                    if ((lane & (32 / VB - 1)) == 0 && idx < PB)
                        reinterpret_cast<float*>(smem + kp.off_beta)[(wc * kp.R + r) * kMaxBasis + idx] = beta[0];
                }
            }
        }
        if constexpr (GRAD) {
            cp_async_wait<0>();
#pragma unroll
            for (int k = 0; k < PB; ++k) retire(cur - P + k, tau[k]);
            if (nb > 0) flush();
            if (ut == 0) {
                int* uh = reinterpret_cast<int*>(uslot);
                uh[0] = ilo; uh[1] = nst; uh[2] = jlo_t; uh[3] = cw_t; uh[4] = 1;
            }
            if constexpr (KNOTS) {
                if (cvalid) {
                    float dk[2 * Q + 1];
                    basis_knot_vjp<Q>(svb, vb, V, Gam, dk);
                    float* dv = reinterpret_cast<float*>(smem + kp.off_dvc) + (wr * kp.C + bl) * kMaxKnotWin;
#pragma unroll
                    for (int k = 0; k < 2 * Q; ++k) dv[k] = dk[k];
                }
            }
        }
    } else if (GRAD && wr < nwr && wc == 0 && lane == 0) {
        int* uh = reinterpret_cast<int*>(uslot);
        uh[0] = 0; uh[1] = 0; uh[2] = 0; uh[3] = 0; uh[4] = 0;
    }

    if constexpr (GRAD) {
        // tile loss: warp tree, then warps in order
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) lossacc += __shfl_xor_sync(0xffffffffu, lossacc, o);
        if (lane == 0) s_red[warp] = lossacc;
        __syncthreads();
        int* sh = reinterpret_cast<int*>(slot);
        if (tid == 0) {
            float L = 0.f;
            for (int w = 0; w < (bs >> 5); ++w) L += s_red[w];
            slot[8] = L;
            sh[4] = bad ? 0 : 1;
        }
        if constexpr (KNOTS) {
            if (!bad) {
                const int nwc_valid = (ncols + 31) / 32;
                // dL/dU: per row, beta summed over the column warps in order, then the
                // reverse-mode knot derivative of the row's basis
                if constexpr (P > 0) {
                    float* s_beta = reinterpret_cast<float*>(smem + kp.off_beta);
                    float* s_duc = reinterpret_cast<float*>(smem + kp.off_duc);
                    for (int r = tid; r < nrows; r += bs) {
                        float bsum[PB];
#pragma unroll
                        for (int k = 0; k < PB; ++k) bsum[k] = 0.f;
                        for (int w = 0; w < nwc_valid; ++w)
#pragma unroll
                            for (int k = 0; k < PB; ++k) bsum[k] += s_beta[(w * kp.R + r) * kMaxBasis + k];
                        float dk[2 * P + 1];
                        basis_knot_vjp<P>(s_su[r], s_u[r], U, bsum, dk);
#pragma unroll
                        for (int k = 0; k < 2 * P; ++k) s_duc[r * kMaxKnotWin + k] = dk[k];
                    }
                }
                __syncthreads();
                if constexpr (P > 0) {
                    const float* s_duc = reinterpret_cast<const float*>(smem + kp.off_duc);
                    const int ku_lo = s_su[0] - P + 1;
                    const int nku = s_su[nrows - 1] + P - ku_lo + 1;
                    for (int K = tid; K < nku; K += bs) {
                        const int kk = ku_lo + K;
                        float acc = 0.f;
                        for (int r = 0; r < nrows; ++r) {
                            const int o = kk - (s_su[r] - P + 1);
                            if (o >= 0 && o < 2 * P) acc += s_duc[r * kMaxKnotWin + o];
                        }
                        slot[12 + K] = acc;
                    }
                    if (tid == 0) { sh[0] = ku_lo; sh[1] = nku; }
                } else {
                    if (tid == 0) { sh[0] = 0; sh[1] = 0; }
                }
                // dL/dV: per column knot derivative, summed over row groups and columns in order
                const float* s_dvc = reinterpret_cast<const float*>(smem + kp.off_dvc);
                const int kv_lo = s_sv[0] - Q + 1;
                const int nkv = s_sv[ncols - 1] + Q - kv_lo + 1;
                for (int K = tid; K < nkv; K += bs) {
                    const int kk = kv_lo + K;
                    const int clo = lower_bound_i(s_sv, ncols, kk - Q);
                    const int chi = lower_bound_i(s_sv, ncols, kk + Q);
                    float acc = 0.f;
                    for (int g = 0; g < nwr; ++g) {
                        if (g * rpg >= nrows) break;
                        for (int c = clo; c < chi; ++c) {
                            const int o = kk - (s_sv[c] - Q + 1);
                            acc += s_dvc[(g * kp.C + c) * kMaxKnotWin + o];
                        }
                    }
                    slot[12 + it.ku_cap + K] = acc;
                }
                if (tid == 0) { sh[2] = kv_lo; sh[3] = nkv; }
            } else if (tid == 0) {
                sh[0] = 0; sh[1] = 0; sh[2] = 0; sh[3] = 0;
            }
        } else if (tid == 0) {
            sh[0] = 0; sh[1] = 0; sh[2] = 0; sh[3] = 0;
        }
        // publish the partials; the last tile of the item reduces them
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(kp.counts + tl.item, 1u);
            s_flag[1] = (prev + 1 == (unsigned)it.ntiles) ? 1 : 0;
        }
        __syncthreads();
        if (s_flag[1]) {
            __threadfence();
            final_reduce(kp, tl.item);
            if (tid == 0) kp.counts[tl.item] = 0u;
        }
    }
    __syncthreads();
}

}  // namespace nurbs
