// The libnurbs tile kernels.
//
// Work decomposition.  A surface item is cut into tiles of consecutive sample
// rows (u) and up to 32*warps sample columns (v).  A curve item is mapped onto
// the v direction (degree-0 u direction with a single row), so one code path
// serves both.  Inside a tile each warp owns 32 consecutive columns and one row
// group; lane b keeps its column's span and v-basis in registers and walks the
// rows of its group in order.  Because the samples are non-decreasing, the
// u-span is non-decreasing along that walk, so the lane holds a sliding window
// of P+1 v-contracted homogeneous control rows
//     Qw[r](b) = sum_h Nv_h(b) Pw[s_u - P + r][s_v(b) - Q + h]
// and each point costs (P+1) 4-wide FMAs (the separable form of Eq. 3).
//
// Backward (Eq. 7, Eq. 8, Eq. 9, knot derivative of Sec. 3.2, Alg. 2) with the
// homogeneous adjoint lambda = (g / W, -S.g / W):
//   tau[r](b)   = sum_a Nu_r(a) lambda_ab      (same sliding window, registers)
//   A[i][j]     = sum_b Nv_{j-s_v(b)+Q}(b) tau[i](b)   (v-contraction when row i
//                 leaves the window; staged through shared memory per warp)
//   beta_r(a)   = sum_b Qw[r](b) . lambda_ab    (warp shuffle reduction)
//   Gamma_h(b)  = sum_i tau[i](b) . Pw[i][s_v(b)-Q+h]
// dL/dU and dL/dV follow from beta and Gamma by the reverse-mode knot derivative
// of the basis.  Every sum is taken in a fixed order: per-warp partials go to the
// workspace and the last CTA to finish an item adds them tile by tile, warp by
// warp, so results do not depend on scheduling.
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
    int off_misc, off_su, off_u, off_nu, off_sv, off_v, off_nv, off_stage, off_beta, off_duc, off_dvc, off_acc;
    int acc_cap;             // float4 entries available to the final reduction
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
        // u knots (surfaces only)
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

    float4* acc = reinterpret_cast<float4*>(smem + kp.off_acc);
    const int m1 = it.m1;
    const int ch = max(1, kp.acc_cap / m1);
    for (int i0 = 0; i0 < it.n1; i0 += ch) {
        const int nr = min(ch, it.n1 - i0);
        for (int e = tid; e < nr * m1; e += bs) acc[e] = f4zero();
        __syncthreads();
        for (int t = 0; t < it.ntiles; ++t) {
            const TileDev tl = T[t];
            const float* sl = tile_slot(kp, tl);
            const int nws = tl.nwc * tl.nwr;
            for (int w = 0; w < nws; ++w) {
                const float* ws = sl + it.wbase + (long long)w * it.warp_slot;
                const int* wi = reinterpret_cast<const int*>(ws);
                const int nst = __ldcg(wi + 0), jlo = __ldcg(wi + 1), cw = __ldcg(wi + 2), valid = __ldcg(wi + 3);
                if (valid && nst > 0) {
                    const float4* A = reinterpret_cast<const float4*>(ws + it.abase);
                    for (int e = tid; e < nst * cw; e += bs) {
                        const int k = e / cw, jj = e - k * cw;
                        const int i = __ldcg(wi + 4 + k);
                        if (i >= i0 && i < i0 + nr) {
                            float4 a = __ldcg(A + (long long)k * m1 + jj);
                            float4& d = acc[(i - i0) * m1 + jlo + jj];
                            d.x += a.x; d.y += a.y; d.z += a.z; d.w += a.w;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int e = tid; e < nr * m1; e += bs) {
            const long long idx = it.ctrl + (long long)(i0 + e / m1) * m1 + (e % m1);
            const float4 c = kp.ctrl[idx];
            const float4 a = acc[e];
            // Pw = (w x, w y, w z, w): dL/dx = w A.x, ..., dL/dw = x A.x + y A.y + z A.z + A.w
            float4 g = make_float4(c.w * a.x, c.w * a.y, c.w * a.z, fmaf(c.x, a.x, fmaf(c.y, a.y, fmaf(c.z, a.z, a.w))));
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
        __syncthreads();
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

    int* s_flag = reinterpret_cast<int*>(smem + kp.off_misc);     // [0] bad, [1] last
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
    const int nvw = min(32, ncols - wcol0);            // valid columns of this warp
    const bool wactive = !bad && wr < nwr && ra < rb && nvw > 0;
    const int bl = wcol0 + lane;
    const bool cvalid = wactive && lane < nvw;
    const int blc = min(bl, ncols - 1);

    float* slot = GRAD ? tile_slot(kp, tl) : nullptr;
    float* wslot = GRAD ? slot + it.wbase + (long long)warp * it.warp_slot : nullptr;

    float lossacc = 0.f;
    float Gam[QB];
#pragma unroll
    for (int h = 0; h < QB; ++h) Gam[h] = 0.f;

    if (wactive) {
        const int svb = s_sv[blc];
        const float vb = s_v[blc];
        float Nv[QB];
#pragma unroll
        for (int h = 0; h < QB; ++h) Nv[h] = s_nv[blc * kMaxBasis + h];
        const float4* __restrict__ cbase = kp.ctrl + it.ctrl + (svb - Q);  // column of h = 0
        const long long m1 = it.m1;

        auto computeQ = [&](int i) -> float4 {
            const float4* cr = cbase + (long long)i * m1;
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

        // warp's v-knot column range and, for lane-as-column jj = lane, its sample range
        const int jlo_w = s_sv[wcol0] - Q;
        const int cw_w = s_sv[wcol0 + nvw - 1] - jlo_w + 1;
        int bj_lo = 0, bj_hi = 0;
        if (GRAD && lane < cw_w) {
            const int j = jlo_w + lane;
            bj_lo = lower_bound_i(s_sv + wcol0, nvw, j);
            bj_hi = lower_bound_i(s_sv + wcol0, nvw, j + Q + 1);
        }
        float4* stage = reinterpret_cast<float4*>(smem + kp.off_stage) + warp * 32;
        int nst = 0;
        int* wil = GRAD ? reinterpret_cast<int*>(wslot) + 4 : nullptr;
        float4* wA = GRAD ? reinterpret_cast<float4*>(wslot + it.abase) : nullptr;

        // Row i of the window is complete for this warp: fold it into A (and Gamma).
        auto retire = [&](int i, float4 tv) {
            if constexpr (KNOTS) {
                const float4* cr = cbase + (long long)i * m1;
#pragma unroll
                for (int h = 0; h < QB; ++h) Gam[h] += dot4(tv, homog(__ldg(cr + h)));
            }
            stage[lane] = tv;
            __syncwarp();
            for (int jj = lane; jj < cw_w; jj += 32) {
                const int j = jlo_w + jj;
                int lo = bj_lo, hi = bj_hi;
                if (jj >= 32) {
                    lo = lower_bound_i(s_sv + wcol0, nvw, j);
                    hi = lower_bound_i(s_sv + wcol0, nvw, j + Q + 1);
                }
                float4 acc = f4zero();
                for (int b = lo; b < hi; ++b) {
                    const int h = j - s_sv[wcol0 + b] + Q;
                    acc = fma4(s_nv[(wcol0 + b) * kMaxBasis + h], stage[b], acc);
                }
                wA[(long long)nst * m1 + jj] = acc;
            }
            if (lane == 0) wil[nst] = i;
            ++nst;
            __syncwarp();
        };

        float4 Qw[PB];
        float4 tau[PB];
        int cur = -1;
        for (int r = ra; r < rb; ++r) {
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
            const float inv = 1.f / Sw.w;
            const float Sx = Sw.x * inv, Sy = Sw.y * inv, Sz = Sw.z * inv;
            const long long pidx = it.pts + (long long)(tl.row0 + r) * it.nv + (tl.col0 + bl);
            if constexpr (!GRAD) {
                if (cvalid) {
                    float* o = kp.pts + 3 * pidx;
                    o[0] = Sx; o[1] = Sy; o[2] = Sz;
                }
            } else {
                float gx = 0.f, gy = 0.f, gz = 0.f;
                if (cvalid) {
                    const float* gp = kp.gin + 3 * pidx;
                    if (kp.gsrc == 0) {
                        gx = __ldg(gp + 0); gy = __ldg(gp + 1); gz = __ldg(gp + 2);
                    } else {
                        const float dx = Sx - __ldg(gp + 0), dy = Sy - __ldg(gp + 1), dz = Sz - __ldg(gp + 2);
                        lossacc = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, lossacc)));
                        gx = kp.grad_scale * dx; gy = kp.grad_scale * dy; gz = kp.grad_scale * dz;
                    }
                    if (kp.pts != nullptr) {
                        float* o = kp.pts + 3 * pidx;
                        o[0] = Sx; o[1] = Sy; o[2] = Sz;
                    }
                }
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
#pragma unroll
            for (int k = 0; k < PB; ++k) retire(cur - P + k, tau[k]);
            if (lane == 0) {
                int* wh = reinterpret_cast<int*>(wslot);
                wh[0] = nst; wh[1] = jlo_w; wh[2] = cw_w; wh[3] = 1;
            }
            if constexpr (KNOTS) {
                if (cvalid) {
                    float dk[2 * Q + 1];
                    basis_knot_vjp<Q>(svb, vb, V, Gam, dk);
                    float* dv = reinterpret_cast<float*>(smem + kp.off_dvc) + ((wr * nwc * 32) + bl) * kMaxKnotWin;
#pragma unroll
                    for (int k = 0; k < 2 * Q; ++k) dv[k] = dk[k];
                }
            }
        }
    } else if (GRAD && warp < nwc * nwr && lane == 0) {
        int* wh = reinterpret_cast<int*>(wslot);
        wh[0] = 0; wh[1] = 0; wh[2] = 0; wh[3] = 0;
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
                // dL/dU: per row, beta summed over column warps in order, then the
                // reverse-mode knot derivative of the row's basis
                if constexpr (P > 0) {
                    float* s_beta = reinterpret_cast<float*>(smem + kp.off_beta);
                    float* s_duc = reinterpret_cast<float*>(smem + kp.off_duc);
                    for (int r = tid; r < nrows; r += bs) {
                        float bsum[PB];
#pragma unroll
                        for (int k = 0; k < PB; ++k) bsum[k] = 0.f;
                        for (int w = 0; w < nwc; ++w)
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
                            acc += s_dvc[((g * nwc * 32) + c) * kMaxKnotWin + o];
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
