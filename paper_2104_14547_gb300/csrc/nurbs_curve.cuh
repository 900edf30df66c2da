// Curve kernels: one warp per curve.
//
// A curve C(u) = sum_r N_r(u) Pw_r / W (the curve form of Eq. 3) has no second
// direction to share work across, so the tile kernels' row/column split does
// not fit it.  The forward alone interleaves the samples over the lanes
// (curve_eval_body).  The gradient kernels accumulate the adjoint of the net
// instead: lane L of a warp takes the contiguous samples [L*nb, (L+1)*nb) of
// its curve.  Samples are non-decreasing, so the lane walks
// them with the knot span never decreasing and keeps in registers:
//   - the window of the P+1 homogeneous control points Pw[s-P .. s];
//   - their adjoint accumulators tau[r] = sum_b N_r(u_b) lambda_b, where
//     lambda = (g / W, -S.g / W) and g = dL/dS (Eq. 7, Eq. 8);
//   - with knot gradients, the 2P knot accumulators of the same span (the
//     reverse-mode knot derivative of the basis, the sigma -> 0 reading of
//     Sec. 3.2).
//
// Retiring rows.  A control point (or knot) leaves the window as the span
// advances.  It then goes to the warp's shared block if this lane is its first
// covering lane.  Otherwise it is one of the at most P+1 points (2P knots) this
// lane shares with the previous lane, and it goes to the lane's overflow block.
//
// The final pass adds, for every point, the first lane's block entry and the
// later lanes' overflow entries in lane order.  It then writes the Cartesian
// gradient (and runs Adam, in a fit step), so results are deterministic.
//
// Parameters and dL/dS (or the MSE target) stream through a cp.async ring per
// lane, kCurveStages rounds of kCurveRound samples deep.
#pragma once
#include "nurbs_tile.cuh"

namespace nurbs {

constexpr int kCurveWarps = 4;        // curves in flight per CTA
constexpr int kCurveRound = 4;        // samples per lane per staged round
constexpr int kCurveStages = 2;       // rounds in flight per lane (power of two)
constexpr int kCurveCtrlCap = 256;    // control points per curve on this path (larger: tile kernels)

// Per-warp shared layout (bytes) for degree P and control capacity mc:
//   [0, 4 kc)            knots (kc = mc + P + 1 rounded up to 4)
//   A      16 mc         adjoint block (one float4 per control point)
//   K      4 kc          knot-derivative block
//   lanes  512           int[4][32]: first span, last span, previous lane's last span, -
//   Aov    512 (P+1)     [32][P+1] float4: each lane's overflow block of control points
//   Kov    256 P         [32][2P] floats: each lane's overflow block of knots
//   net    16 mc         the curve's control points (x, y, z, w)
//   ring   2048 stages   [stages][32][4] float4: per lane one chunk of 4 parameters and three
//                        chunks of 4 targets (x y z); lane L's chunk c sits at slot
//                        (c + ((L >> 1) & 3)) mod 4 so that the lanes' reads of one
//                        chunk hit distinct bank groups per quarter warp, and word x
//                        of the lane's 16 at (x + 4 ((L >> 1) & 3)) mod 16
// The forward-only kernels (curve_eval_body) keep just the knots [0, 4 kc) and the
// net as homogeneous points (16 mc).
__host__ __device__ constexpr int curve_kc(int mc, int P) { return (mc + P + 1 + 3) & ~3; }
__host__ __device__ constexpr int curve_off_lanes(int mc, int P) { return 8 * curve_kc(mc, P) + 16 * mc; }
__host__ __device__ constexpr int curve_off_aov(int mc, int P) { return curve_off_lanes(mc, P) + 512; }
__host__ __device__ constexpr int curve_off_net(int mc, int P)
{
    return (curve_off_aov(mc, P) + 512 * (P + 1) + 256 * P + 15) & ~15;
}
__host__ __device__ constexpr int curve_off_ring(int mc, int P) { return curve_off_net(mc, P) + 16 * mc; }
__host__ __device__ constexpr int curve_warp_bytes(int mc, int P, bool grad)
{
    return grad ? curve_off_ring(mc, P) + kCurveStages * 32 * 16 * 4 : 4 * curve_kc(mc, P) + 16 * mc;
}

// 16 bytes from shared to global memory (both 16-byte aligned)
__device__ __forceinline__ void st_global16(float* dst, const float* src)
{
    *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
}

// This lane's share of a curve's samples: [b0, b1), a whole number of rounds of
// kCurveRound samples (the last active lane may be short).
struct CurveLane {
    int nb, b0, b1, rounds;
    bool al16;   // parameters and targets start on 16-byte boundaries
};

__device__ __forceinline__ CurveLane curve_lane(const ItemDev& it, int lane)
{
    CurveLane c;
    const int ns = it.nv;
    c.nb = (ns + 32 * kCurveRound - 1) / (32 * kCurveRound) * kCurveRound;
    c.b0 = min(lane * c.nb, ns);
    c.b1 = min(c.b0 + c.nb, ns);
    c.rounds = c.nb / kCurveRound;
    c.al16 = ((it.param_v & 3) == 0) && ((it.pts & 3) == 0);
    return c;
}

// Stage round k of this lane's parameters and targets: one cp.async group (empty
// past the lane's last round).
__device__ __forceinline__ void curve_issue(const KParams& kp, const ItemDev& it, const CurveLane& c, float* s_ring,
                                            int lane, int k)
{
    constexpr int R = kCurveRound;
    if (k < c.rounds) {
        const float* __restrict__ gu = kp.params + it.param_v;
        const float* __restrict__ gt = kp.gin + 3 * it.pts;
        const int swz = (lane >> 1) & 3;
        const int bb = c.b0 + k * R;
        float* dst = s_ring + ((k & (kCurveStages - 1)) * 32 + lane) * 16;
        if (c.al16 && bb + R <= c.b1) {
            cp_async16(dst + 4 * (swz & 3), gu + bb);
            cp_async16(dst + 4 * ((1 + swz) & 3), gt + 3 * bb);
            cp_async16(dst + 4 * ((2 + swz) & 3), gt + 3 * bb + 4);
            cp_async16(dst + 4 * ((3 + swz) & 3), gt + 3 * bb + 8);
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (bb + j < c.b1) {
                    cp_async4(dst + ((j + 4 * swz) & 15), gu + bb + j);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int w = 3 * j + q;   // target word of the round
                        cp_async4(dst + ((4 + w + 4 * swz) & 15), gt + 3 * (bb + j) + q);
                    }
                }
            }
        }
    }
    cp_async_commit();
}

// Issue the staging of curve t: its knots and control net (one group), then its
// first kCurveStages rounds.  A warp stages its next curve while its final pass of
// the current one runs: that pass reads none of these buffers.
template <int P>
__device__ __forceinline__ void curve_stage(const KParams& kp, int t, unsigned char* wsm)
{
    const int lane = threadIdx.x & 31;
    const int mc = kp.c_mc;
    float* s_kn = reinterpret_cast<float*>(wsm);
    float4* s_net = reinterpret_cast<float4*>(wsm + curve_off_net(mc, P));
    float* s_ring = reinterpret_cast<float*>(wsm + curve_off_ring(mc, P));
    const ItemDev it = kp.items[kp.tiles[t].item];
    const int nc = it.m1, nk = nc + P + 1;
    const float* __restrict__ gU = kp.knots + it.knot_v;
    const float4* __restrict__ gP = kp.ctrl + it.ctrl;
    for (int k = lane; k < nk; k += 32) cp_async4(s_kn + k, gU + k);
    for (int i = lane; i < nc; i += 32)
        cp_async16(reinterpret_cast<float*>(s_net + i), reinterpret_cast<const float*>(gP + i));
    cp_async_commit();
    const CurveLane c = curve_lane(it, lane);
#pragma unroll
    for (int k = 0; k < kCurveStages; ++k) curve_issue(kp, it, c, s_ring, lane, k);
}

// Gradient kernels (backward, MSE, fit step): the per-lane window walk above.  The
// curve's staging (curve_stage) was issued before the call; returns the warp's next
// curve, already staged.
template <int P, bool KNOTS, bool MSE>
__device__ __forceinline__ int curve_body(const KParams& kp, int t, unsigned char* wsm)
{
    constexpr int PB = P + 1;
    constexpr int KW = 2 * P;
    constexpr int R = kCurveRound;
    const int lane = threadIdx.x & 31;
    const int mc = kp.c_mc;
    const int kc = curve_kc(mc, P);
    float* s_kn = reinterpret_cast<float*>(wsm);
    float4* s_A = reinterpret_cast<float4*>(wsm + 4 * kc);
    float* s_K = reinterpret_cast<float*>(wsm + 4 * kc + 16 * mc);
    int* s_ln = reinterpret_cast<int*>(wsm + curve_off_lanes(mc, P));
    float4* s_Aov = reinterpret_cast<float4*>(wsm + curve_off_aov(mc, P));
    float* s_Kov = reinterpret_cast<float*>(wsm + curve_off_aov(mc, P) + 512 * PB);
    float4* s_net = reinterpret_cast<float4*>(wsm + curve_off_net(mc, P));
    float* s_ring = reinterpret_cast<float*>(wsm + curve_off_ring(mc, P));

    const int item = kp.tiles[t].item;
    const ItemDev it = kp.items[item];
    const int nc = it.m1, n = nc - 1, ns = it.nv, nk = nc + P + 1;
    const float* __restrict__ gu = kp.params + it.param_v;

    const CurveLane cl = curve_lane(it, lane);
    const int nb = cl.nb, b0 = cl.b0, b1 = cl.b1, rounds = cl.rounds;
    const bool act = b0 < b1;
    const int nact = nb > 0 ? (ns + nb - 1) / nb : 0;   // active lanes form a prefix
    const int swz = (lane >> 1) & 3;
    auto issue = [&](int k) { curve_issue(kp, it, cl, s_ring, lane, k); };
    cp_async_wait<kCurveStages>();   // the knots and the control net
    __syncwarp();
    for (int i = lane; i < nc; i += 32) s_net[i] = homog(s_net[i]);   // kept as Pw from here on
    __syncwarp();

    // device checks and the spans of this lane's first and last samples
    unsigned err = 0;
    for (int k = lane; k < nk - 1; k += 32)
        if (s_kn[k] > s_kn[k + 1]) err |= kErrKnots;
    if (lane == 0 && !(s_kn[n] < s_kn[n + 1])) err |= kErrKnots;
    const float ulo = s_kn[P], uhi = s_kn[n + 1];
    int sf = P, sl = -1;
    if (act) {
        const float uf = gu[b0], ul = gu[b1 - 1];
        sf = find_span(n, P, fminf(fmaxf(uf, ulo), uhi), s_kn);
        sl = find_span(n, P, fminf(fmaxf(ul, ulo), uhi), s_kn);
        if (b0 > 0 && gu[b0 - 1] > uf) err |= kErrOrder;
    }
    const int pm0 = __shfl_up_sync(0xffffffffu, sl, 1);
    const int pm = lane == 0 ? -1 : pm0;    // the previous lane's last span
    s_ln[lane] = sf;
    s_ln[32 + lane] = sl;
    s_ln[64 + lane] = pm;

    const int ilo = sf - P, klo = sf - P + 1;   // this lane's first control point and knot
    float4 Qw[PB], tau[PB];
    float kacc[KW > 0 ? KW : 1];
#pragma unroll
    for (int r = 0; r < PB; ++r) { Qw[r] = f4zero(); tau[r] = f4zero(); }
#pragma unroll
    for (int k = 0; k < (KW > 0 ? KW : 1); ++k) kacc[k] = 0.f;
    float lossacc = 0.f, uprev = -3.0e38f;
    const float gsc = it.gscale > 0.f ? it.gscale : kp.grad_scale;   // the item's own dL/dS scale, if set
    int cur = -1;

    auto retire_row = [&](int i, float4 v) {
        if (i > pm) s_A[i] = v;
        else if (i - ilo <= P) s_Aov[lane * PB + (i - ilo)] = v;
    };
    auto retire_knot = [&](int kk, float v) {
        if (kk > pm + P) s_K[kk] = v;
        else if (kk - klo < KW) s_Kov[lane * KW + (kk - klo)] = v;
    };
    // the window starts at the span of the lane's first sample
    if (act) {
#pragma unroll
        for (int r = 0; r < PB; ++r) Qw[r] = s_net[sf - P + r];
        cur = sf;
    }
    // move the window to span s (s >= cur): retire what leaves, load what enters
    auto advance = [&](int s) {
        while (cur < s) {
            retire_row(cur - P, tau[0]);
            if constexpr (KNOTS) retire_knot(cur - P + 1, kacc[0]);
#pragma unroll
            for (int r = 0; r < P; ++r) { Qw[r] = Qw[r + 1]; tau[r] = tau[r + 1]; }
            tau[P] = f4zero();
            if constexpr (KNOTS) {
#pragma unroll
                for (int k = 0; k + 1 < KW; ++k) kacc[k] = kacc[k + 1];
                kacc[KW - 1] = 0.f;
            }
            ++cur;
            if (cur > s - PB) Qw[P] = s_net[cur];   // only the last P+1 matter
        }
    };

    const bool has_pts = kp.pts != nullptr;
    // Points of a round take the place of its targets in the ring and leave in three
    // 16-byte stores per lane: scattered 4-byte stores, 384 bytes apart across the
    // warp, cost several times more than the point's arithmetic.  The knot-gradient
    // kernels have no registers to spare for it and store points directly.
    constexpr bool kStage = !KNOTS;
    // this lane's chunk offsets in a ring stage (floats); word w = 3j + c of a round's
    // targets (and points) sits in chunk 1 + w / 4
    const int kb = 4 * swz;
    const int o1 = 4 * ((1 + swz) & 3), o2 = 4 * ((2 + swz) & 3), o3 = 4 * ((3 + swz) & 3);
    auto word = [&](int w) { return (4 + w + kb) & 15; };   // target (point) word w of the round
    // one sample: span, basis, point, MSE and the adjoint accumulations
    // Samples past the lane's end (the last active lane's short tail, lanes without
    // samples) run the body too, as no-ops: every lane takes the same path, so the
    // window step below is a warp-uniform branch.
    auto process = [&](int b, float u, float gx, float gy, float gz, float* rb, int j, bool valid) {
        if (valid) {
            if (!(u >= ulo && u <= uhi)) err |= kErrDomain;
            if (u < uprev) err |= kErrOrder;
            uprev = u;
        }
        u = fminf(fmaxf(u, ulo), uhi);
        // The samples are non-decreasing, so the span only moves forward, almost always
        // by one knot.  Lanes change span at different samples; a loop per lane made
        // the warp run it at almost every sample, so the one-knot step is taken by all
        // lanes together (selects), and only a sample more than one span ahead falls
        // back to the binary search and the per-lane loop.
        const bool adv = valid && cur < n && !(u < s_kn[cur + 1]);
        if (__any_sync(0xffffffffu, adv)) {
            if (adv) {
                retire_row(cur - P, tau[0]);
                if constexpr (KNOTS) retire_knot(cur - P + 1, kacc[0]);
            }
#pragma unroll
            for (int r = 0; r < P; ++r) {
                Qw[r] = adv ? Qw[r + 1] : Qw[r];
                tau[r] = adv ? tau[r + 1] : tau[r];
            }
            tau[P] = adv ? f4zero() : tau[P];
            if constexpr (KNOTS) {
#pragma unroll
                for (int k = 0; k + 1 < KW; ++k) kacc[k] = adv ? kacc[k + 1] : kacc[k];
                kacc[KW - 1] = adv ? 0.f : kacc[KW - 1];
            }
            if (adv) {
                ++cur;
                Qw[P] = s_net[cur];
            }
            const bool more = adv && cur < n && !(u < s_kn[cur + 1]);
            if (__any_sync(0xffffffffu, more)) {
                if (more) advance(find_span(n, P, u, s_kn));
            }
        }
        const int s = cur < 0 ? P : cur;   // lanes without samples compute on a valid span
        float N[PB];
        basis_funs<P>(s, u, s_kn, N);
        float4 Cw = f4zero();
#pragma unroll
        for (int r = 0; r < PB; ++r) Cw = fma4(N[r], Qw[r], Cw);
        const float inv = rcp_approx(Cw.w);
        const float Sx = Cw.x * inv, Sy = Cw.y * inv, Sz = Cw.z * inv;
        if (has_pts && valid) {
            if constexpr (kStage) {
                rb[word(3 * j)] = Sx; rb[word(3 * j + 1)] = Sy; rb[word(3 * j + 2)] = Sz;
            } else {
                float* o = kp.pts + 3 * (it.pts + b);
                o[0] = Sx; o[1] = Sy; o[2] = Sz;
            }
        }
        float ginv = inv;
        if constexpr (MSE) {
            gx = valid ? Sx - gx : 0.f; gy = valid ? Sy - gy : 0.f; gz = valid ? Sz - gz : 0.f;
            lossacc = fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, lossacc)));
            ginv *= gsc;
        }
        const float lx = gx * ginv, ly = gy * ginv, lz = gz * ginv;
        const float4 lam = valid ? make_float4(lx, ly, lz, -fmaf(Sx, lx, fmaf(Sy, ly, Sz * lz))) : f4zero();
#pragma unroll
        for (int r = 0; r < PB; ++r) tau[r] = fma4(N[r], lam, tau[r]);
        if constexpr (KNOTS) {
            float beta[PB];
#pragma unroll
            for (int r = 0; r < PB; ++r) beta[r] = dot4(Qw[r], lam);
            float dk[2 * P + 1];
            basis_knot_vjp<P>(s, u, s_kn, beta, dk);
            if (kp.knot_sigma > 0.f) knot_sigma_terms<P>(s, u, s_kn, beta, kp.knot_sigma, dk);
#pragma unroll
            for (int q = 0; q < KW; ++q) kacc[q] += dk[q];
        }
    };

    const bool st16 = has_pts && (it.pts & 3) == 0;
    for (int k = 0; k < rounds; ++k) {
        cp_async_wait<kCurveStages - 1>();   // round k has landed (later ones may be in flight)
        float* rb = s_ring + ((k & (kCurveStages - 1)) * 32 + lane) * 16;
        const int bb = b0 + k * R;
        // one copy of the per-sample body (unrolling it four times costs more in
        // instruction fetch than it saves)
#pragma unroll 1
        for (int j = 0; j < R; ++j) {
            float g[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) g[c] = rb[word(3 * j + c)];
            process(bb + j, rb[(j + kb) & 15], g[0], g[1], g[2], rb, j, bb + j < b1);
        }
        if (kStage && has_pts) {   // sample j's targets were read before its point was written
            float* o = kp.pts + 3 * (it.pts + (long long)bb);
            if (st16 && bb + R <= b1) {
                st_global16(o, rb + o1);
                st_global16(o + 4, rb + o2);
                st_global16(o + 8, rb + o3);
            } else {
                for (int w = 0; w < 3 * min(R, b1 - bb); ++w) o[w] = rb[word(w)];
            }
        }
        __syncwarp();
        issue(k + kCurveStages);   // the stage just read is refilled for a later round
    }
    if (cur >= 0) {
#pragma unroll
        for (int r = 0; r < PB; ++r) retire_row(cur - P + r, tau[r]);
        if constexpr (KNOTS) {
#pragma unroll
            for (int q = 0; q < KW; ++q) retire_knot(cur - P + 1 + q, kacc[q]);
        }
    }
    cp_async_wait<0>();
    if (err) atomicOr(&kp.hdr->error, err);
    __syncwarp();

#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) lossacc += __shfl_xor_sync(0xffffffffu, lossacc, o);
    if (lane == 0 && kp.loss_items != nullptr) kp.loss_items[item] = lossacc;
    // The warp's next curve is taken now, when this one has only its final pass left
    // (so the queue still hands curves to the warps that finish first), and staged
    // while that pass runs.
    int nq = 0;
    if (lane == 0) nq = kp.t0 + (int)gridDim.x * kCurveWarps + (int)atomicAdd(kp.queue, 1u);
    const int nt = __shfl_sync(0xffffffffu, nq, 0);   // every lane is past its reads of knots, net and ring
    if (nt < kp.t1) curve_stage<P>(kp, nt, wsm);

    // First lane whose last span reaches index x (spans of active lanes are sorted).
    auto first_lane = [&](int x) {
        int lo = 0, hi = nact;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_ln[32 + mid] < x) lo = mid + 1; else hi = mid;
        }
        return lo;
    };

    if (kp.grad_ctrl != nullptr || kp.fit) {
        float lr_t, isb2;
        adam_corrections(kp, it, lr_t, isb2);
        constexpr int EB = 2;
        for (int i0 = lane; i0 < nc; i0 += EB * 32) {
            float4 a[EB], c[EB], mm[EB], vv[EB];
#pragma unroll
            for (int e = 0; e < EB; ++e) {
                const int i = i0 + 32 * e;
                a[e] = c[e] = mm[e] = vv[e] = f4zero();
                if (i >= nc) continue;
                c[e] = kp.ctrl[it.ctrl + i];
                if (kp.fit) { mm[e] = kp.adam_m[it.ctrl + i]; vv[e] = kp.adam_v[it.ctrl + i]; }
                bool first = true;
                for (int l = first_lane(i); l < nact && s_ln[l] - P <= i; ++l) {
                    if (first) {
                        a[e] = s_A[i];
                        first = false;
                    } else {
                        const int d = i - (s_ln[l] - P);
                        if (d >= 0 && d < PB) {
                            const float4 v = s_Aov[l * PB + d];
                            a[e].x += v.x; a[e].y += v.y; a[e].z += v.z; a[e].w += v.w;
                        }
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < EB; ++e) {
                const int i = i0 + 32 * e;
                if (i < nc) finish_point(kp, it.ctrl + i, c[e], a[e], mm[e], vv[e], lr_t, isb2);
            }
        }
    }
    if constexpr (KNOTS) {
        if (kp.grad_knots != nullptr) {
            for (int kk = lane; kk < nk; kk += 32) {
                float acc = 0.f;
                if (kk >= P + 1 && kk <= n) {   // the p+1 end knots on each side get 0
                    bool first = true;
                    for (int l = first_lane(kk - P); l < nact && s_ln[l] - P + 1 <= kk; ++l) {
                        if (first) {
                            acc = s_K[kk];
                            first = false;
                        } else {
                            const int d = kk - (s_ln[l] - P + 1);
                            if (d >= 0 && d < KW) acc += s_Kov[l * KW + d];
                        }
                    }
                }
                kp.grad_knots[it.knot_v + kk] = acc;
            }
        }
    }
    __syncwarp();
    return nt;
}

// Forward (points, and tangents when DER): no adjoint to accumulate, so no
// window walk.  Lane L takes samples L, L + 32, ... of the curve: the warp's 32
// samples are consecutive, the stores of a step are contiguous and no lane has a
// span change of its own for the warp to wait on.  The spans of one step are
// non-decreasing across the lanes and not below the previous step's last span
// s0, so the warp stages the 32 knots U[s0+1 .. s0+32] one per lane and each lane
// counts those <= u by a shuffle binary search (the largest k with U_k <= u, as
// find_span).  A lane whose u lies past all 32 (fewer samples than spans) falls
// back to the binary search over the whole knot vector.
template <int P, bool DER>
__device__ __forceinline__ void curve_eval_body(const KParams& kp, int t, unsigned char* wsm)
{
    constexpr int PB = P + 1;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int kc = curve_kc(kp.c_mc, P);
    float* s_kn = reinterpret_cast<float*>(wsm);
    float4* s_net = reinterpret_cast<float4*>(wsm + 4 * kc);   // homogeneous Pw

    const int item = kp.tiles[t].item;
    const ItemDev it = kp.items[item];
    const int nc = it.m1, n = nc - 1, ns = it.nv, nk = nc + P + 1;
    const float* __restrict__ gU = kp.knots + it.knot_v;
    const float* __restrict__ gu = kp.params + it.param_v;
    const float4* __restrict__ gP = kp.ctrl + it.ctrl;
    for (int k = lane; k < nk; k += 32) s_kn[k] = __ldg(gU + k);
    for (int i = lane; i < nc; i += 32) s_net[i] = homog(__ldg(gP + i));
    __syncwarp();

    unsigned err = 0;
    for (int k = lane; k < nk - 1; k += 32)
        if (s_kn[k] > s_kn[k + 1]) err |= kErrKnots;
    if (lane == 0 && !(s_kn[n] < s_kn[n + 1])) err |= kErrKnots;
    const float ulo = s_kn[P], uhi = s_kn[n + 1];
    float* __restrict__ pts = kp.pts != nullptr ? kp.pts + 3 * it.pts : nullptr;
    float* __restrict__ tan = DER && kp.d_dv != nullptr ? kp.d_dv + 3 * it.pts : nullptr;

    int s0 = P;               // last span of the previous step
    float ulast = -3.0e38f;   // last sample of the previous step
    // parameters two steps ahead are in flight while a step computes (lanes past the
    // end take the last knot)
    auto load_u = [&](int b) { return b < ns ? __ldg(gu + b) : uhi; };
    float u1 = load_u(lane), u2 = load_u(32 + lane);
    for (int b0 = 0; b0 < ns; b0 += 32) {
        const int b = b0 + lane;
        const bool act = b < ns;
        float u = u1;
        u1 = u2;
        u2 = load_u(b0 + 64 + lane);
        if (act && !(u >= ulo && u <= uhi)) err |= kErrDomain;
        const float up = __shfl_up_sync(full, u, 1);
        if (act && u < (lane == 0 ? ulast : up)) err |= kErrOrder;
        ulast = __shfl_sync(full, u, 31);
        u = fminf(fmaxf(u, ulo), uhi);
        // count the staged knots U[s0+1 .. s0+32] (only those up to U[n]) that are <= u
        const int kk = s0 + 1 + lane;
        const float kv = kk <= n ? s_kn[kk] : 3.0e38f;
        int cnt = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const float k = __shfl_sync(full, kv, cnt + step - 1);
            if (k <= u) cnt += step;
        }
        const float kv31 = __shfl_sync(full, kv, 31);   // every lane takes part in each shuffle
        int s = min(s0 + cnt, n);   // (the bound matters only for non-finite knots)
        if (cnt == 31 && kv31 <= u) s = find_span(n, P, u, s_kn);
        s0 = __shfl_sync(full, s, 31);
        if (!act) continue;
        float N[PB];
        float dN[DER ? PB : 1];
        if constexpr (DER) basis_funs_d<P>(s, u, s_kn, N, dN);
        else basis_funs<P>(s, u, s_kn, N);
        float4 Cw = f4zero(), Cd = f4zero();
#pragma unroll
        for (int r = 0; r < PB; ++r) {
            const float4 pw = s_net[s - P + r];
            Cw = fma4(N[r], pw, Cw);
            if constexpr (DER) Cd = fma4(dN[r], pw, Cd);
        }
        const float inv = rcp_approx(Cw.w);
        const float Sx = Cw.x * inv, Sy = Cw.y * inv, Sz = Cw.z * inv;
        if (pts != nullptr) {
            float* o = pts + 3 * (long long)b;
            o[0] = Sx; o[1] = Sy; o[2] = Sz;
        }
        if constexpr (DER) {
            // tangent C' = (A' - W' C) / W with (A', W') = sum_r dN_r Pw_r
            if (tan != nullptr) {
                float* o = tan + 3 * (long long)b;
                o[0] = (Cd.x - Cd.w * Sx) * inv;
                o[1] = (Cd.y - Cd.w * Sy) * inv;
                o[2] = (Cd.z - Cd.w * Sz) * inv;
            }
        }
    }
    if (err) atomicOr(&kp.hdr->error, err);
    __syncwarp();
}

// Resident CTAs per SM: the gradient kernels need 128 registers a thread.
template <int P, bool GRAD>
constexpr int curve_min_blocks() { return GRAD ? 4 : 8; }

template <int P, bool GRAD, bool KNOTS, bool MSE, bool DER = false>
__global__ void __launch_bounds__(32 * kCurveWarps, curve_min_blocks<P, GRAD>())
    curves_kernel(const __grid_constant__ KParams kp)
{
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wsm = reinterpret_cast<unsigned char*>(smem4) + warp * kp.c_wbytes;
    // the first curve of each warp is its own index; later ones come from the queue
    int t = kp.t0 + (int)blockIdx.x * kCurveWarps + warp;
    if constexpr (GRAD) {
        if (t < kp.t1) curve_stage<P>(kp, t, wsm);
        while (t < kp.t1) t = curve_body<P, KNOTS, MSE>(kp, t, wsm);
    } else {
        while (t < kp.t1) {
            curve_eval_body<P, DER>(kp, t, wsm);
            int nt = 0;
            if (lane == 0) nt = kp.t0 + (int)gridDim.x * kCurveWarps + (int)atomicAdd(kp.queue, 1u);
            t = __shfl_sync(0xffffffffu, nt, 0);
        }
    }
    __syncthreads();
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

}  // namespace nurbs
