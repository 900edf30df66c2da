// Device building blocks shared by the libnurbs kernels: knot-span search,
// nonzero Cox-de Boor basis and its reverse-mode knot derivative.  The knot
// vectors are read through plain pointers (the kernels stage them in shared
// memory first).
#pragma once
#include <cuda_runtime.h>

namespace nurbs {

// Reciprocal with one MUFU op (relative error below 2^-22 for normal inputs);
// every denominator here is a positive knot difference.
__device__ __forceinline__ float frcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Knot-span search (Sec. 3.1 step 1): the largest k in [p, n] with U[k] <= u,
// and n when u >= U[n+1].  Half-open spans, so a zero-length span is never
// returned.
__device__ __forceinline__ int find_span(int n, int p, float u, const float* U)
{
    if (u >= U[n + 1]) return n;
    int lo = p, hi = n;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (U[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The P+1 nonzero basis functions N_{s-P..s}^P(u) of Eq. 4, evaluated with the
// triangular scheme (each level from the previous one; the denominators
// U_{s+r+1} - U_{s+1-j+r} are positive on a non-empty span).
template <int P>
__device__ __forceinline__ void basis_funs(int s, float u, const float* U, float (&N)[P + 1])
{
    N[0] = 1.f;
    if constexpr (P > 0) {
        float left[P + 1], right[P + 1];
#pragma unroll
        for (int j = 1; j <= P; ++j) {
            left[j] = u - U[s + 1 - j];
            right[j] = U[s + j] - u;
            float saved = 0.f;
#pragma unroll
            for (int r = 0; r < j; ++r) {
                float temp = N[r] * frcp(right[r + 1] + left[j - r]);
                N[r] = fmaf(right[r + 1], temp, saved);
                saved = left[j - r] * temp;
            }
            N[j] = saved;
        }
    }
}

// The P+1 nonzero basis functions and their first u-derivatives on span s:
// the triangle of basis_funs up to degree P-1 is kept, and
//   dN_i^P / du = P N_i^{P-1} / (U_{i+P} - U_i) - P N_{i+1}^{P-1} / (U_{i+P+1} - U_{i+1})
// (the u-derivative of Eq. 4; both denominators are positive on a non-empty span).
template <int P>
__device__ __forceinline__ void basis_funs_d(int s, float u, const float* U, float (&N)[P + 1], float (&dN)[P + 1])
{
    N[0] = 1.f;
    dN[0] = 0.f;
    if constexpr (P > 0) {
        float left[P + 1], right[P + 1], prev[P + 1];
#pragma unroll
        for (int j = 1; j <= P; ++j) {
            left[j] = u - U[s + 1 - j];
            right[j] = U[s + j] - u;
            if (j == P) {
#pragma unroll
                for (int r = 0; r < P; ++r) prev[r] = N[r];   // N^{P-1}_{s-P+1+r}
            }
            float saved = 0.f;
#pragma unroll
            for (int r = 0; r < j; ++r) {
                float temp = N[r] * frcp(right[r + 1] + left[j - r]);
                N[r] = fmaf(right[r + 1], temp, saved);
                saved = left[j - r] * temp;
            }
            N[j] = saved;
        }
#pragma unroll
        for (int r = 0; r <= P; ++r) {
            const float a = r >= 1 ? prev[r - 1] * frcp(U[s + r] - U[s - P + r]) : 0.f;
            const float b = r <= P - 1 ? prev[r] * frcp(U[s + r + 1] - U[s - P + r + 1]) : 0.f;
            dN[r] = (float)P * (a - b);
        }
    }
}

// Reverse-mode derivative of basis_funs with respect to the knots (the knot
// derivative of Sec. 3.2 in its sigma -> 0 reading: the degree-0 indicators
// contribute nothing, every coefficient of Eq. 4 is differentiated).
// Given the cotangent nb[r] = dL/dN_{s-P+r}(u), writes
//   dk[k] = sum_r nb[r] * dN_{s-P+r}(u) / dU[s-P+1+k],  k = 0 .. 2P-1.
template <int P>
__device__ __forceinline__ void basis_knot_vjp(int s, float u, const float* U,
                                               const float (&nb_in)[P + 1], float (&dk)[2 * P + 1])
{
    if constexpr (P == 0) {
        dk[0] = 0.f;
    } else {
        float left[P + 1], right[P + 1];
        float tri[P + 1][P + 1];  // tri[j][r] = N^j_{s-j+r}
        tri[0][0] = 1.f;
#pragma unroll
        for (int j = 1; j <= P; ++j) {
            left[j] = u - U[s + 1 - j];
            right[j] = U[s + j] - u;
            float saved = 0.f;
#pragma unroll
            for (int r = 0; r < j; ++r) {
                float temp = tri[j - 1][r] * frcp(right[r + 1] + left[j - r]);
                tri[j][r] = fmaf(right[r + 1], temp, saved);
                saved = left[j - r] * temp;
            }
            tri[j][j] = saved;
        }
        float nb[P + 1], lb[P + 1], rb[P + 1];
#pragma unroll
        for (int r = 0; r <= P; ++r) { nb[r] = nb_in[r]; lb[r] = 0.f; rb[r] = 0.f; }
#pragma unroll
        for (int j = P; j >= 1; --j) {
            float pb[P + 1];
#pragma unroll
            for (int r = 0; r < j; ++r) {
                const float iden = frcp(right[r + 1] + left[j - r]);
                float temp = tri[j - 1][r] * iden;
                // temp feeds tri[j][r] (times right[r+1]) and tri[j][r+1] (times left[j-r])
                float tb = fmaf(right[r + 1], nb[r], left[j - r] * nb[r + 1]);
                float denb = -tb * temp * iden;
                rb[r + 1] += fmaf(temp, nb[r], denb);
                lb[j - r] += fmaf(temp, nb[r + 1], denb);
                pb[r] = tb * iden;
            }
#pragma unroll
            for (int r = 0; r < j; ++r) nb[r] = pb[r];
        }
        // left[j] = u - U[s+1-j]  -> knot index s+1-j = (s-P+1) + (P-j)
        // right[j] = U[s+j] - u   -> knot index s+j   = (s-P+1) + (P-1+j)
#pragma unroll
        for (int j = 1; j <= P; ++j) {
            dk[P - j] = -lb[j];
            dk[P - 1 + j] = rb[j];
        }
    }
}

// The Gaussian-smoothed indicator term of the knot derivative (Sec. 3.2, the
// paper's form with bandwidth sigma > 0), added to dk of basis_knot_vjp.
//
// The degree-0 functions' smoothed knot derivatives, -G(u - U_j) at U_j and
// +G(u - U_{j+1}) at U_{j+1} with G(x) = exp(-x^2 / 2 sigma^2) / (sigma sqrt(2 pi)),
// reach dL/dU_k through the adjoints of every degree-0 function N^0_j,
// j in [s-P, s+P].  Those adjoints are the cotangent nb pushed back through the
// full triangle of Eq. 4 (zero-valued functions included; a coefficient with a
// zero denominator is 0):
//   dk[k - (s-P+1)] += G(u - U_k) (adj N^0_{k-1} - adj N^0_k),  k in [s-P+1, s+P].
// The two knots just outside the window, U_{s-P} and U_{s+P+1}, lie at least P
// spans from u; their terms are left out.
template <int P>
__device__ __forceinline__ void knot_sigma_terms(int s, float u, const float* U, const float (&nb)[P + 1],
                                                 float sigma, float (&dk)[2 * P + 1])
{
    if constexpr (P > 0) {
        float a[2 * P + 1];   // a[t]: adjoint of N^d_{s-P+t} at the current level d
#pragma unroll
        for (int t = 0; t <= 2 * P; ++t) a[t] = t <= P ? nb[t] : 0.f;
#pragma unroll
        for (int d = P; d >= 1; --d) {
            float b[2 * P + 1];
#pragma unroll
            for (int t = 0; t <= 2 * P; ++t) b[t] = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * P - d; ++t) {
                const int i = s - P + t;
                const float ad = U[i + d] - U[i], bd = U[i + d + 1] - U[i + 1];
                const float al = ad > 0.f ? (u - U[i]) * frcp(ad) : 0.f;
                const float be = bd > 0.f ? (U[i + d + 1] - u) * frcp(bd) : 0.f;
                b[t] = fmaf(al, a[t], b[t]);
                b[t + 1] = fmaf(be, a[t], b[t + 1]);
            }
#pragma unroll
            for (int t = 0; t <= 2 * P; ++t) a[t] = b[t];
        }
        const float is = frcp(sigma);
        const float gn = 0.3989422804014327f * is;   // 1 / (sigma sqrt(2 pi))
#pragma unroll
        for (int k = 0; k < 2 * P; ++k) {
            const float x = (u - U[s - P + 1 + k]) * is;
            dk[k] = fmaf(gn * expf(-0.5f * x * x), a[k] - a[k + 1], dk[k]);
        }
    }
}

}  // namespace nurbs
