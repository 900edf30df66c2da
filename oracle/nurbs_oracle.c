/*
 * FP64 CPU oracle for NURBS-Diff (arXiv 2104.14547): rational B-spline curve and
 * surface evaluation and the derivatives of the evaluated points with respect to
 * control points, weights and knots.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA path
 * is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header or table with the CUDA
 * library and includes nothing from it.
 *
 * Everything is computed in double precision from the caller's values (the tests
 * feed it the same FP32 values the GPU sees, widened exactly to double).
 *
 * Layouts (all row-major, caller-owned):
 *   control net  ctrl[i][j][4] = (x, y, z, w): Cartesian point and its weight,
 *                i = 0..n1-1 (u direction), j = 0..m1-1 (v direction)
 *   knot vectors U[n1+p+1], V[m1+q+1], non-decreasing
 *   samples      u[nu], v[nv]; output point (a, b) is S(u[a], v[b])
 *   points       out[a][b][3]
 *   gradients    dctrl[i][j][4] = (dL/dx, dL/dy, dL/dz, dL/dw), dU[n1+p+1], dV[m1+q+1]
 *
 * Readings of the paper taken here (each one is listed with its reason in the design notes):
 *   - span intervals are half-open [U_k, U_k+1); the end of the domain u = U_{n+1}
 *     belongs to the last non-empty span k = n (the text's step-1 wording and the
 *     Piegl-Tiller span search the paper cites; Eq. 5 prints a closed interval);
 *   - 0/0 in the Cox-de Boor recursion (Eq. 4) is taken as 0;
 *   - knot derivative: the exact almost-everywhere derivative of the recursion
 *     (Eq. 4) with the degree-0 indicator's knot derivative set to zero, i.e. the
 *     sigma -> 0 limit of the Gaussian-smoothed indicator of Sec. 3.2;
 *   - knot gradients are reported for interior knots k in [p+1, n] only; the
 *     2(p+1) end knots get 0 (the domain is fixed to [0,1], Sec. 3.1);
 *   - gradients are with respect to the Cartesian control points and the weights
 *     (Psi = {P, U, V, W}, Sec. 3).
 */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDEG 16

/* ---------------------------------------------------------------------------
 * Span search (Sec. 3.1 step 1; Piegl & Tiller, The NURBS Book, A2.1).
 * Returns the k in [p, n] with U[k] <= u < U[k+1]; u >= U[n+1] gives n.
 * Binary search for the largest such k, so zero-length spans are never chosen.
 * ------------------------------------------------------------------------- */
int nurbs_oracle_find_span(int n, int p, double u, const double* U)
{
    if (u >= U[n + 1]) return n;
    if (u <= U[p]) {
        /* largest k in [p, n] with U[k] <= u: walk right over repeated U[p]. */
        int k = p;
        while (k < n && U[k + 1] <= u) ++k;
        return k;
    }
    int low = p, high = n + 1;
    int mid = (low + high) / 2;
    while (u < U[mid] || u >= U[mid + 1]) {
        if (u < U[mid]) high = mid; else low = mid;
        mid = (low + high) / 2;
    }
    return mid;
}

/* ---------------------------------------------------------------------------
 * The p+1 nonzero basis functions N_{span-p..span}^p(u) (Sec. 3.1 step 2, the
 * Cox-de Boor recursion of Eq. 4 organised as in Piegl & Tiller A2.2).
 * ------------------------------------------------------------------------- */
void nurbs_oracle_basis_funs(int span, double u, int p, const double* U, double* N)
{
    double left[OR_MAXDEG + 1], right[OR_MAXDEG + 1];
    N[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = u - U[span + 1 - j];
        right[j] = U[span + j] - u;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double temp = N[r] / (right[r + 1] + left[j - r]);
            N[r] = saved + right[r + 1] * temp;
            saved = left[j - r] * temp;
        }
        N[j] = saved;
    }
}

/* ---------------------------------------------------------------------------
 * Brute-force Cox-de Boor (Eq. 4 and Eq. 5) for ONE basis function N_i^p(u),
 * recursing all the way down, with the half-open indicator and 0/0 := 0.
 * nknots = n + p + 2 (so n = nknots - p - 2).  Exponential in p; tiny cases only.
 * ------------------------------------------------------------------------- */
static double cdb_rec(int i, int k, double u, const double* U, int last_span)
{
    if (k == 0) {
        if (U[i] <= u && u < U[i + 1]) return 1.0;
        /* u at the right end of the domain belongs to the last non-empty span */
        if (i == last_span && u == U[i + 1]) return 1.0;
        return 0.0;
    }
    double a = 0.0, b = 0.0;
    double d1 = U[i + k] - U[i];
    double d2 = U[i + k + 1] - U[i + 1];
    if (d1 != 0.0) a = (u - U[i]) / d1 * cdb_rec(i, k - 1, u, U, last_span);
    if (d2 != 0.0) b = (U[i + k + 1] - u) / d2 * cdb_rec(i + 1, k - 1, u, U, last_span);
    return a + b;
}

double nurbs_oracle_basis_cox_de_boor(int i, int p, double u, const double* U, int nknots)
{
    int n = nknots - p - 2;
    int last_span = nurbs_oracle_find_span(n, p, U[n + 1], U);
    return cdb_rec(i, p, u, U, last_span);
}

/* ---------------------------------------------------------------------------
 * Knot Jacobian of the nonzero basis by forward-mode dual numbers pushed through
 * the same recursion as nurbs_oracle_basis_funs (Sec. 3.2, knot derivative,
 * sigma -> 0 reading).  The p+1 functions depend on the 2p knots
 * U[span-p+1 .. span+p]; dN[r*(2p) + k] = d N_{span-p+r}(u) / d U[span-p+1+k].
 * ------------------------------------------------------------------------- */
void nurbs_oracle_basis_knot_jac(int span, double u, int p, const double* U, double* N, double* dN)
{
    int K = 2 * p;
    double left[OR_MAXDEG + 1], right[OR_MAXDEG + 1];
    double dleft[OR_MAXDEG + 1][2 * OR_MAXDEG], dright[OR_MAXDEG + 1][2 * OR_MAXDEG];
    double dn[OR_MAXDEG + 1][2 * OR_MAXDEG];
    memset(dn, 0, sizeof dn);
    N[0] = 1.0;
    int base = span - p + 1;             /* knot index of dual direction 0 */
    for (int j = 1; j <= p; ++j) {
        left[j] = u - U[span + 1 - j];
        right[j] = U[span + j] - u;
        for (int k = 0; k < K; ++k) { dleft[j][k] = 0.0; dright[j][k] = 0.0; }
        dleft[j][span + 1 - j - base] = -1.0;
        dright[j][span + j - base] = 1.0;
        double saved = 0.0, dsaved[2 * OR_MAXDEG];
        for (int k = 0; k < K; ++k) dsaved[k] = 0.0;
        for (int r = 0; r < j; ++r) {
            double den = right[r + 1] + left[j - r];
            double temp = N[r] / den;
            double dtemp[2 * OR_MAXDEG];
            for (int k = 0; k < K; ++k) {
                double dden = dright[r + 1][k] + dleft[j - r][k];
                dtemp[k] = (dn[r][k] * den - N[r] * dden) / (den * den);
            }
            double nr = saved + right[r + 1] * temp;
            for (int k = 0; k < K; ++k)
                dn[r][k] = dsaved[k] + dright[r + 1][k] * temp + right[r + 1] * dtemp[k];
            N[r] = nr;
            saved = left[j - r] * temp;
            for (int k = 0; k < K; ++k)
                dsaved[k] = dleft[j - r][k] * temp + left[j - r] * dtemp[k];
        }
        N[j] = saved;
        for (int k = 0; k < K; ++k) dn[j][k] = dsaved[k];
    }
    for (int r = 0; r <= p; ++r)
        for (int k = 0; k < K; ++k) dN[r * K + k] = dn[r][k];
}

/* ---------------------------------------------------------------------------
 * Knot Jacobian with the Gaussian-smoothed degree-0 indicator of Sec. 3.2 (the
 * paper's own form of the knot derivative, bandwidth sigma > 0).  The forward
 * stays exact; the degree-0 functions get the derivative of their smoothed
 * form  N^0_j ~ Phi((u - U_j)/sigma) - Phi((u - U_{j+1})/sigma):
 *   dN^0_j/dU_j = -G(u - U_j),   dN^0_j/dU_{j+1} = +G(u - U_{j+1}),
 *   G(x) = exp(-x^2 / (2 sigma^2)) / (sigma sqrt(2 pi)),
 * and both these and the recursion coefficients' derivatives are pushed
 * through the full triangle of Eq. 4 (every function N^d_i with i in
 * [span-p, span+p-d], zero-valued ones included), one knot at a time in
 * forward mode.  Knots U[span-p .. span+p+1] (2p+2 of them);
 * J[r*(2p+2) + k] = dN_{span-p+r}(u) / dU[span-p+k].  0/0 in a coefficient := 0.
 * ------------------------------------------------------------------------- */
static double gauss(double x, double sigma)
{
    return exp(-0.5 * (x / sigma) * (x / sigma)) / (sigma * sqrt(2.0 * M_PI));
}

void nurbs_oracle_basis_knot_jac_sigma(int span, double u, int p, const double* U, double sigma, double* N,
                                       double* J)
{
    int K = 2 * p + 2, lo = span - p;
    for (int k = 0; k < K; ++k) {
        int kk = lo + k;                      /* the knot whose derivative this pass carries */
        double val[2 * OR_MAXDEG + 1], dot[2 * OR_MAXDEG + 1];
        for (int j = lo; j <= span + p; ++j) {
            val[j - lo] = (j == span) ? 1.0 : 0.0;
            double d = 0.0;
            if (sigma > 0.0) {
                if (j == kk) d -= gauss(u - U[j], sigma);
                if (j + 1 == kk) d += gauss(u - U[j + 1], sigma);
            }
            dot[j - lo] = d;
        }
        for (int d = 1; d <= p; ++d) {
            for (int i = lo; i <= span + p - d; ++i) {
                double an = u - U[i], ad = U[i + d] - U[i];
                double bn = U[i + d + 1] - u, bd = U[i + d + 1] - U[i + 1];
                double dan = (i == kk) ? -1.0 : 0.0;
                double dad = ((i + d == kk) ? 1.0 : 0.0) - ((i == kk) ? 1.0 : 0.0);
                double dbn = (i + d + 1 == kk) ? 1.0 : 0.0;
                double dbd = ((i + d + 1 == kk) ? 1.0 : 0.0) - ((i + 1 == kk) ? 1.0 : 0.0);
                double al = 0.0, dal = 0.0, be = 0.0, dbe = 0.0;
                if (ad != 0.0) { al = an / ad; dal = (dan * ad - an * dad) / (ad * ad); }
                if (bd != 0.0) { be = bn / bd; dbe = (dbn * bd - bn * dbd) / (bd * bd); }
                int t = i - lo;
                double v = al * val[t] + be * val[t + 1];
                double dv = dal * val[t] + al * dot[t] + dbe * val[t + 1] + be * dot[t + 1];
                val[t] = v;      /* level d overwrites level d-1 in increasing i */
                dot[t] = dv;
            }
        }
        for (int r = 0; r <= p; ++r) {
            if (k == 0) N[r] = val[r];
            J[r * K + k] = dot[r];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Surface forward (Eq. 3 evaluated as in Sec. 3.1: span, nonzero basis,
 * homogeneous weighted sum, perspective divide).
 * ------------------------------------------------------------------------- */
static void surface_point(int p, int q, int n1, int m1, const double* U, const double* V,
                          const double* ctrl, double u, double v, double* Sw /*4*/)
{
    double Nu[OR_MAXDEG + 1], Nv[OR_MAXDEG + 1];
    int su = nurbs_oracle_find_span(n1 - 1, p, u, U);
    int sv = nurbs_oracle_find_span(m1 - 1, q, v, V);
    nurbs_oracle_basis_funs(su, u, p, U, Nu);
    nurbs_oracle_basis_funs(sv, v, q, V, Nv);
    Sw[0] = Sw[1] = Sw[2] = Sw[3] = 0.0;
    for (int r = 0; r <= p; ++r)
        for (int h = 0; h <= q; ++h) {
            const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
            double b = Nu[r] * Nv[h];
            Sw[0] += b * c[3] * c[0];
            Sw[1] += b * c[3] * c[1];
            Sw[2] += b * c[3] * c[2];
            Sw[3] += b * c[3];
        }
}

void nurbs_oracle_surface_eval(int p, int q, int n1, int m1, const double* U, const double* V,
                               const double* ctrl, int nu, const double* u, int nv, const double* v,
                               double* out)
{
    for (int a = 0; a < nu; ++a)
        for (int b = 0; b < nv; ++b) {
            double Sw[4];
            surface_point(p, q, n1, m1, U, V, ctrl, u[a], v[b], Sw);
            double* o = out + 3 * ((size_t)a * nv + b);
            o[0] = Sw[0] / Sw[3];
            o[1] = Sw[1] / Sw[3];
            o[2] = Sw[2] / Sw[3];
        }
}

/* ---------------------------------------------------------------------------
 * Surface vector-Jacobian product: given g = dL/dS (out layout), accumulate
 *   dL/dP_ij  = sum_ab R_ij(a,b) g_ab                              (Eq. 7)
 *   dL/dw_ij  = sum_ab N_i N_j (P_ij - S_ab) . g_ab / W_ab          (Eq. 8)
 *   dL/dU_k   = sum_ab sum_r g_ab . dS/dN_{i_r}(u_a) * dN_{i_r}/dU_k (Eq. 9 and
 *               the knot derivative of Sec. 3.2), likewise dL/dV_k.
 * Outputs are overwritten.  Sum order: a, then b.
 * ------------------------------------------------------------------------- */
/* Knot Jacobian of one sample: the sigma -> 0 reading over the 2p knots
 * [span-p+1, span+p] (sigma == 0), or the smoothed-indicator form over the 2p+2
 * knots [span-p, span+p+1].  Returns the width; *base = first knot index. */
static int knot_jacobian(int span, double u, int p, const double* U, double sigma, double* N, double* J, int* base)
{
    if (sigma > 0.0) {
        nurbs_oracle_basis_knot_jac_sigma(span, u, p, U, sigma, N, J);
        *base = span - p;
        return 2 * p + 2;
    }
    nurbs_oracle_basis_knot_jac(span, u, p, U, N, J);
    *base = span - p + 1;
    return 2 * p;
}

void nurbs_oracle_surface_vjp_sigma(int p, int q, int n1, int m1, const double* U, const double* V,
                                    const double* ctrl, int nu, const double* u, int nv, const double* v,
                                    const double* g, double* dctrl, double* dU, double* dV, double sigma)
{
    int nU = n1 + p + 1, nV = m1 + q + 1;
    if (dctrl) memset(dctrl, 0, sizeof(double) * 4 * (size_t)n1 * m1);
    if (dU) memset(dU, 0, sizeof(double) * nU);
    if (dV) memset(dV, 0, sizeof(double) * nV);
    double Nu[OR_MAXDEG + 1], Nv[OR_MAXDEG + 1];
    double dNu[(OR_MAXDEG + 1) * (2 * OR_MAXDEG + 2)], dNv[(OR_MAXDEG + 1) * (2 * OR_MAXDEG + 2)];
    for (int a = 0; a < nu; ++a) {
        int su = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        int bu = 0, ku = knot_jacobian(su, u[a], p, U, sigma, Nu, dNu, &bu);
        for (int b = 0; b < nv; ++b) {
            int sv = nurbs_oracle_find_span(m1 - 1, q, v[b], V);
            int bv = 0, kv = knot_jacobian(sv, v[b], q, V, sigma, Nv, dNv, &bv);
            /* NR (3-vector) and W of Eq. 6 */
            double NR[3] = {0, 0, 0}, W = 0;
            for (int r = 0; r <= p; ++r)
                for (int h = 0; h <= q; ++h) {
                    const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                    double bw = Nu[r] * Nv[h] * c[3];
                    NR[0] += bw * c[0]; NR[1] += bw * c[1]; NR[2] += bw * c[2];
                    W += bw;
                }
            const double* ga = g + 3 * ((size_t)a * nv + b);
            if (dctrl) {
                for (int r = 0; r <= p; ++r)
                    for (int h = 0; h <= q; ++h) {
                        size_t ij = (size_t)(su - p + r) * m1 + (sv - q + h);
                        const double* c = ctrl + 4 * ij;
                        double NN = Nu[r] * Nv[h];
                        double R = NN * c[3] / W;                       /* Eq. 7 */
                        dctrl[4 * ij + 0] += R * ga[0];
                        dctrl[4 * ij + 1] += R * ga[1];
                        dctrl[4 * ij + 2] += R * ga[2];
                        /* Eq. 8: (N N P W - NR N N) / W^2, dotted with g */
                        double sw = 0;
                        for (int c3 = 0; c3 < 3; ++c3)
                            sw += (NN * c[c3] * W - NR[c3] * NN) / (W * W) * ga[c3];
                        dctrl[4 * ij + 3] += sw;
                    }
            }
            if (dU) {
                /* Eq. 9: dS/dN_i(u) = (sum_j N_j w_ij P_ij)/W - NR (sum_j N_j w_ij)/W^2 */
                for (int r = 0; r <= p; ++r) {
                    double Qi[3] = {0, 0, 0}, Qw = 0;
                    for (int h = 0; h <= q; ++h) {
                        const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                        Qi[0] += Nv[h] * c[3] * c[0];
                        Qi[1] += Nv[h] * c[3] * c[1];
                        Qi[2] += Nv[h] * c[3] * c[2];
                        Qw += Nv[h] * c[3];
                    }
                    double coef = 0;
                    for (int c3 = 0; c3 < 3; ++c3)
                        coef += (Qi[c3] / W - NR[c3] * Qw / (W * W)) * ga[c3];
                    for (int k = 0; k < ku; ++k)
                        dU[bu + k] += coef * dNu[r * ku + k];
                }
            }
            if (dV) {
                for (int h = 0; h <= q; ++h) {
                    double Qi[3] = {0, 0, 0}, Qw = 0;
                    for (int r = 0; r <= p; ++r) {
                        const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                        Qi[0] += Nu[r] * c[3] * c[0];
                        Qi[1] += Nu[r] * c[3] * c[1];
                        Qi[2] += Nu[r] * c[3] * c[2];
                        Qw += Nu[r] * c[3];
                    }
                    double coef = 0;
                    for (int c3 = 0; c3 < 3; ++c3)
                        coef += (Qi[c3] / W - NR[c3] * Qw / (W * W)) * ga[c3];
                    for (int k = 0; k < kv; ++k)
                        dV[bv + k] += coef * dNv[h * kv + k];
                }
            }
        }
    }
    /* end knots carry no gradient (fixed domain) */
    if (dU) for (int k = 0; k < nU; ++k) if (k < p + 1 || k > n1 - 1) dU[k] = 0.0;
    if (dV) for (int k = 0; k < nV; ++k) if (k < q + 1 || k > m1 - 1) dV[k] = 0.0;
}

void nurbs_oracle_surface_vjp(int p, int q, int n1, int m1, const double* U, const double* V,
                              const double* ctrl, int nu, const double* u, int nv, const double* v,
                              const double* g, double* dctrl, double* dU, double* dV)
{
    nurbs_oracle_surface_vjp_sigma(p, q, n1, m1, U, V, ctrl, nu, u, nv, v, g, dctrl, dU, dV, 0.0);
}

/* ---------------------------------------------------------------------------
 * Curve forward and VJP: the same method with one parametric direction (Sec. 3,
 * curves handled "by suitably adjusting the dimensions").  ctrl[i][4], out[a][3].
 * ------------------------------------------------------------------------- */
void nurbs_oracle_curve_eval(int p, int n1, const double* U, const double* ctrl,
                             int nu, const double* u, double* out)
{
    double N[OR_MAXDEG + 1];
    for (int a = 0; a < nu; ++a) {
        int s = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        nurbs_oracle_basis_funs(s, u[a], p, U, N);
        double Cw[4] = {0, 0, 0, 0};
        for (int r = 0; r <= p; ++r) {
            const double* c = ctrl + 4 * (s - p + r);
            Cw[0] += N[r] * c[3] * c[0];
            Cw[1] += N[r] * c[3] * c[1];
            Cw[2] += N[r] * c[3] * c[2];
            Cw[3] += N[r] * c[3];
        }
        out[3 * a + 0] = Cw[0] / Cw[3];
        out[3 * a + 1] = Cw[1] / Cw[3];
        out[3 * a + 2] = Cw[2] / Cw[3];
    }
}

void nurbs_oracle_curve_vjp_sigma(int p, int n1, const double* U, const double* ctrl,
                                  int nu, const double* u, const double* g, double* dctrl, double* dU,
                                  double sigma)
{
    int nU = n1 + p + 1;
    if (dctrl) memset(dctrl, 0, sizeof(double) * 4 * (size_t)n1);
    if (dU) memset(dU, 0, sizeof(double) * nU);
    double N[OR_MAXDEG + 1], dN[(OR_MAXDEG + 1) * (2 * OR_MAXDEG + 2)];
    for (int a = 0; a < nu; ++a) {
        int s = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        int base = 0, kw = knot_jacobian(s, u[a], p, U, sigma, N, dN, &base);
        double NR[3] = {0, 0, 0}, W = 0;
        for (int r = 0; r <= p; ++r) {
            const double* c = ctrl + 4 * (s - p + r);
            double bw = N[r] * c[3];
            NR[0] += bw * c[0]; NR[1] += bw * c[1]; NR[2] += bw * c[2];
            W += bw;
        }
        const double* ga = g + 3 * a;
        for (int r = 0; r <= p; ++r) {
            const double* c = ctrl + 4 * (s - p + r);
            if (dctrl) {
                double R = N[r] * c[3] / W;
                double* d = dctrl + 4 * (s - p + r);
                d[0] += R * ga[0]; d[1] += R * ga[1]; d[2] += R * ga[2];
                double sw = 0;
                for (int c3 = 0; c3 < 3; ++c3)
                    sw += (N[r] * c[c3] * W - NR[c3] * N[r]) / (W * W) * ga[c3];
                d[3] += sw;
            }
            if (dU) {
                double coef = 0;
                for (int c3 = 0; c3 < 3; ++c3)
                    coef += (c[3] * c[c3] / W - NR[c3] * c[3] / (W * W)) * ga[c3];
                for (int k = 0; k < kw; ++k)
                    dU[base + k] += coef * dN[r * kw + k];
            }
        }
    }
    if (dU) for (int k = 0; k < nU; ++k) if (k < p + 1 || k > n1 - 1) dU[k] = 0.0;
}

void nurbs_oracle_curve_vjp(int p, int n1, const double* U, const double* ctrl,
                            int nu, const double* u, const double* g, double* dctrl, double* dU)
{
    nurbs_oracle_curve_vjp_sigma(p, n1, U, ctrl, nu, u, g, dctrl, dU, 0.0);
}

/* ---------------------------------------------------------------------------
 * Gradients with respect to the homogeneous control points Pw = (w x, w y, w z, w)
 * (the optional parameterisation of the library).  S = NR / W with NR and W
 * linear in Pw (Eq. 3 written homogeneously), so
 *   dS/dPw.xyz_ij = N_i N_j / W (identity on xyz),  dS/dPw.w_ij = -N_i N_j S / W.
 * dpw[i][j][4] = (dL/dPw.x, dL/dPw.y, dL/dPw.z, dL/dPw.w).
 */
void nurbs_oracle_surface_vjp_homog(int p, int q, int n1, int m1, const double* U, const double* V,
                                    const double* ctrl, int nu, const double* u, int nv, const double* v,
                                    const double* g, double* dpw)
{
    memset(dpw, 0, sizeof(double) * 4 * (size_t)n1 * m1);
    double Nu[OR_MAXDEG + 1], Nv[OR_MAXDEG + 1];
    for (int a = 0; a < nu; ++a) {
        int su = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        nurbs_oracle_basis_funs(su, u[a], p, U, Nu);
        for (int b = 0; b < nv; ++b) {
            int sv = nurbs_oracle_find_span(m1 - 1, q, v[b], V);
            nurbs_oracle_basis_funs(sv, v[b], q, V, Nv);
            double NR[3] = {0, 0, 0}, W = 0;
            for (int r = 0; r <= p; ++r)
                for (int h = 0; h <= q; ++h) {
                    const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                    double bw = Nu[r] * Nv[h] * c[3];
                    NR[0] += bw * c[0]; NR[1] += bw * c[1]; NR[2] += bw * c[2];
                    W += bw;
                }
            const double* ga = g + 3 * ((size_t)a * nv + b);
            double Sg = (NR[0] * ga[0] + NR[1] * ga[1] + NR[2] * ga[2]) / W;
            for (int r = 0; r <= p; ++r)
                for (int h = 0; h <= q; ++h) {
                    double* d = dpw + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                    double NN = Nu[r] * Nv[h];
                    d[0] += NN * ga[0] / W;
                    d[1] += NN * ga[1] / W;
                    d[2] += NN * ga[2] / W;
                    d[3] -= NN * Sg / W;
                }
        }
    }
}

void nurbs_oracle_curve_vjp_homog(int p, int n1, const double* U, const double* ctrl,
                                  int nu, const double* u, const double* g, double* dpw)
{
    memset(dpw, 0, sizeof(double) * 4 * (size_t)n1);
    double N[OR_MAXDEG + 1];
    for (int a = 0; a < nu; ++a) {
        int s = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        nurbs_oracle_basis_funs(s, u[a], p, U, N);
        double NR[3] = {0, 0, 0}, W = 0;
        for (int r = 0; r <= p; ++r) {
            const double* c = ctrl + 4 * (s - p + r);
            double bw = N[r] * c[3];
            NR[0] += bw * c[0]; NR[1] += bw * c[1]; NR[2] += bw * c[2];
            W += bw;
        }
        const double* ga = g + 3 * a;
        double Sg = (NR[0] * ga[0] + NR[1] * ga[1] + NR[2] * ga[2]) / W;
        for (int r = 0; r <= p; ++r) {
            double* d = dpw + 4 * (s - p + r);
            d[0] += N[r] * ga[0] / W;
            d[1] += N[r] * ga[1] / W;
            d[2] += N[r] * ga[2] / W;
            d[3] -= N[r] * Sg / W;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Parametric derivatives (the u-derivative of Eq. 4, for the surface tangents
 * and normals the paper's offsetting application uses, Sec. 3.1 and Sec. 4).
 *
 * d/du N_i^p(u) = p N_i^{p-1}(u) / (U_{i+p} - U_i) - p N_{i+1}^{p-1}(u) / (U_{i+p+1} - U_{i+1}),
 * a term with a zero denominator taken as 0.  The degree p-1 functions come from
 * nurbs_oracle_basis_funs on the same span (those of other indices vanish on it).
 * dN[r] = dN_{span-p+r}(u) / du, r = 0..p.
 * ------------------------------------------------------------------------- */
void nurbs_oracle_basis_ders(int span, double u, int p, const double* U, double* dN)
{
    if (p == 0) {
        dN[0] = 0.0;
        return;
    }
    double Nm1[OR_MAXDEG + 1];
    nurbs_oracle_basis_funs(span, u, p - 1, U, Nm1);   /* N^{p-1}_{span-p+1 .. span} */
    for (int r = 0; r <= p; ++r) {
        int i = span - p + r;
        double left = (r >= 1) ? Nm1[r - 1] : 0.0;    /* N^{p-1}_i */
        double right = (r <= p - 1) ? Nm1[r] : 0.0;   /* N^{p-1}_{i+1} */
        double d1 = U[i + p] - U[i], d2 = U[i + p + 1] - U[i + 1];
        double a = (d1 != 0.0) ? p * left / d1 : 0.0;
        double b = (d2 != 0.0) ? p * right / d2 : 0.0;
        dN[r] = a - b;
    }
}

/* Rational derivative of the quotient S = A / W: S' = (A' - W' S) / W. */
static void rational_deriv(const double* A, double W, const double* Ad, double Wd, const double* S, double* out)
{
    for (int c = 0; c < 3; ++c) out[c] = (Ad[c] - Wd * S[c]) / W;
    (void)A;
}

/* Surface points, tangents S_u, S_v and unit normals (S_u x S_v normalised; a zero
 * cross product gives a zero normal).  Each output may be NULL; layout [a][b][3]. */
void nurbs_oracle_surface_derivs(int p, int q, int n1, int m1, const double* U, const double* V,
                                 const double* ctrl, int nu, const double* u, int nv, const double* v,
                                 double* out_S, double* out_Su, double* out_Sv, double* out_N)
{
    for (int a = 0; a < nu; ++a) {
        double Nu[OR_MAXDEG + 1], dNu[OR_MAXDEG + 1];
        int su = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        nurbs_oracle_basis_funs(su, u[a], p, U, Nu);
        nurbs_oracle_basis_ders(su, u[a], p, U, dNu);
        for (int b = 0; b < nv; ++b) {
            double Nv[OR_MAXDEG + 1], dNv[OR_MAXDEG + 1];
            int sv = nurbs_oracle_find_span(m1 - 1, q, v[b], V);
            nurbs_oracle_basis_funs(sv, v[b], q, V, Nv);
            nurbs_oracle_basis_ders(sv, v[b], q, V, dNv);
            double A[3] = {0, 0, 0}, Au[3] = {0, 0, 0}, Av[3] = {0, 0, 0}, W = 0, Wu = 0, Wv = 0;
            for (int r = 0; r <= p; ++r)
                for (int h = 0; h <= q; ++h) {
                    const double* c = ctrl + 4 * ((size_t)(su - p + r) * m1 + (sv - q + h));
                    double w = c[3];
                    for (int k = 0; k < 3; ++k) {
                        A[k] += Nu[r] * Nv[h] * w * c[k];
                        Au[k] += dNu[r] * Nv[h] * w * c[k];
                        Av[k] += Nu[r] * dNv[h] * w * c[k];
                    }
                    W += Nu[r] * Nv[h] * w;
                    Wu += dNu[r] * Nv[h] * w;
                    Wv += Nu[r] * dNv[h] * w;
                }
            double S[3] = {A[0] / W, A[1] / W, A[2] / W}, Su[3], Sv[3];
            rational_deriv(A, W, Au, Wu, S, Su);
            rational_deriv(A, W, Av, Wv, S, Sv);
            size_t o = 3 * ((size_t)a * nv + b);
            for (int k = 0; k < 3; ++k) {
                if (out_S) out_S[o + k] = S[k];
                if (out_Su) out_Su[o + k] = Su[k];
                if (out_Sv) out_Sv[o + k] = Sv[k];
            }
            if (out_N) {
                double n[3] = {Su[1] * Sv[2] - Su[2] * Sv[1], Su[2] * Sv[0] - Su[0] * Sv[2],
                               Su[0] * Sv[1] - Su[1] * Sv[0]};
                double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                for (int k = 0; k < 3; ++k) out_N[o + k] = len > 0.0 ? n[k] / len : 0.0;
            }
        }
    }
}

/* Curve points and tangents C'(u); either output may be NULL; layout [a][3]. */
void nurbs_oracle_curve_derivs(int p, int n1, const double* U, const double* ctrl, int nu, const double* u,
                               double* out_C, double* out_Cu)
{
    for (int a = 0; a < nu; ++a) {
        double N[OR_MAXDEG + 1], dN[OR_MAXDEG + 1];
        int s = nurbs_oracle_find_span(n1 - 1, p, u[a], U);
        nurbs_oracle_basis_funs(s, u[a], p, U, N);
        nurbs_oracle_basis_ders(s, u[a], p, U, dN);
        double A[3] = {0, 0, 0}, Ad[3] = {0, 0, 0}, W = 0, Wd = 0;
        for (int r = 0; r <= p; ++r) {
            const double* c = ctrl + 4 * (s - p + r);
            for (int k = 0; k < 3; ++k) {
                A[k] += N[r] * c[3] * c[k];
                Ad[k] += dN[r] * c[3] * c[k];
            }
            W += N[r] * c[3];
            Wd += dN[r] * c[3];
        }
        double C[3] = {A[0] / W, A[1] / W, A[2] / W}, Cu[3];
        rational_deriv(A, W, Ad, Wd, C, Cu);
        for (int k = 0; k < 3; ++k) {
            if (out_C) out_C[3 * a + k] = C[k];
            if (out_Cu) out_Cu[3 * a + k] = Cu[k];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Mean squared error between evaluated points and a target (the L2 loss of
 * Sec. 4 read as a mean of squared coordinate differences):
 *   L = sum (S - T)^2 / count,  g = 2 (S - T) / count.
 * Returns L; g may be NULL.
 * ------------------------------------------------------------------------- */
double nurbs_oracle_mse(size_t nvals, const double* S, const double* T, double count, double* g)
{
    double acc = 0.0;
    for (size_t k = 0; k < nvals; ++k) {
        double d = S[k] - T[k];
        acc += d * d;
        if (g) g[k] = 2.0 * d / count;
    }
    return acc / count;
}

/* ---------------------------------------------------------------------------
 * One Adam step (Kingma & Ba, with bias correction; the optimiser of Sec. 4):
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2
 *   theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 * step t starts at 1.
 * ------------------------------------------------------------------------- */
void nurbs_oracle_adam(size_t n, double* theta, const double* g, double* m, double* v,
                       int t, double lr, double b1, double b2, double eps)
{
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    for (size_t k = 0; k < n; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        double mhat = m[k] / bc1, vhat = v[k] / bc2;
        theta[k] -= lr * mhat / (sqrt(vhat) + eps);
    }
}
