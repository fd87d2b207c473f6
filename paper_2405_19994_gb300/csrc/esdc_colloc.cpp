// Host-side collocation data of the HSDC library (Sec. 3.1.2, App. A).
//
//  * Radau IIA nodes: c_M = 1 and the M-1 roots in (0,1) of
//    R(x) = P_M(2x-1) - P_{M-1}(2x-1), found together by the Aberth-Ehrlich
//    simultaneous Newton iteration (each root's Newton step is deflated by the
//    others, including the fixed root x = 1).
//  * w_j^k = k! [s^k] l_j(s): the Taylor coefficients at 0 of the Lagrange basis
//    polynomial l_j (eq. fornberg_ell), from its monomial expansion.  These are
//    the Fornberg weights of eq. (fornberg).
//  * B_ijk = c_i^k w_j^{k-1}, so that a_ij(z) = sum_k B_ijk phi_k(c_i z)
//    (eq. def_aij_computable), and a_ij(0) = sum_k B_ijk / k!.
//  * X1 / nser: the switch point and series length of the device phi_k
//    evaluation (see phi_all in esdc_step.cu).
#include <cmath>
#include <cstring>

#include "esdc_internal.h"

namespace {

// R(x) and R'(x) via the Legendre recurrences P_{k+1} = ((2k+1) t P_k - k P_{k-1})/(k+1),
// P'_{k+1} = P'_{k-1} + (2k+1) P_k, with t = 2x - 1 (dt/dx = 2).
void radau_poly(int M, double x, double* R, double* dR)
{
    double t = 2.0 * x - 1.0;
    double pm1 = 1.0, p = t;          // P_0, P_1
    double dpm1 = 0.0, dp = 1.0;      // P_0', P_1'
    if (M == 1) { *R = p - pm1; *dR = 2.0 * (dp - dpm1); return; }
    for (int k = 1; k < M; ++k) {
        double pn = ((2.0 * k + 1.0) * t * p - k * pm1) / (k + 1.0);
        double dpn = dpm1 + (2.0 * k + 1.0) * p;
        pm1 = p; p = pn;
        dpm1 = dp; dp = dpn;
    }
    *R = p - pm1;
    *dR = 2.0 * (dp - dpm1);
}

int radau_nodes(int M, double* c)
{
    c[0] = 0.0;
    c[M] = 1.0;
    int n = M - 1;
    if (n == 0) return 0;
    double x[ESDC_MMAX];
    for (int i = 0; i < n; ++i)
        x[i] = 0.5 * (1.0 - std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * M)));
    for (int it = 0; it < 500; ++it) {
        double maxstep = 0.0;
        for (int i = 0; i < n; ++i) {
            double R, dR;
            radau_poly(M, x[i], &R, &dR);
            if (R == 0.0) continue;
            double ratio = R / dR;
            double s = 1.0 / (x[i] - 1.0);          // deflate the known root x = 1
            for (int j = 0; j < n; ++j)
                if (j != i) s += 1.0 / (x[i] - x[j]);
            double step = ratio / (1.0 - ratio * s);
            x[i] -= step;
            maxstep = std::fmax(maxstep, std::fabs(step));
        }
        if (maxstep < 1e-17) break;
    }
    // sort ascending
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (x[j] < x[i]) { double t = x[i]; x[i] = x[j]; x[j] = t; }
    for (int i = 0; i < n; ++i) {
        if (!(x[i] > 0.0 && x[i] < 1.0)) return -1;
        if (i > 0 && !(x[i] > x[i - 1])) return -1;
        c[i + 1] = x[i];
    }
    return 0;
}

}  // namespace

int esdc_colloc_build(int M, ColloData* out)
{
    if (M < 1 || M > ESDC_MMAX) return -1;
    std::memset(out, 0, sizeof(*out));
    double* c = out->c;
    if (radau_nodes(M, c)) return -1;
    for (int i = 1; i <= M; ++i) out->d[i] = c[i] - c[i - 1];

    // monomial coefficients of l_j, then w_j^k = k! coef_k
    double w[ESDC_MMAX][ESDC_MMAX];   // w[j-1][k]
    for (int j = 1; j <= M; ++j) {
        double poly[ESDC_MMAX + 1] = {1.0};
        int deg = 0;
        double scale = 1.0;
        for (int m = 1; m <= M; ++m) {
            if (m == j) continue;
            // poly *= (s - c_m)
            poly[deg + 1] = 0.0;
            for (int e = deg + 1; e >= 1; --e) poly[e] = poly[e - 1] - c[m] * poly[e];
            poly[0] *= -c[m];
            ++deg;
            scale *= (c[j] - c[m]);
        }
        double fact = 1.0;
        for (int k = 0; k < M; ++k) {
            if (k > 0) fact *= k;
            w[j - 1][k] = fact * poly[k] / scale;
        }
    }
    for (int i = 1; i <= M; ++i)
        for (int j = 1; j <= M; ++j) {
            double cik = 1.0, a0 = 0.0, kf = 1.0;
            for (int k = 1; k <= M; ++k) {
                cik *= c[i];
                kf *= k;
                out->B[i - 1][j - 1][k - 1] = cik * w[j - 1][k - 1];
                a0 += cik * w[j - 1][k - 1] / kf;
            }
            out->A0[i - 1][j - 1] = a0;
        }
    for (int i = 1; i <= M; ++i)
        for (int j = 1; j <= M; ++j)
            out->S0[i - 1][j - 1] = out->A0[i - 1][j - 1] - (i > 1 ? out->A0[i - 2][j - 1] : 0.0);

    // phi_k switch: forward recurrence from phi_1 amplifies rounding by about
    // M!/|x|^{M-1}, the series + backward recurrence by |x|^{M-1}/(M-1)!;
    // X1 balances the two.  nser: terms until X1^n/n! < 2e-17.
    if (M == 1) { out->X1 = 0.0; out->nser = 0; }
    else {
        double f = 1.0;
        for (int k = 2; k < M; ++k) f *= k;
        out->X1 = std::pow(f * std::sqrt((double)M), 1.0 / (M - 1));
        double t = 1.0;
        int n = 0;
        while (t > 2e-17 || n < 4) { ++n; t *= out->X1 / n; }
        out->nser = n;
        if (out->nser + M >= ESDC_NSER) return -1;
        // ser[m] = 1/((M-1)! m! (m+M))
        double fm1 = 1.0;
        for (int k = 2; k < M; ++k) fm1 *= k;
        double mf = 1.0;
        for (int m = 0; m <= n; ++m) {
            if (m > 0) mf *= m;
            out->ser[m] = 1.0 / (fm1 * mf * (m + M));
        }
        // Truncating after term n leaves a relative tail below
        // X^{n+1} M / ((n+1)! (n+1+M)) (the sum is at least its first term).
        for (int l = 0; l < 5; ++l) {
            const double X = out->X1 / (double)(1 << (4 - l));
            int k = 0;
            double tail = X * M / (1.0 + M);       // n = 0
            while (tail > 1e-17 && k < out->nser) {
                ++k;
                tail *= X / (k + 1.0) * (k + M) / (k + 1.0 + M);
            }
            out->xb[l] = X;
            out->nb[l] = k;
        }
        out->nb[4] = out->nser;
    }
    return 0;
}
