/*
 * orc_colloc.c -- collocation data for the HSDC oracle (test infrastructure
 * only; see esdc_oracle.h).  Plain FP64 loops, no blocking or reordering.
 *
 *   - Radau IIA nodes (Sec. 3.1.2): the roots of P_M(2x-1) - P_{M-1}(2x-1) on
 *     (0,1], found by a sign-change scan plus bisection.
 *   - q_ij = int_0^{c_i} l_j(s) ds (eq. piN; a_ij(0), Sec. 3.1.2) by a
 *     Gauss-Legendre rule that is exact for the degree of l_j.
 *   - Fornberg weights (App. A, eq. fornberg), Fornberg's 1988 recursion.
 *   - phi_k(z) (App. A, eq. def_phik) by composite Gauss-Legendre quadrature,
 *     as the paper does, with panels graded toward the peak of e^{(1-r) z}.
 *   - a_ij(z) = sum_k c_i^k w_j^{k-1} phi_k(c_i z)  (App. A, eq. def_aij_computable).
 */
#include "esdc_oracle.h"
#include <math.h>
#include <string.h>

/* Legendre polynomial P_n(t) by the three-term recurrence. */
static double legendre(int n, double t)
{
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
    }
    return p1;
}

static double radau_poly(int M, double x)
{
    return legendre(M, 2.0 * x - 1.0) - legendre(M - 1, 2.0 * x - 1.0);
}

int orc_radau_nodes(int M, double* c)
{
    if (M < 1 || M > ORC_MMAX) return -1;
    c[0] = 0.0;
    c[M] = 1.0;                       /* x = 1 is always a root               */
    if (M == 1) return 0;
    /* The other M-1 roots lie in (0,1).  Scan for sign changes, then bisect. */
    const int nscan = 200000;
    int found = 0;
    double xa = 1e-12, fa = radau_poly(M, xa);
    for (int s = 1; s <= nscan && found < M - 1; ++s) {
        double xb = (double)s / (nscan + 1.0), fb = radau_poly(M, xb);
        if (fa == 0.0) { c[++found] = xa; }
        else if (fa * fb < 0.0) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), fm = radau_poly(M, mid);
                if (mid <= lo || mid >= hi) break;
                if (flo * fm <= 0.0) { hi = mid; } else { lo = mid; flo = fm; }
            }
            c[++found] = 0.5 * (lo + hi);
        }
        xa = xb; fa = fb;
    }
    return found == M - 1 ? 0 : -2;
}

void orc_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn = legendre(n, t), pn1 = legendre(n - 1, t);
            double dp = n * (t * pn - pn1) / (t * t - 1.0);   /* P_n'(t) */
            double dt = pn / dp;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        double pn1 = legendre(n - 1, t), pn = legendre(n, t);
        double dp = n * (t * pn - pn1) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* l_j(s) = prod_{k != j} (s - c_k)/(c_j - c_k)  (eq. piN), product form. */
static double lagrange(int M, const double* c, int j, double s)
{
    double p = 1.0;
    for (int k = 1; k <= M; ++k)
        if (k != j) p *= (s - c[k]) / (c[j] - c[k]);
    return p;
}

/* q_ij = int_0^{c_i} l_j(s) ds.  l_j has degree M-1, so a 16-point
 * Gauss-Legendre rule on [0, c_i] integrates it exactly (degree <= 31). */
void orc_collocation_q(int M, const double* c, double* q)
{
    enum { NG = 16 };
    double gx[NG], gw[NG];
    orc_gauss_legendre(NG, gx, gw);
    for (int i = 1; i <= M; ++i)
        for (int j = 1; j <= M; ++j) {
            double s = 0.0, half = 0.5 * c[i];
            for (int g = 0; g < NG; ++g) s += gw[g] * half * lagrange(M, c, j, half * (gx[g] + 1.0));
            q[(i - 1) * M + (j - 1)] = s;
        }
}

/*
 * Fornberg (1988): weights of the derivatives 0..M-1 at the point 0 of the
 * polynomial interpolating values at c_1..c_M.  The recursion adds one node
 * at a time; table C[node][order] holds the weights for the nodes added so
 * far.  Output w[k*M + (l-1)] = weight of p(c_l) in p^{(k)}(0).
 */
void orc_fornberg_weights(int M, const double* c, double* w)
{
    const double z = 0.0;
    double C[ORC_MMAX][ORC_MMAX];
    memset(C, 0, sizeof C);
    const double* x = c + 1;          /* nodes x[0..M-1] = c_1..c_M */
    int m = M - 1;                    /* highest derivative         */
    double prod_prev = 1.0;
    double dx_prev = x[0] - z;
    C[0][0] = 1.0;
    for (int i = 1; i < M; ++i) {
        int top = i < m ? i : m;
        double prod = 1.0;
        double dx_old = dx_prev;
        dx_prev = x[i] - z;
        for (int j = 0; j < i; ++j) {
            double gap = x[i] - x[j];
            prod *= gap;
            if (j == i - 1) {
                for (int k = top; k >= 1; --k)
                    C[i][k] = prod_prev * (k * C[i - 1][k - 1] - dx_old * C[i - 1][k]) / prod;
                C[i][0] = -prod_prev * dx_old * C[i - 1][0] / prod;
            }
            for (int k = top; k >= 1; --k)
                C[j][k] = (dx_prev * C[j][k] - k * C[j][k - 1]) / gap;
            C[j][0] = dx_prev * C[j][0] / gap;
        }
        prod_prev = prod;
    }
    for (int k = 0; k < M; ++k)
        for (int l = 0; l < M; ++l)
            w[k * M + l] = C[l][k];
}

/*
 * phi_k(z) = 1/(k-1)! int_0^1 e^{(1-r) z} r^{k-1} dr  (App. A).
 * Composite 16-point Gauss-Legendre.  With s = 1 - r the integrand is
 * e^{z s} (1-s)^{k-1}; for z < -2 it decays on the scale 1/|z| away from s=0,
 * so the panels in s are [0,1/|z|], [1/|z|,2/|z|], [2/|z|,4/|z|], ... (each
 * spans at most a doubling of the exponent) until s reaches 1 or the
 * exponent passes -800 (where e^{z s} underflows).
 */
void orc_phi(double z, int kmax, double* phi)
{
    enum { NG = 16 };
    static double gx[NG], gw[NG];
    static int init = 0;
    if (!init) { orc_gauss_legendre(NG, gx, gw); init = 1; }
    for (int k = 0; k < kmax; ++k) phi[k] = 0.0;
    if (z > 2.0) { for (int k = 0; k < kmax; ++k) phi[k] = NAN; return; }

    double edges[128];
    int ne = 0;
    edges[ne++] = 0.0;
    if (z >= -2.0) {
        edges[ne++] = 1.0;
    } else {
        double a = -z;                /* |z| */
        double s = 1.0 / a;
        edges[ne++] = s;
        while (s < 1.0 && a * s < 800.0 && ne < 127) {
            s = (2.0 * s < 1.0) ? 2.0 * s : 1.0;
            edges[ne++] = s;
        }
    }
    double fact[ORC_MMAX + 2];
    fact[0] = 1.0;
    for (int k = 1; k <= ORC_MMAX + 1; ++k) fact[k] = fact[k - 1] * k;

    for (int p = 0; p + 1 < ne; ++p) {
        double lo = edges[p], hi = edges[p + 1];
        double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        for (int g = 0; g < NG; ++g) {
            double s = mid + half * gx[g];
            double r = 1.0 - s;
            double e = exp(z * s) * half * gw[g];
            double rp = 1.0;          /* r^{k-1} */
            for (int k = 1; k <= kmax; ++k) {
                phi[k - 1] += e * rp / fact[k - 1];
                rp *= r;
            }
        }
    }
}

void orc_aij(int M, const double* c, const double* w, double z, double* a)
{
    double phi[ORC_MMAX];
    for (int i = 1; i <= M; ++i) {
        orc_phi(c[i] * z, M, phi);
        for (int j = 1; j <= M; ++j) {
            double s = 0.0, cik = c[i];
            for (int k = 1; k <= M; ++k) {
                s += cik * w[(k - 1) * M + (j - 1)] * phi[k - 1];
                cik *= c[i];
            }
            a[(i - 1) * M + (j - 1)] = s;
        }
    }
}
