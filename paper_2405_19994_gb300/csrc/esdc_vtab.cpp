// The gate functions of the ionic models tabulated in V (host side).
//
// Each gate q has w_inf,q(V) and Lambda_q(V), smooth functions of the
// membrane potential alone:
//   SYN19 (12 gates): w_inf,q(V) = 1/(1 + e^{-(V - Vh_q)/k_q}),
//                     Lambda_q(V) = -r_q exp(ln rho_q / (1 + e^{-(V - Vr_q)/sr_q}));
//   HH1952 (3 gates): Lambda = -(alpha + beta), w_inf = alpha/(alpha + beta)
//                     with the 1952 rates at v = V - V_rest.
// Evaluated directly a SYN19 gate costs three exponentials and two
// reciprocals (about 35 FP64 operations), an HH gate about as much; on a GPU
// with two FP64 lane operations per SM and clock that is most of the node
// kernel.  Here each function is replaced, on each interval
// [V_lo + i w, V_lo + (i+1) w) of width w = 1 mV, by its Chebyshev interpolant
// of degree 8 (9 Chebyshev points, values in long double), written as a
// polynomial in t = V - V_mid,i: 8 FMAs per function.  On the model's
// parameter ranges (slopes k, sr of 4 mV and more) the interpolation error of
// degree 8 over 1 mV is below 1e-15 of the function's magnitude; the table is
// checked at build time against the direct long-double values at 17 points
// per interval and refused (the kernels then evaluate directly) if the FP64
// Horner evaluation misses them by more than ESDC_VTAB_TOL.  The oracle keeps
// the direct formulas; the table is a way of computing the same functions.
//
// Row i of the table (ESDC_VTAB_ROW doubles): V_mid,i, a zero pad, then for
// each gate q the 9 coefficient pairs (w_inf,q, Lambda_q) of t^0, ..., t^8.
#include <cmath>
#include <vector>

#include "esdc_internal.h"

namespace {

using LD = long double;

LD logistic(LD x) { return 1.0L / (1.0L + expl(-x)); }

LD x_over_expm1(LD x) { return x == 0.0L ? 1.0L : x / expm1l(x); }

// alpha, beta of HH gate q (0 = m, 1 = h, 2 = n) at v = V - V_rest (mV, 1/ms).
void hh_rates(int q, LD v, LD& al, LD& be)
{
    if (q == 0) { al = x_over_expm1((25.0L - v) / 10.0L); be = 4.0L * expl(-v / 18.0L); }
    else if (q == 1) { al = 0.07L * expl(-v / 20.0L); be = 1.0L / (expl((30.0L - v) / 10.0L) + 1.0L); }
    else { al = 0.1L * x_over_expm1((10.0L - v) / 10.0L); be = 0.125L * expl(-v / 80.0L); }
}

// Chebyshev interpolant of f on [m - h, m + h] at d + 1 Chebyshev points,
// returned as monomial coefficients in t = V - m.
template <class F>
void cheb_monomial(F f, LD m, LD h, int d, LD* out)
{
    const int n = d + 1;
    std::vector<LD> fx(n), a(n, 0.0L);
    const LD pi = 3.14159265358979323846264338327950288L;
    for (int j = 0; j < n; ++j) fx[j] = f(m + h * cosl(pi * (j + 0.5L) / n));
    for (int k = 0; k < n; ++k) {
        LD s = 0.0L;
        for (int j = 0; j < n; ++j) s += fx[j] * cosl(pi * k * (j + 0.5L) / n);
        a[k] = (k == 0 ? 1.0L : 2.0L) * s / n;
    }
    // sum_k a_k T_k(tau) in powers of tau (T_{k+1} = 2 tau T_k - T_{k-1}), then tau = t/h
    std::vector<LD> tkm(n, 0.0L), tk(n, 0.0L), b(n, 0.0L);
    tkm[0] = 1.0L;                       // T_0 = 1
    tk[1] = 1.0L;                        // T_1 = tau (n >= 2)
    b[0] = a[0];
    b[1] = a[1];
    for (int k = 2; k < n; ++k) {
        std::vector<LD> tn(n, 0.0L);
        for (int p = 0; p < n; ++p) {
            if (p + 1 < n) tn[p + 1] += 2.0L * tk[p];
            tn[p] -= tkm[p];
        }
        for (int p = 0; p < n; ++p) b[p] += a[k] * tn[p];
        tkm = tk;
        tk = tn;
    }
    LD s = 1.0L;
    for (int p = 0; p < n; ++p) {
        out[p] = b[p] * s;
        s /= h;
    }
}

// Horner's rule on every second entry of c (the interleaved pairs), as the
// kernels evaluate it.
double horner2(const double* c, int n, double t)
{
    double r = c[2 * (n - 1)];
    for (int k = n - 2; k >= 0; --k) r = std::fma(r, t, c[2 * k]);
    return r;
}

}  // namespace

int esdc_vtab_build(int model, const double* params, std::vector<double>& rows, double* err_winf, double* err_lam)
{
    rows.clear();
    if (model != ESDC_MODEL_SYN19 && model != ESDC_MODEL_HH1952) return -1;
    const int NC = ESDC_VTAB_NC, d = NC - 1, NG = model == ESDC_MODEL_SYN19 ? 12 : 3;
    rows.assign((size_t)ESDC_VTAB_N * ESDC_VTAB_ROW, 0.0);
    double ew = 0.0, el = 0.0;
    LD coef[ESDC_VTAB_NC];
    for (int i = 0; i < ESDC_VTAB_N; ++i) {
        const LD lo = (LD)ESDC_VTAB_VLO + (LD)i * ESDC_VTAB_W;
        const LD h = 0.5L * ESDC_VTAB_W, mid = lo + h;
        double* row = rows.data() + (size_t)i * ESDC_VTAB_ROW;
        row[0] = (double)mid;                         // exact: multiples of 1/2 mV
        for (int q = 0; q < NG; ++q) {
            const bool syn = model == ESDC_MODEL_SYN19;
            const double* p = params + (syn ? 6 * q : 0);     // SYN19: Vh, k, r, ln rho, Vr, sr
            const LD Vrest = syn ? 0.0L : (LD)params[6];
            auto winf = [&](LD V) {
                if (syn) return logistic((V - (LD)p[0]) / (LD)p[1]);
                LD al, be;
                hh_rates(q, V - Vrest, al, be);
                return al / (al + be);
            };
            auto lam = [&](LD V) {
                if (syn) return -(LD)p[2] * expl((LD)p[3] * logistic((V - (LD)p[4]) / (LD)p[5]));
                LD al, be;
                hh_rates(q, V - Vrest, al, be);
                return -(al + be);
            };
            double* cw = row + 2 + q * 2 * NC;             // w_inf at even, Lambda at odd offsets
            double* cl = cw + 1;
            cheb_monomial(winf, mid, h, d, coef);
            for (int c = 0; c < NC; ++c) cw[2 * c] = (double)coef[c];
            cheb_monomial(lam, mid, h, d, coef);
            for (int c = 0; c < NC; ++c) cl[2 * c] = (double)coef[c];
            for (int s = 0; s <= 16; ++s) {           // the FP64 evaluation against the direct values
                const double V = (double)(lo + (LD)ESDC_VTAB_W * s / 16.0L);
                const double t = V - row[0];
                const LD w0 = winf((LD)V), l0 = lam((LD)V);
                ew = std::fmax(ew, (double)fabsl((LD)horner2(cw, NC, t) - w0));
                el = std::fmax(el, (double)(fabsl((LD)horner2(cl, NC, t) - l0) / fabsl(l0)));
            }
        }
    }
    if (err_winf) *err_winf = ew;
    if (err_lam) *err_lam = el;
    if (!(ew <= ESDC_VTAB_TOL) || !(el <= ESDC_VTAB_TOL)) {
        rows.clear();
        return -2;
    }
    return 0;
}
