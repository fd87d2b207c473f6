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
// [V_lo + i w, V_lo + (i+1) w) of width w = ESDC_VTAB_W (1/128 mV), by its
// Chebyshev interpolant of degree ESDC_VTAB_NC - 1 (3: 4 Chebyshev points,
// values in long double), written as a polynomial in t = V - V_mid,i:
// ESDC_VTAB_NC - 1 FMAs per function.  The functions are analytic in a strip
// about the real axis of half-width about pi k (k, sr >= 4 mV on the models'
// parameter ranges), so the interpolation error falls like (w / (4 pi k))^NC:
// narrow intervals allow a low degree.  Measured (FP64 Horner against long
// double, 17 points per interval, SYN19): degree 8 on 1 mV, 7 on 1/2, 6 on
// 1/4, 5 on 1/8 and 4 on 1/32 mV all stay at the rounding floor (at most
// 4.0e-16 absolute for w_inf, 2.2e-16 relative for Lambda); 4 on 1/16 mV
// reaches 2.9e-15, 3 on 1/64 mV 7.6e-15 and 3 on 1/128 mV 5.4e-16.  Fewer
// FMAs per evaluation paid for more than the larger table (24 MB at degree 3,
// held in L2) cost: the headline node class went from 9.53 to 9.06, 8.59,
// 8.16, 7.28 and 6.93 ms per step along that series.  The table in use is
// checked at 9 points per interval.
// A table whose FP64 evaluation misses by more than ESDC_VTAB_TOL is refused
// (the kernels then evaluate directly).  The oracle keeps the direct
// formulas; the table is a way of computing the same functions.
//
// Row i of the table (ESDC_VTAB_ROW doubles): V_mid,i, a zero pad, then for
// each gate q the ESDC_VTAB_NC coefficient pairs (b_q, Lambda_q) of t^0, t^1,
// ..., with b_q = -Lambda_q w_inf,q (for HH, alpha_q).  The kernels need the
// gate's rate Lambda (u - w_inf) = Lambda u + b, one FMA from (Lambda, b);
// w_inf itself (diagnostics) is -b / Lambda.  The error check scales b's error
// by |Lambda|, which makes it the error in w_inf.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <thread>
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

// Rows [i0, i1) of the table; returns the largest errors of their FP64
// evaluation against the direct long-double values.
void build_rows(int model, const double* params, int i0, int i1, double* out, double& ew, double& el)
{
    const int NC = ESDC_VTAB_NC, d = NC - 1, NG = model == ESDC_MODEL_SYN19 ? 12 : 3;
    ew = 0.0;
    el = 0.0;
    LD coef[ESDC_VTAB_NC];
    for (int i = i0; i < i1; ++i) {
        const LD lo = (LD)ESDC_VTAB_VLO + (LD)i * ESDC_VTAB_W;
        const LD h = 0.5L * ESDC_VTAB_W, mid = lo + h;
        double* row = out + (size_t)i * ESDC_VTAB_ROW;
        row[0] = (double)mid;                         // exact: multiples of ESDC_VTAB_W / 2
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
            auto bfun = [&](LD V) { return -lam(V) * winf(V); };
            double* cb = row + 2 + q * 2 * NC;             // b at even, Lambda at odd offsets
            double* cl = cb + 1;
            cheb_monomial(bfun, mid, h, d, coef);
            for (int c = 0; c < NC; ++c) cb[2 * c] = (double)coef[c];
            cheb_monomial(lam, mid, h, d, coef);
            for (int c = 0; c < NC; ++c) cl[2 * c] = (double)coef[c];
            for (int s = 0; s <= 8; ++s) {            // the FP64 evaluation against the direct values
                const double V = (double)(lo + (LD)ESDC_VTAB_W * s / 8.0L);
                const double t = V - row[0];
                const LD l0 = lam((LD)V), b0 = -l0 * winf((LD)V);
                // b's error relative to |Lambda|: the error it makes in w_inf
                ew = std::fmax(ew, (double)(fabsl((LD)horner2(cb, NC, t) - b0) / fabsl(l0)));
                el = std::fmax(el, (double)(fabsl((LD)horner2(cl, NC, t) - l0) / fabsl(l0)));
            }
        }
    }
}

// Tables already built in this process, keyed by the model and the parameters
// the gate functions depend on (SYN19: the six of each gate; HH: V_rest), so
// that handles of the same model and a change of conductances reuse them.
struct Cached {
    int model;
    std::vector<double> key, rows;
    double ew, el;
};
std::mutex g_cache_mu;
std::vector<Cached> g_cache;            // most recent last, at most kCacheSize
constexpr size_t kCacheSize = 8;

}  // namespace

int esdc_vtab_build(int model, const double* params, std::vector<double>& rows, double* err_winf, double* err_lam)
{
    rows.clear();
    if (model != ESDC_MODEL_SYN19 && model != ESDC_MODEL_HH1952) return -1;
    const std::vector<double> key = model == ESDC_MODEL_SYN19 ? std::vector<double>(params, params + 72)
                                                               : std::vector<double>{params[6]};
    double ew = 0.0, el = 0.0;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (size_t k = 0; k < g_cache.size(); ++k)
            if (g_cache[k].model == model && g_cache[k].key == key) {
                Cached c = g_cache[k];
                g_cache.erase(g_cache.begin() + (long)k);
                g_cache.push_back(c);
                rows = c.rows;
                ew = c.ew;
                el = c.el;
                hit = true;
                break;
            }
    }
    if (!hit) {
        rows.assign((size_t)ESDC_VTAB_N * ESDC_VTAB_ROW, 0.0);
        // rows are independent: split them over the host's cores; the maxima
        // do not depend on the split
        unsigned nt = std::thread::hardware_concurrency();
        nt = std::max(1u, std::min(nt, 16u));
        std::vector<double> tw(nt, 0.0), tl(nt, 0.0);
        std::vector<std::thread> th;
        const int per = (ESDC_VTAB_N + (int)nt - 1) / (int)nt;
        for (unsigned t = 0; t < nt; ++t) {
            const int i0 = (int)t * per, i1 = std::min(ESDC_VTAB_N, i0 + per);
            if (i0 >= i1) break;
            th.emplace_back(build_rows, model, params, i0, i1, rows.data(), std::ref(tw[t]), std::ref(tl[t]));
        }
        for (auto& x : th) x.join();
        for (unsigned t = 0; t < nt; ++t) {
            ew = std::fmax(ew, tw[t]);
            el = std::fmax(el, tl[t]);
        }
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (g_cache.size() >= kCacheSize) g_cache.erase(g_cache.begin());
        g_cache.push_back(Cached{model, key, rows, ew, el});
    }
    if (err_winf) *err_winf = ew;
    if (err_lam) *err_lam = el;
    if (!(ew <= ESDC_VTAB_TOL) || !(el <= ESDC_VTAB_TOL)) {
        rows.clear();
        return -2;
    }
    return 0;
}
