// The set-up's exponential coefficients tabulated in z (host side).
//
// For each gate the set-up computes, from z = dt Lambda_n (App. A):
//   dt S_ij(z) = dt (a_ij(z) - a_{i-1,j}(z)),  a_ij(z) = sum_k B_ijk phi_k(c_i z),
//   dt d_i phi_1(d_i z),
// i, j = 1..M: M (M + 1) functions of z alone for given M and dt.  Evaluated
// directly they cost about 200 FP64 operations per gate (phi_1..phi_M at the M
// points c_i z by series or recurrence, phi_1 at d_i z, the M^3 contraction).
// Here each function is replaced by polynomial pieces in y = 1 - z on a
// floating-point-like grid: octave e (2^e <= y < 2^(e+1), e < ESDC_ZTAB_OCT)
// is cut into 2^ESDC_ZTAB_SUB equal intervals, so the interval of y is read off
// its exponent and leading mantissa bits (integer work).  The phi functions are
// entire and their n-th derivatives fall like |z|^-(n+1) for large |z|, so the
// interpolation error is about the same in every octave.  On each interval
// every function is its Chebyshev interpolant of degree ESDC_ZTAB_NC - 1
// (values in long double), stored as a polynomial in t = y - y_mid.  Beyond
// the last octave (|z| >= 2^ESDC_ZTAB_OCT - 1) the kernels evaluate directly.
//
// phi_k(x), x <= 0, in long double: for |x| <= 32 the series
//   phi_k(x) = e^x / (k-1)! sum_m (-x)^m / (m! (m + k))
// (phi_k(x) = int_0^1 e^{(1-s)x} s^{k-1}/(k-1)! ds with e^{-sx} expanded; all
// terms positive, no cancellation); beyond, phi_1 = (e^x - 1)/x and the
// forward recurrence phi_{k+1} = (phi_k - 1/k!)/x, whose error shrinks by
// k/|x| < 1 per step there.
//
// The table is checked when it is built: the FP64 Horner evaluation against
// the long-double functions at 9 points per interval, the error measured in
// units of dt (a_ij and phi_1 are of order one).  A table that misses by more
// than ESDC_ZTAB_TOL is refused and the kernels evaluate directly.  Measured
// (the error does not depend on dt; checked from 1e-3 to 10 ms): degree 4 on
// 256 intervals per octave, at most 1.2e-16 for M = 4 and 2.0e-15 for M = 8;
// degree 3 on 512 intervals per octave misses the tolerance; degree 3 on 1024
// (12 octaves, 12288 rows, the table in use), at most 6.6e-16 for M = 4 and
// 2.0e-15 over M = 1..8.  On the synthetic slab the set-up went from 2.90 ms
// per step (direct) to 1.16 (degree 4) and 0.94 ms (degree 3).
//
// Row r of the table (ESDC_ZTAB_ROW(M) doubles): y_mid, a zero pad, then for
// i = 0..M-1 the function dt d_{i+1} phi_1 and the M functions dt S_{i+1,j},
// ESDC_ZTAB_NC coefficients each, lowest power first.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "esdc_internal.h"

namespace {

using LD = long double;

// phi_1 .. phi_M at x <= 0 (see above).
void phi_ld(int M, LD x, LD* ph)
{
    const LD ax = -x;
    if (ax <= 32.0L) {
        const LD ex = expl(x);
        LD fact = 1.0L;                                   // (k-1)!
        for (int k = 1; k <= M; ++k) {
            if (k > 1) fact *= (LD)(k - 1);
            LD term = 1.0L, s = 1.0L / (LD)k;             // m = 0
            for (int m = 1; m < 400; ++m) {
                term *= ax / (LD)m;                       // (-x)^m / m!
                const LD add = term / (LD)(m + k);
                s += add;
                if (add < s * 1e-40L) break;
            }
            ph[k - 1] = ex * s / fact;
        }
        return;
    }
    ph[0] = expm1l(x) / x;
    LD fact = 1.0L;                                       // k!
    for (int k = 1; k < M; ++k) {
        fact *= (LD)k;
        ph[k] = (ph[k - 1] - 1.0L / fact) / x;
    }
}

// Chebyshev interpolant of f on [m - h, m + h] at d + 1 Chebyshev points, as
// monomial coefficients in t = y - m.  f fills all nf function values at y.
template <class F>
void cheb_fit(F f, int nf, LD m, LD h, int d, std::vector<LD>& out)
{
    const int n = d + 1;
    const LD pi = 3.14159265358979323846264338327950288L;
    std::vector<LD> fx((size_t)n * nf), vals(nf);
    for (int j = 0; j < n; ++j) {
        f(m + h * cosl(pi * (j + 0.5L) / n), vals.data());
        for (int q = 0; q < nf; ++q) fx[(size_t)j * nf + q] = vals[q];
    }
    out.assign((size_t)nf * n, 0.0L);
    for (int q = 0; q < nf; ++q) {
        std::vector<LD> a(n, 0.0L);
        for (int k = 0; k < n; ++k) {
            LD s = 0.0L;
            for (int j = 0; j < n; ++j) s += fx[(size_t)j * nf + q] * cosl(pi * k * (j + 0.5L) / n);
            a[k] = (k == 0 ? 1.0L : 2.0L) * s / n;
        }
        // sum_k a_k T_k(tau) in powers of tau, then tau = t / h
        std::vector<LD> tkm(n, 0.0L), tk(n, 0.0L), b(n, 0.0L);
        tkm[0] = 1.0L;
        b[0] = a[0];
        if (n > 1) {
            tk[1] = 1.0L;
            b[1] = a[1];
        }
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
            out[(size_t)q * n + p] = b[p] * s;
            s /= h;
        }
    }
}

double horner(const double* c, int n, double t)
{
    double r = c[n - 1];
    for (int k = n - 2; k >= 0; --k) r = std::fma(r, t, c[k]);
    return r;
}

// The M (M + 1) functions of y = 1 - z, in row order (see above).
void functions(int M, const ColloData& C, LD dt, LD y, LD* out)
{
    const LD z = 1.0L - y;
    LD ph[ESDC_MMAX], ph1[1], aprev[ESDC_MMAX] = {};
    for (int i = 0; i < M; ++i) {
        phi_ld(1, (LD)C.d[i + 1] * z, ph1);
        out[i * (M + 1)] = dt * (LD)C.d[i + 1] * ph1[0];
        phi_ld(M, (LD)C.c[i + 1] * z, ph);
        for (int j = 0; j < M; ++j) {
            LD aij = 0.0L;
            for (int k = 0; k < M; ++k) aij += (LD)C.B[i][j][k] * ph[k];
            out[i * (M + 1) + 1 + j] = dt * (aij - aprev[j]);
            aprev[j] = aij;
        }
    }
}

void build_rows(int M, const ColloData& C, double dt, int r0, int r1, double* rows, double& err)
{
    const int NC = ESDC_ZTAB_NC, nf = M * (M + 1), row_len = ESDC_ZTAB_ROW(M);
    err = 0.0;
    std::vector<LD> coef, exact(nf);
    for (int r = r0; r < r1; ++r) {
        const int e = r >> ESDC_ZTAB_SUB, s = r & ((1 << ESDC_ZTAB_SUB) - 1);
        const LD w = ldexpl(1.0L, e - ESDC_ZTAB_SUB);     // interval width in octave e
        const LD lo = ldexpl(1.0L, e) + w * s, h = 0.5L * w, mid = lo + h;
        double* row = rows + (size_t)r * row_len;
        row[0] = (double)mid;                             // exact: a dyadic rational
        cheb_fit([&](LD y, LD* v) { functions(M, C, (LD)dt, y, v); }, nf, mid, h, NC - 1, coef);
        for (int q = 0; q < nf; ++q)
            for (int p = 0; p < NC; ++p) row[2 + q * NC + p] = (double)coef[(size_t)q * NC + p];
        for (int k = 0; k <= 8; ++k) {
            const double y = (double)(lo + w * k / 8.0L);
            functions(M, C, (LD)dt, (LD)y, exact.data());
            const double t = y - row[0];
            for (int q = 0; q < nf; ++q) {
                const LD got = (LD)horner(row + 2 + q * NC, NC, t);
                err = std::fmax(err, (double)(fabsl(got - exact[q]) / (LD)dt));
            }
        }
    }
}

struct Cached {
    int M;
    double dt;
    ColloData C;
    std::vector<double> rows;
    double err;
};
std::mutex g_mu;
std::vector<Cached> g_cache;          // most recent last
constexpr size_t kCacheSize = 8;

}  // namespace

int esdc_ztab_build(int M, double dt, const ColloData& C, std::vector<double>& rows, double* err_out)
{
    rows.clear();
    if (M < 1 || M > ESDC_MMAX || !(dt > 0.0) || !std::isfinite(dt)) return -1;
    double err = 0.0;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (size_t k = 0; k < g_cache.size(); ++k)
            if (g_cache[k].M == M && g_cache[k].dt == dt &&
                std::memcmp(&g_cache[k].C, &C, sizeof(ColloData)) == 0) {
                Cached c = g_cache[k];
                g_cache.erase(g_cache.begin() + (long)k);
                g_cache.push_back(c);
                rows = c.rows;
                err = c.err;
                hit = true;
                break;
            }
    }
    if (!hit) {
        const int nrow = ESDC_ZTAB_OCT << ESDC_ZTAB_SUB;
        rows.assign((size_t)nrow * ESDC_ZTAB_ROW(M), 0.0);
        unsigned nt = std::thread::hardware_concurrency();
        nt = std::max(1u, std::min(nt, 16u));
        std::vector<double> te(nt, 0.0);
        std::vector<std::thread> th;
        const int per = (nrow + (int)nt - 1) / (int)nt;
        for (unsigned t = 0; t < nt; ++t) {
            const int r0 = (int)t * per, r1 = std::min(nrow, r0 + per);
            if (r0 >= r1) break;
            th.emplace_back(build_rows, M, std::cref(C), dt, r0, r1, rows.data(), std::ref(te[t]));
        }
        for (auto& x : th) x.join();
        for (double v : te) err = std::fmax(err, v);
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_cache.size() >= kCacheSize) g_cache.erase(g_cache.begin());
        g_cache.push_back(Cached{M, dt, C, rows, err});
    }
    if (err_out) *err_out = err;
    if (!(err <= ESDC_ZTAB_TOL)) {
        rows.clear();
        return -2;
    }
    return 0;
}
