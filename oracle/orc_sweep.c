/*
 * orc_sweep.c -- the HSDC time step of the oracle (test infrastructure only;
 * see esdc_oracle.h), written in the paper's non-recursive form.
 *
 * For the step [t_n, t_n + dt] (Sec. 3.1):
 *   Lambda_n = Lambda(y_n), frozen for the whole step (eq. def_ode_esdc, the
 *              matrix of eq. def_C is A(dt Lambda_{n,0}) with y_{n,0} = y_n)
 *   g_n(y)   = f_I(y) + f_E(y) + f_e(y) + Lambda_n (y_n - y)          eq. (def_g)
 *   C_i(y)   = y_i - dt sum_{j=1..M} a_ij(dt Lambda_n) g_n(y_j)        eq. (def_C)
 *   P_i(y)   = y_i - dt sum_{j=1..i} d_j E_j(y)                        eq. (def_P)
 *   E_j(y)   = f_I(y_j) + f_E(y_{j-1})
 *              + phi_1(d_j dt Lambda_n) (f_e(y_{j-1}) + Lambda_n (y_n - y_{j-1}))
 * and the preconditioned Picard iteration  P(y^{k+1}) = (P - C)(y^k) + 1 (x) y_n
 * (eq. prec_picard) from y^0 = 1 (x) y_n, i.e. row by row
 *   y_i^{k+1} - dt d_i f_I(y_i^{k+1})
 *      = y_n + dt sum_j a_ij G_j^k + dt sum_{j<i} d_j (E_j^{k+1} - E_j^k)
 *        + dt d_i (E_i^{k+1} - f_I(y_i^{k+1}) - E_i^k),      G_j^k = g_n(y_j^k).
 * Each row is solved for y_i^{k+1} with the problem's implicit solve; rows are
 * taken in order i = 1..M because P is lower triangular.
 *
 * Time arguments (the paper drops t in eq. def_P): f_E inside E_j is taken at
 * t_{n,j-1} (the node it is evaluated at) and inside g_n(y_j) at t_{n,j}.
 * Residual (eq. def_C; Algorithm 1): r_i = y_n + dt sum_j a_ij G_j - y_i, and the
 * norm is the max norm (the paper does not name it), relative to
 * ||(y_{n,0},...,y_{n,M})||_inf.
 */
#include "esdc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP loops of the oracle use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ALLOC(n) ((double*)calloc((size_t)(n), sizeof(double)))

/* f_e(y) = Lambda(y) (y - y_inf(y))  (eq. def_fe) */
static void eval_fe(const orc_problem* P, const double* y, double* fe, double* lam, double* yinf)
{
    P->lam_yinf(P, y, lam, yinf);
    for (int64_t e = 0; e < P->n; ++e) fe[e] = lam[e] * (y[e] - yinf[e]);
}

/* G = g_n(t, y)  (eq. def_g) */
static void eval_g(const orc_problem* P, double t, const double* y, const double* yn,
                   const double* lam_n, double* G, double* t1, double* t2, double* t3)
{
    const int64_t n = P->n;
    P->f_I(P, y, G);
    P->f_E(P, t, y, t1);
    eval_fe(P, y, t2, t3, t3 + n);
    for (int64_t e = 0; e < n; ++e) G[e] += t1[e] + t2[e] + lam_n[e] * (yn[e] - y[e]);
}

/* Explicit part of E_j: f_E(t, u) + phi1_j (f_e(u) + Lambda_n (y_n - u)), u = y_{j-1}. */
static void eval_E_explicit(const orc_problem* P, double t, const double* u, const double* yn,
                            const double* lam_n, const double* phi1, double* out,
                            double* t1, double* t2, double* t3)
{
    const int64_t n = P->n;
    P->f_E(P, t, u, out);
    eval_fe(P, u, t1, t2, t3);
    for (int64_t e = 0; e < n; ++e) out[e] += phi1[e] * (t1[e] + lam_n[e] * (yn[e] - u[e]));
}

int orc_hsdc_step(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                  double t_n, double dt, const double* y_n, double* y_next,
                  double* colloc, double* resid, orc_stats* st)
{
    return orc_hsdc_step_from(P, M, K, tol, plain_sdc, t_n, dt, y_n, NULL, y_next, colloc, resid, st);
}

int orc_hsdc_step_from(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                       double t_n, double dt, const double* y_n, const double* colloc_in,
                       double* y_next, double* colloc, double* resid, orc_stats* st)
{
    return orc_hsdc_step_tau(P, M, K, tol, plain_sdc, t_n, dt, y_n, colloc_in, NULL, y_next, colloc, resid, st);
}

int orc_hsdc_step_tau(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                      double t_n, double dt, const double* y_n, const double* colloc_in, const double* tau,
                      double* y_next, double* colloc, double* resid, orc_stats* st)
{
    if (M < 1 || M > ORC_MMAX || K < 0 || !(dt > 0.0)) return -1;
    const int64_t n = P->n;
    double c[ORC_MMAX + 1], d[ORC_MMAX + 1], w[ORC_MMAX * ORC_MMAX], a0[ORC_MMAX * ORC_MMAX];
    if (orc_radau_nodes(M, c)) return -2;
    for (int i = 1; i <= M; ++i) d[i] = c[i] - c[i - 1];
    orc_fornberg_weights(M, c, w);
    orc_aij(M, c, w, 0.0, a0);
    { double tmp[ORC_MMAX]; orc_phi(0.0, 1, tmp); }   /* initialise the quadrature rule */

    double* lam_n = ALLOC(n);
    double* t1 = ALLOC(n); double* t2 = ALLOC(n); double* t3 = ALLOC(2 * n);
    P->lam_yinf(P, y_n, lam_n, t1);
    if (plain_sdc) memset(lam_n, 0, sizeof(double) * n);

    /* a_ij(dt Lambda_n) entrywise (Lambda_n is diagonal), a[(i*M + j) n + e] */
    double* a = ALLOC((int64_t)M * M * n);
    double* phi1 = ALLOC((int64_t)M * n);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t e = 0; e < n; ++e) {
        double ae[ORC_MMAX * ORC_MMAX];
        const double* src = a0;
        if (lam_n[e] != 0.0) { orc_aij(M, c, w, dt * lam_n[e], ae); src = ae; }
        for (int ij = 0; ij < M * M; ++ij) a[ij * n + e] = src[ij];
        for (int j = 1; j <= M; ++j) {
            double ph;
            orc_phi(d[j] * dt * lam_n[e], 1, &ph);
            phi1[(j - 1) * n + e] = ph;
        }
    }

    double* Y    = ALLOC((int64_t)(M + 1) * n);   /* y^k_{0..M}       */
    double* Yn   = ALLOC((int64_t)(M + 1) * n);   /* y^{k+1}_{0..M}   */
    double* G    = ALLOC((int64_t)M * n);         /* G^k_{1..M}       */
    double* E    = ALLOC((int64_t)M * n);         /* E^k_{1..M}       */
    double* En   = ALLOC((int64_t)M * n);         /* E^{k+1}_{1..M}   */
    double* Ex   = ALLOC(n);
    double* rhs  = ALLOC(n);
    double* fI   = ALLOC(n);
    double* R    = ALLOC((int64_t)M * n);
    int rc = 0;

    /* y^0 = 1 (x) y_n (eq. prec_picard), or the given iterate with y_{n,0} = y_n */
    for (int j = 0; j <= M; ++j)
        memcpy(Y + j * n, (j > 0 && colloc_in) ? colloc_in + (int64_t)(j - 1) * n : y_n, sizeof(double) * n);
    for (int j = 1; j <= M; ++j) {
        eval_g(P, t_n + c[j] * dt, Y + j * n, y_n, lam_n, G + (j - 1) * n, t1, t2, t3);
        eval_E_explicit(P, t_n + c[j - 1] * dt, Y + (j - 1) * n, y_n, lam_n, phi1 + (j - 1) * n,
                        E + (j - 1) * n, t1, t2, t3);
        P->f_I(P, Y + j * n, fI);
        for (int64_t e = 0; e < n; ++e) E[(j - 1) * n + e] += fI[e];
    }

    double res_inf = 0.0, y_inf = 0.0;
    int k = 0;
    for (k = 0; k < K; ++k) {
        memcpy(Yn, y_n, sizeof(double) * n);
        for (int i = 1; i <= M; ++i) {
            eval_E_explicit(P, t_n + c[i - 1] * dt, Yn + (i - 1) * n, y_n, lam_n,
                            phi1 + (i - 1) * n, Ex, t1, t2, t3);
            for (int64_t e = 0; e < n; ++e) {
                double s = 0.0;
                for (int j = 1; j <= M; ++j)
                    s += a[((i - 1) * M + (j - 1)) * n + e] * G[(j - 1) * n + e];
                double corr = 0.0;
                for (int j = 1; j < i; ++j)
                    corr += d[j] * (En[(j - 1) * n + e] - E[(j - 1) * n + e]);
                corr += d[i] * (Ex[e] - E[(i - 1) * n + e]);
                rhs[e] = y_n[e] + dt * s + dt * corr + (tau ? tau[(i - 1) * n + e] : 0.0);
            }
            double* yi = Yn + i * n;
            memcpy(yi, Y + i * n, sizeof(double) * n);            /* initial guess y_i^k */
            if (P->solve_I(P, dt * d[i], rhs, yi)) { rc = -3; goto done; }
            P->f_I(P, yi, fI);
            for (int64_t e = 0; e < n; ++e) En[(i - 1) * n + e] = fI[e] + Ex[e];
        }
        memcpy(Y, Yn, sizeof(double) * (M + 1) * n);
        memcpy(E, En, sizeof(double) * M * n);
        for (int j = 1; j <= M; ++j)
            eval_g(P, t_n + c[j] * dt, Y + j * n, y_n, lam_n, G + (j - 1) * n, t1, t2, t3);

        /* residual of the collocation system at y^{k+1} */
        res_inf = 0.0; y_inf = 0.0;
        for (int64_t e = 0; e < n; ++e) if (fabs(y_n[e]) > y_inf) y_inf = fabs(y_n[e]);
        for (int i = 1; i <= M; ++i)
            for (int64_t e = 0; e < n; ++e) {
                double s = 0.0;
                for (int j = 1; j <= M; ++j)
                    s += a[((i - 1) * M + (j - 1)) * n + e] * G[(j - 1) * n + e];
                double r = y_n[e] + dt * s - Y[i * n + e] + (tau ? tau[(i - 1) * n + e] : 0.0);
                R[(i - 1) * n + e] = r;
                if (fabs(r) > res_inf) res_inf = fabs(r);
                if (fabs(Y[i * n + e]) > y_inf) y_inf = fabs(Y[i * n + e]);
            }
        if (tol > 0.0 && res_inf < tol * y_inf) { ++k; break; }
    }
    if (K == 0) {
        for (int i = 1; i <= M; ++i)
            for (int64_t e = 0; e < n; ++e) {
                double s = 0.0;
                for (int j = 1; j <= M; ++j)
                    s += a[((i - 1) * M + (j - 1)) * n + e] * G[(j - 1) * n + e];
                R[(i - 1) * n + e] = y_n[e] + dt * s - Y[i * n + e] + (tau ? tau[(i - 1) * n + e] : 0.0);
            }
    }
    memcpy(y_next, Y + M * n, sizeof(double) * n);
    if (colloc) memcpy(colloc, Y + n, sizeof(double) * M * n);
    if (resid) memcpy(resid, R, sizeof(double) * M * n);
    if (st) { st->sweeps_done = k; st->res_inf = res_inf; st->y_inf = y_inf; st->solve_fail = 0; }
done:
    if (rc && st) st->solve_fail = 1;
    free(lam_n); free(t1); free(t2); free(t3); free(a); free(phi1);
    free(Y); free(Yn); free(G); free(E); free(En); free(Ex); free(rhs); free(fI); free(R);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Monodomain problem (eq. sd_sys, eq. def_monodomain_rhs)             */
/* ------------------------------------------------------------------ */
static int64_t mono_N(const orc_mono* m) { return (int64_t)m->nx * m->ny * m->nz; }

/* f_I = ((chi C_m)^{-1} A V, 0, 0) with A = div(sigma grad) (orc_conductivity) */
static void mono_fI(const orc_problem* P, const double* y, double* out)
{
    const orc_mono* m = P->ctx;
    const int64_t N = mono_N(m);
    memset(out, 0, sizeof(double) * P->n);
    orc_conductivity(m, y, out);
    const double s = 1.0 / (m->chi * m->Cm);
    for (int64_t p = 0; p < N; ++p) out[p] *= s;
}

static int mono_solve(const orc_problem* P, double gamma, const double* rhs, double* x)
{
    const orc_mono* m = P->ctx;
    const int64_t N = mono_N(m);
    memcpy(x + N, rhs + N, sizeof(double) * (P->n - N));   /* non-V rows: x = rhs */
    const double g = gamma / (m->chi * m->Cm);
    return orc_solve_A(m, m->solver, g, rhs, x);
}

static double stim_at(const orc_mono* m, double t, int ix, int iy, int iz)
{
    double s = 0.0;
    for (int b = 0; b < m->nbox; ++b) {
        const int* bx = m->box + 6 * b;
        if (t >= m->t_on[b] && t < m->t_off[b] &&
            ix >= bx[0] && ix < bx[1] && iy >= bx[2] && iy < bx[3] && iz >= bx[4] && iz < bx[5])
            s += m->amp[b];
    }
    return s;
}

/* f_E = (C_m^{-1}(I_stim - I_ion), h_a, 0) */
static void mono_fE(const orc_problem* P, double t, const double* y, double* out)
{
    const orc_mono* m = P->ctx;
    const int64_t N = mono_N(m);
    const int ns = orc_mono_nstate(m->model);
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        double u[19], fE[19], lam[19], yinf[19];
        for (int s = 0; s < ns; ++s) u[s] = y[s * N + p];
        int ix = (int)(p % m->nx), iy = (int)((p / m->nx) % m->ny), iz = (int)(p / ((int64_t)m->nx * m->ny));
        if (m->ionic_off) for (int s = 0; s < ns; ++s) fE[s] = 0.0;
        else orc_ionic_point(m->model, m->mp, u, fE, lam, yinf);
        out[p] = (stim_at(m, t, ix, iy, iz) + fE[0]) / m->Cm;
        for (int s = 1; s < ns; ++s) out[s * N + p] = fE[s];
    }
}

static void mono_lam_yinf(const orc_problem* P, const double* y, double* lam, double* yinf)
{
    const orc_mono* m = P->ctx;
    const int64_t N = mono_N(m);
    const int ns = orc_mono_nstate(m->model);
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        double u[19], fE[19], l[19], yi[19];
        for (int s = 0; s < ns; ++s) u[s] = y[s * N + p];
        if (m->ionic_off) for (int s = 0; s < ns; ++s) { l[s] = 0.0; yi[s] = 0.0; }
        else orc_ionic_point(m->model, m->mp, u, fE, l, yi);
        for (int s = 0; s < ns; ++s) { lam[s * N + p] = l[s]; yinf[s * N + p] = yi[s]; }
    }
}

int orc_mono_problem(orc_mono* m, orc_problem* P)
{
    if (m->dim < 1 || m->dim > 3 || m->nx < 1 || m->ny < 1 || m->nz < 1 || !(m->h > 0.0)) return -1;
    if (m->model != ORC_HH1952 && m->model != ORC_SYN19) return -1;
    if (m->n_mp < (m->model == ORC_HH1952 ? 7 : 88)) return -1;
    if (m->order != 0 && m->order != 2 && m->order != 4) return -1;
    if (m->order == 4 && (m->lay_sxx || m->sig_node)) return -1;   /* fourth order: scalar sigma only */
    P->n = mono_N(m) * orc_mono_nstate(m->model);
    P->ctx = m;
    P->f_I = mono_fI;
    P->solve_I = mono_solve;
    P->f_E = mono_fE;
    P->lam_yinf = mono_lam_yinf;
    return 0;
}

void orc_mono_init(const orc_mono* m, double V0, double* y)
{
    const int64_t N = mono_N(m);
    const int ns = orc_mono_nstate(m->model);
    double u[19];
    orc_ionic_rest(m->model, m->mp, V0, u);
    for (int s = 0; s < ns; ++s)
        for (int64_t p = 0; p < N; ++p) y[s * N + p] = u[s];
}

/* ------------------------------------------------------------------ */
/* Scalar test equation (Sec. 4, eq. test): f_I = lI y, f_E = lE y,     */
/* f_e = le y = Lambda (y - y_inf) with Lambda = le, y_inf = 0.          */
/* ------------------------------------------------------------------ */
typedef struct { double lI, lE, le; } scalar_ctx;

static void sc_fI(const orc_problem* P, const double* y, double* out)
{ const scalar_ctx* s = P->ctx; out[0] = s->lI * y[0]; }
static int sc_solve(const orc_problem* P, double gamma, const double* rhs, double* x)
{ const scalar_ctx* s = P->ctx; x[0] = rhs[0] / (1.0 - gamma * s->lI); return 0; }
static void sc_fE(const orc_problem* P, double t, const double* y, double* out)
{ (void)t; const scalar_ctx* s = P->ctx; out[0] = s->lE * y[0]; }
static void sc_lam(const orc_problem* P, const double* y, double* lam, double* yinf)
{ (void)y; const scalar_ctx* s = P->ctx; lam[0] = s->le; yinf[0] = 0.0; }

double orc_stability_R1(double lI, double lE, double le, int M, int K, double tol, int plain_sdc)
{
    scalar_ctx s = { lI, lE, le };
    orc_problem P = { 1, &s, sc_fI, sc_solve, sc_fE, sc_lam };
    double y0 = 1.0, y1 = NAN;
    orc_stats st;
    if (orc_hsdc_step(&P, M, K, tol, plain_sdc, 0.0, 1.0, &y0, &y1, NULL, NULL, &st)) return NAN;
    return y1;
}
