/*
 * esdc_oracle.h -- plain, slow FP64 CPU oracle of the hybrid exponential /
 * semi-implicit SDC (HSDC, "ES-SDC") step for the semi-discrete monodomain
 * equation  y' = f_I(t,y) + f_E(t,y) + f_e(t,y)  (Sec. 1, eq. (1); Sec. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no source with the CUDA library (no headers, tables,
 * helpers or constants); both sides only receive the same seeded inputs.
 *
 * Everything here follows the paper's notation:
 *   c_0 = 0 < c_1 < ... < c_M = 1   Radau IIA nodes (Sec. 3.1.2)
 *   d_i = c_i - c_{i-1}
 *   a_ij(z) = int_0^{c_i} e^{(c_i - s) z} l_j(s) ds             eq. (def_aij)
 *           = sum_k c_i^k w_j^{k-1} phi_k(c_i z)                  App. A
 *   phi_k(z) = 1/(k-1)! int_0^1 e^{(1-r) z} r^{k-1} dr            App. A
 *   P(y^{k+1}) = (P - C)(y^k) + 1 (x) y_n                         eq. (prec_picard)
 *
 * Parity with the paper: the paper prints no worked numerical example, so
 * every routine here is pinned by closed forms, invariants and brute force
 * (see tests/test_oracle_*.py), not by printed values.
 */
#ifndef ESDC_ORACLE_H
#define ESDC_ORACLE_H
#include <stdint.h>

#define ORC_MMAX 8          /* largest number of collocation nodes supported */

/* ------------------------------------------------------------------ */
/* Collocation data (Sec. 3.1.2, App. A)                               */
/* ------------------------------------------------------------------ */
/* Radau IIA (right) nodes c[0..M]; c[0] = 0, c[M] = 1.  Returns 0 on success. */
int    orc_radau_nodes(int M, double* c);
/* n-point Gauss-Legendre rule on [-1,1]. */
void   orc_gauss_legendre(int n, double* x, double* w);
/* q[(i-1)*M + (j-1)] = int_0^{c_i} l_j(s) ds, by a Gauss-Legendre rule exact
 * for polynomials of degree <= 31. */
void   orc_collocation_q(int M, const double* c, double* q);
/* Fornberg weights: w[k*M + (l-1)] with p^{(k)}(0) = sum_l w^k_l p(c_l),
 * k = 0..M-1 (eq. (fornberg)). */
void   orc_fornberg_weights(int M, const double* c, double* w);
/* phi_k(z), k = 1..kmax, by composite Gauss-Legendre quadrature of the
 * integral definition (App. A, eq. (def_phik)).  Requires z <= 2. */
void   orc_phi(double z, int kmax, double* phi /* [kmax], phi[k-1] = phi_k */);
/* a_ij(z), i,j = 1..M, out[(i-1)*M + (j-1)] (App. A, eq. (def_aij_computable)). */
void   orc_aij(int M, const double* c, const double* w, double z, double* a);

/* ------------------------------------------------------------------ */
/* Generic problem y' = f_I + f_E + f_e with f_I linear (Sec. 1)       */
/* ------------------------------------------------------------------ */
typedef struct orc_problem orc_problem;
struct orc_problem {
    int64_t n;                     /* unknowns in y                          */
    void*   ctx;
    /* out = f_I(y) (linear in y)                                            */
    void (*f_I)(const orc_problem*, const double* y, double* out);
    /* solve x - gamma f_I(x) = rhs; x holds the initial guess on entry.    */
    int  (*solve_I)(const orc_problem*, double gamma, const double* rhs, double* x);
    /* out = f_E(t, y)                                                      */
    void (*f_E)(const orc_problem*, double t, const double* y, double* out);
    /* diagonal Lambda(y) and y_inf(y), f_e = Lambda (y - y_inf)  (eq. def_fe) */
    void (*lam_yinf)(const orc_problem*, const double* y, double* lam, double* yinf);
};

typedef struct {
    int    sweeps_done;            /* sweeps actually taken                   */
    double res_inf;                /* ||r||_inf over all collocation nodes    */
    double y_inf;                  /* ||y^k||_inf over collocation nodes 0..M */
    int    solve_fail;             /* non-zero if a linear solve failed       */
} orc_stats;

/*
 * One HSDC time step in the non-recursive preconditioned-Picard form
 * eq. (prec_picard) with P from eq. (def_P) and C from eq. (def_C):
 *   y_n   : [n] state at t_n;   y_next: [n] receives y_{n+1} = y_{n,M}^K
 *   K     : maximum sweeps; tol > 0 stops after the first sweep with
 *           ||r|| < tol ||y|| (Algorithm 1 stop test), tol <= 0 runs K sweeps
 *   plain_sdc != 0 replaces Lambda_n by 0 (the plain SDC of Sec. 4.2)
 *   colloc: optional [M*n] receives y_{n,1..M}^K; resid: optional [M*n]
 *   receives r_i = y_n + dt sum_j a_ij G_j - y_i (eq. def_C) at the final iterate.
 * Returns 0 on success, <0 on failure (bad arguments or a failed solve).
 */
int orc_hsdc_step(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                  double t_n, double dt, const double* y_n, double* y_next,
                  double* colloc, double* resid, orc_stats* st);

/* The same step started from a given iterate instead of y^0 = 1 (x) y_n:
 * colloc_in [M*n] holds y_{n,1..M}^0 (y_{n,0} = y_n).  G^0 and E^0 are
 * evaluated on that iterate with Lambda_n = Lambda(y_n), so the step is the
 * single-step sweep of eq. prec_picard applied to it.  One such sweep per
 * slice, with y_n the previous slice's last node, is the Q^par iteration of
 * eq. def_Q (Sec. 3.2).  colloc_in = NULL is orc_hsdc_step. */
int orc_hsdc_step_from(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                       double t_n, double dt, const double* y_n, const double* colloc_in,
                       double* y_next, double* colloc, double* resid, orc_stats* st);

/* The FAS form of the step (Sec. 3.2, Algorithm HSDC): a correction tau
 * [M*n] (rows 1..M; NULL = 0) is added to the right-hand side 1 (x) y_n of
 * the collocation system, so the sweeps solve P(y^{k+1}) = (P - C)(y^k) +
 * 1 (x) y_n + tau and the residual is r_i = y_n + tau_i + dt sum_j a_ij G_j - y_i. */
int orc_hsdc_step_tau(const orc_problem* P, int M, int K, double tol, int plain_sdc,
                      double t_n, double dt, const double* y_n, const double* colloc_in, const double* tau,
                      double* y_next, double* colloc, double* resid, orc_stats* st);

/* ------------------------------------------------------------------ */
/* Monodomain problem on a uniform cell-centred mesh (Sec. 2)          */
/* ------------------------------------------------------------------ */
enum { ORC_HH1952 = 0, ORC_SYN19 = 1 };
enum { ORC_SOLVE_DCT = 0, ORC_SOLVE_CG = 1, ORC_SOLVE_DENSE = 2 };

typedef struct {
    int    dim, nx, ny, nz;        /* dim 1, 2 or 3; unused extents = 1        */
    double h;                      /* mesh size [mm]                           */
    double sigma, chi, Cm;         /* [mS/mm], [1/mm], [uF/mm^2]               */
    int    model;                  /* ORC_HH1952 or ORC_SYN19                  */
    const double* mp; int n_mp;    /* ionic-model parameters                   */
    int    nbox;                   /* stimulus boxes                           */
    const int* box;                /* [nbox][6]: x0,x1,y0,y1,z0,z1 (half-open) */
    const double* amp;             /* [nbox] uA/mm^2                           */
    const double* t_on;            /* [nbox] ms                                */
    const double* t_off;           /* [nbox] ms, active on [t_on, t_off)       */
    int    solver;                 /* ORC_SOLVE_*                              */
    double cg_tol; int cg_maxit;   /* for ORC_SOLVE_CG                         */
    int    ionic_off;              /* 1: I_ion = 0, h_a = 0 (diffusion only)   */
    /* Layered anisotropic conductivity (NULL: isotropic sigma): per z-layer
     * tensor entries [nz] sigma_xx, sigma_yy, sigma_xy, sigma_zz (in-plane
     * fibres; sigma_xz = sigma_yz = 0). */
    const double *lay_sxx, *lay_syy, *lay_sxy, *lay_szz;
    /* Heterogeneous isotropic conductivity (NULL: sigma): one value per node,
     * [N] mS/mm; the flux through a face uses the mean of its two nodes. */
    const double* sig_node;
    /* Order of the Laplacian: 2 (3-/5-/7-point, default; 0 means 2) or 4
     * (the paper's fourth-order differences, Sec. 5: per axis
     * (-v_{i-2} + 16 v_{i-1} - 30 v_i + 16 v_{i+1} - v_{i+2}) / (12 h^2) with
     * mirrored ghost cells, repeated for axes shorter than the stencil).
     * Order 4 needs the scalar sigma. */
    int order;
    /* private workspace, owned by the oracle */
    void*  work;
} orc_mono;

int  orc_mono_nstate(int model);   /* 1 + m1 + m2 */
int  orc_mono_ngate(int model);    /* m2          */
/* Builds the generic problem view of a monodomain description. */
int  orc_mono_problem(orc_mono* m, orc_problem* P);
void orc_mono_free(orc_mono* m);
/* Rest-like initial state: V = V0 everywhere, gates at w_inf(V0), auxiliaries
 * at their V0 steady state (model defined). y: [n_state * N]. */
void orc_mono_init(const orc_mono* m, double V0, double* y);

/* Rest-like state of one node: V0, gates at w_inf(V0), auxiliaries at their
 * V0 steady state. u[n_state]. */
void orc_ionic_rest(int model, const double* mp, double V0, double* u);
/* Pointwise ionic model, one node: u[n_state] -> fE[n_state] = (-I_ion, h_a, 0)
 * (the caller forms (I_stim - I_ion)/C_m), lam[n_state], yinf[n_state]. */
void orc_ionic_point(int model, const double* mp, const double* u,
                     double* fE, double* lam, double* yinf);

/* Discrete Neumann Laplacian (cell-centred, mirror ghosts).  Order 2:
 * out = (1/h^2) sum_{q in nbr(p)} (v_q - v_p) (5-/7-point).  Order 4: the
 * five-point fourth-order difference along every axis (see orc_mono.order).
 * Both are diagonalised by DCT-II, so ORC_SOLVE_DCT is exact for both. (Sec. 2.2) */
void orc_laplacian(const orc_mono* m, const double* v, double* out);
/* Solve (I - g L) x = b with L the Laplacian above, by the chosen method. */
int  orc_solve_shifted(const orc_mono* m, int method, double g, const double* b, double* x);
/* The conductivity operator A = div(sigma grad) in flux form (conductivity
 * included): sigma L for an isotropic sigma; for a per-node field
 *   (A v)_p = (1/h^2) sum_{q in nbr(p)} (sigma_p + sigma_q)/2 (v_q - v_p);
 * for layered anisotropic sigma
 *   (A v)_p = (1/h^2) [ sum_x-faces sxx (v_q - v_p) + sum_y-faces syy (v_q - v_p)
 *                     + sum_z-faces (szz_k + szz_l)/2 (v_q - v_p)
 *                     + sum_{a,b = +-1} (a b sxy / 2) (v_{i+a,j+b} - v_p) ],
 * with terms of absent neighbours dropped (zero flux through boundary faces). */
void orc_conductivity(const orc_mono* m, const double* v, double* out);
/* Solve (I - g A) x = b.  Isotropic sigma: the chosen method on sigma L.
 * Layered sigma or a per-node field: CG or dense (a DCT request falls back
 * to CG). */
int  orc_solve_A(const orc_mono* m, int method, double g, const double* b, double* x);

/* ------------------------------------------------------------------ */
/* Scalar test equation y' = (lI + lE + le) y  (Sec. 4, eq. (test))    */
/* ------------------------------------------------------------------ */
/* Stability function R_1 after one step of size dt = 1 (L = 1, P = 1). */
double orc_stability_R1(double lI, double lE, double le, int M, int K, double tol,
                        int plain_sdc);

/* Threads used by the oracle's parallel loops. */
int orc_threads(void);

#endif
