/*
 * orc_space.c -- space discretisation and linear solves for the HSDC oracle
 * (test infrastructure only; see esdc_oracle.h).
 *
 * Mesh: uniform cell-centred grid with nx*ny*nz nodes, node index
 * p = ix + nx*(iy + ny*iz).  The Laplacian is the 3-/5-/7-point stencil with
 * mirror ghosts (zero normal flux, eq. (monodomain) boundary condition):
 *   (L v)_p = (1/h^2) sum_{q in nbr(p)} (v_q - v_p).
 * The paper uses fourth-order differences (Sec. 2.2) and solves with DCT-II
 * (Sec. 5); the second-order stencil is the default reading (it is also
 * diagonalised by DCT-II, so the paper's solver applies to it unchanged).
 * orc_mono.order = 4 selects the fourth-order five-point differences per
 * axis, with the ghost cells mirrored about the boundary faces; DCT-II
 * diagonalises that operator too.
 *
 * The layered anisotropic operator (orc_conductivity) keeps the same flux form:
 * the in-plane cross term sigma_xy V_xy uses the four diagonal neighbours, each
 * with weight a b sigma_xy/(2 h^2), and terms of absent neighbours are dropped,
 * so the matrix stays symmetric with zero row sums (reading of the conormal
 * zero-flux condition; checked by dense eigenvalues in the tests).
 *
 * Solvers for (I - g L) x = b:
 *   ORC_SOLVE_DCT   exact: orthonormal DCT-II along each axis, divide by the
 *                   eigenvalues 1 - g sum_axes mu_k, mu_k = -(4/h^2) sin^2(pi k/(2n)),
 *                   transform back (the paper's solver, Sec. 5).
 *   ORC_SOLVE_CG    textbook conjugate gradients from the given initial guess.
 *   ORC_SOLVE_DENSE dense matrix + Cholesky (tiny meshes only).
 */
#include "esdc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t mesh_n(const orc_mono* m) { return (int64_t)m->nx * m->ny * m->nz; }

/* Index of the cell that a (possibly ghost) index j of an axis of n cells
 * mirrors: reflection about the outer faces, repeated while outside. */
static int mirror(int j, int n)
{
    while (j < 0 || j >= n) j = j < 0 ? -j - 1 : 2 * n - 1 - j;
    return j;
}

/* (-v_{i-2} + 16 v_{i-1} - 30 v_i + 16 v_{i+1} - v_{i+2}) along one axis (axes of one cell contribute 0). */
static double axis4(const double* v, int64_t p, int i, int n, int64_t stride)
{
    if (n == 1) return 0.0;
    const double a = v[p + (int64_t)(mirror(i - 2, n) - i) * stride], b = v[p + (int64_t)(mirror(i - 1, n) - i) * stride];
    const double c = v[p + (int64_t)(mirror(i + 1, n) - i) * stride], d = v[p + (int64_t)(mirror(i + 2, n) - i) * stride];
    return -a + 16.0 * b - 30.0 * v[p] + 16.0 * c - d;
}

void orc_laplacian(const orc_mono* m, const double* v, double* out)
{
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    const double ih2 = 1.0 / (m->h * m->h);
    if (m->order == 4) {
        const int64_t sy = nx, sz = (int64_t)nx * ny;
        #pragma omp parallel for schedule(static)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    int64_t p = ix + sy * iy + sz * iz;
                    out[p] = (axis4(v, p, ix, nx, 1) + axis4(v, p, iy, ny, sy) + axis4(v, p, iz, nz, sz)) * ih2 / 12.0;
                }
        return;
    }
    #pragma omp parallel for schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t p = ix + (int64_t)nx * (iy + (int64_t)ny * iz);
                double s = 0.0;
                if (ix > 0)      s += v[p - 1] - v[p];
                if (ix < nx - 1) s += v[p + 1] - v[p];
                if (iy > 0)      s += v[p - nx] - v[p];
                if (iy < ny - 1) s += v[p + nx] - v[p];
                if (iz > 0)      s += v[p - (int64_t)nx * ny] - v[p];
                if (iz < nz - 1) s += v[p + (int64_t)nx * ny] - v[p];
                out[p] = s * ih2;
            }
}

static int is_layered(const orc_mono* m) { return m->lay_sxx != NULL; }
static int is_field(const orc_mono* m) { return m->sig_node != NULL; }

void orc_conductivity(const orc_mono* m, const double* v, double* out)
{
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    const int64_t N = mesh_n(m);
    const double ih2 = 1.0 / (m->h * m->h);
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    if (is_field(m)) {
        const double* sg = m->sig_node;
        #pragma omp parallel for schedule(static)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    int64_t p = ix + sy * iy + sz * iz;
                    double s = 0.0;
                    if (ix > 0)      s += 0.5 * (sg[p] + sg[p - 1]) * (v[p - 1] - v[p]);
                    if (ix < nx - 1) s += 0.5 * (sg[p] + sg[p + 1]) * (v[p + 1] - v[p]);
                    if (iy > 0)      s += 0.5 * (sg[p] + sg[p - sy]) * (v[p - sy] - v[p]);
                    if (iy < ny - 1) s += 0.5 * (sg[p] + sg[p + sy]) * (v[p + sy] - v[p]);
                    if (iz > 0)      s += 0.5 * (sg[p] + sg[p - sz]) * (v[p - sz] - v[p]);
                    if (iz < nz - 1) s += 0.5 * (sg[p] + sg[p + sz]) * (v[p + sz] - v[p]);
                    out[p] = s * ih2;
                }
        return;
    }
    if (!is_layered(m)) {
        orc_laplacian(m, v, out);
        for (int64_t p = 0; p < N; ++p) out[p] *= m->sigma;
        return;
    }
    #pragma omp parallel for schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t p = ix + sy * iy + sz * iz;
                double s = 0.0;
                const double sxx = m->lay_sxx[iz], syy = m->lay_syy[iz], sxy = m->lay_sxy[iz];
                if (ix > 0)      s += sxx * (v[p - 1] - v[p]);
                if (ix < nx - 1) s += sxx * (v[p + 1] - v[p]);
                if (iy > 0)      s += syy * (v[p - sy] - v[p]);
                if (iy < ny - 1) s += syy * (v[p + sy] - v[p]);
                if (iz > 0)      s += 0.5 * (m->lay_szz[iz] + m->lay_szz[iz - 1]) * (v[p - sz] - v[p]);
                if (iz < nz - 1) s += 0.5 * (m->lay_szz[iz] + m->lay_szz[iz + 1]) * (v[p + sz] - v[p]);
                for (int a = -1; a <= 1; a += 2)
                    for (int b = -1; b <= 1; b += 2)
                        if (ix + a >= 0 && ix + a < nx && iy + b >= 0 && iy + b < ny)
                            s += 0.5 * sxy * a * b * (v[p + a + sy * b] - v[p]);
                out[p] = s * ih2;
            }
}

/* ---------- DCT-II solve ---------- */

/* Orthonormal DCT-II matrix T[k*n + i] = s_k cos(pi k (i + 1/2) / n). */
static double* dct_matrix(int n)
{
    double* T = malloc(sizeof(double) * n * n);
    for (int k = 0; k < n; ++k) {
        double s = (k == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
        for (int i = 0; i < n; ++i) T[k * n + i] = s * cos(M_PI * k * (i + 0.5) / n);
    }
    return T;
}

/* Apply T (transpose = 0) or T^T (transpose = 1) along one axis of a
 * nx*ny*nz array. stride = distance between consecutive entries of a line. */
static void dct_axis(const orc_mono* m, int axis, int transpose, const double* T, double* a)
{
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    int n = axis == 0 ? nx : axis == 1 ? ny : nz;
    if (n == 1) return;
    int64_t stride = axis == 0 ? 1 : axis == 1 ? nx : (int64_t)nx * ny;
    int64_t nlines = mesh_n(m) / n;
    #pragma omp parallel
    {
        double* in = malloc(sizeof(double) * n);
        #pragma omp for schedule(static)
        for (int64_t l = 0; l < nlines; ++l) {
            /* line start: enumerate the indices orthogonal to the axis */
            int64_t base;
            if (axis == 0) base = l * nx;
            else if (axis == 1) base = (l % nx) + (l / nx) * (int64_t)nx * ny;
            else base = l;
            for (int i = 0; i < n; ++i) in[i] = a[base + i * stride];
            for (int k = 0; k < n; ++k) {
                double s = 0.0;
                if (!transpose) for (int i = 0; i < n; ++i) s += T[k * n + i] * in[i];
                else            for (int i = 0; i < n; ++i) s += T[i * n + k] * in[i];
                a[base + k * stride] = s;
            }
        }
        free(in);
    }
}

/* Eigenvalue of the 1D operator on cosine mode k of n cells, theta = pi k / n:
 * order 2: -(4/h^2) sin^2(theta/2); order 4: (32 cos theta - 2 cos 2 theta - 30)/(12 h^2)
 * (the stencil's symbol; the mirrored extension of a cosine mode is the mode itself). */
static double axis_eig(int order, int k, int n, double h2)
{
    if (n == 1) return 0.0;
    const double th = M_PI * k / n;
    if (order == 4) return (32.0 * cos(th) - 2.0 * cos(2.0 * th) - 30.0) / (12.0 * h2);
    const double s = sin(0.5 * th);
    return -(4.0 / h2) * s * s;
}

static int solve_dct(const orc_mono* m, double g, const double* b, double* x)
{
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    const int64_t N = mesh_n(m);
    double* Tx = dct_matrix(nx);
    double* Ty = dct_matrix(ny);
    double* Tz = dct_matrix(nz);
    memcpy(x, b, sizeof(double) * N);
    dct_axis(m, 0, 0, Tx, x);
    dct_axis(m, 1, 0, Ty, x);
    dct_axis(m, 2, 0, Tz, x);
    const double h2 = m->h * m->h;
    for (int iz = 0; iz < nz; ++iz) {
        const double mz = axis_eig(m->order, iz, nz, h2);
        for (int iy = 0; iy < ny; ++iy) {
            const double my = axis_eig(m->order, iy, ny, h2);
            for (int ix = 0; ix < nx; ++ix) {
                double mu = axis_eig(m->order, ix, nx, h2) + my + mz;
                x[ix + (int64_t)nx * (iy + (int64_t)ny * iz)] /= (1.0 - g * mu);
            }
        }
    }
    dct_axis(m, 0, 1, Tx, x);
    dct_axis(m, 1, 1, Ty, x);
    dct_axis(m, 2, 1, Tz, x);
    free(Tx); free(Ty); free(Tz);
    return 0;
}

/* ---------- conjugate gradients ---------- */

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* out = v - g L v (use_A = 0) or v - g A v (use_A = 1) */
static void apply_shifted_op(const orc_mono* m, int use_A, double g, const double* v, double* out)
{
    if (use_A) orc_conductivity(m, v, out);
    else orc_laplacian(m, v, out);
    const int64_t N = mesh_n(m);
    for (int64_t i = 0; i < N; ++i) out[i] = v[i] - g * out[i];
}

static void apply_shifted(const orc_mono* m, double g, const double* v, double* out)
{
    apply_shifted_op(m, 0, g, v, out);
}

static int solve_cg_op(const orc_mono* m, int use_A, double g, const double* b, double* x);

static int solve_cg(const orc_mono* m, double g, const double* b, double* x)
{
    return solve_cg_op(m, 0, g, b, x);
}

static int solve_cg_op(const orc_mono* m, int use_A, double g, const double* b, double* x)
{
    const int64_t N = mesh_n(m);
    double* r = malloc(sizeof(double) * N);
    double* p = malloc(sizeof(double) * N);
    double* q = malloc(sizeof(double) * N);
    apply_shifted_op(m, use_A, g, x, q);
    for (int64_t i = 0; i < N; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rr = dot(N, r, r), bb = dot(N, b, b);
    double tol2 = m->cg_tol * m->cg_tol * bb;
    int it = 0, ok = (rr <= tol2);
    while (!ok && it < m->cg_maxit) {
        apply_shifted_op(m, use_A, g, p, q);
        double alpha = rr / dot(N, p, q);
        for (int64_t i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rr_new = dot(N, r, r);
        ++it;
        if (rr_new <= tol2) { ok = 1; break; }
        double beta = rr_new / rr;
        rr = rr_new;
        for (int64_t i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
    }
    free(r); free(p); free(q);
    return ok ? 0 : -1;
}

/* ---------- dense Cholesky (tiny meshes) ---------- */

typedef struct { double g; int use_A; double* Lf; } dense_fac;
typedef struct { int nf; dense_fac f[16]; } dense_cache;

static double* dense_factor(const orc_mono* m, int use_A, double g)
{
    const int64_t N = mesh_n(m);
    double* A = calloc((size_t)(N * N), sizeof(double));
    double* e = calloc((size_t)N, sizeof(double));
    double* col = malloc(sizeof(double) * N);
    for (int64_t j = 0; j < N; ++j) {          /* column j = (I - g L) e_j */
        e[j] = 1.0;
        apply_shifted_op(m, use_A, g, e, col);
        for (int64_t i = 0; i < N; ++i) A[i * N + j] = col[i];
        e[j] = 0.0;
    }
    /* in-place lower Cholesky */
    for (int64_t j = 0; j < N; ++j) {
        double s = A[j * N + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * N + k] * A[j * N + k];
        if (s <= 0.0) { free(A); A = NULL; break; }
        double ljj = sqrt(s);
        A[j * N + j] = ljj;
        for (int64_t i = j + 1; i < N; ++i) {
            double t = A[i * N + j];
            for (int64_t k = 0; k < j; ++k) t -= A[i * N + k] * A[j * N + k];
            A[i * N + j] = t / ljj;
        }
    }
    free(e); free(col);
    return A;
}

static int solve_dense(orc_mono* m, int use_A, double g, const double* b, double* x)
{
    const int64_t N = mesh_n(m);
    if (N > 2048) return -2;
    dense_cache* dc = m->work;
    if (!dc) { dc = calloc(1, sizeof(dense_cache)); m->work = dc; }
    double* Lf = NULL;
    for (int i = 0; i < dc->nf; ++i) if (dc->f[i].g == g && dc->f[i].use_A == use_A) Lf = dc->f[i].Lf;
    if (!Lf) {
        Lf = dense_factor(m, use_A, g);
        if (!Lf) return -3;
        if (dc->nf < 16) { dc->f[dc->nf].g = g; dc->f[dc->nf].use_A = use_A; dc->f[dc->nf].Lf = Lf; dc->nf++; }
    }
    for (int64_t i = 0; i < N; ++i) {           /* L y = b */
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= Lf[i * N + k] * x[k];
        x[i] = s / Lf[i * N + i];
    }
    for (int64_t i = N - 1; i >= 0; --i) {      /* L^T x = y */
        double s = x[i];
        for (int64_t k = i + 1; k < N; ++k) s -= Lf[k * N + i] * x[k];
        x[i] = s / Lf[i * N + i];
    }
    int cached = 0;
    for (int i = 0; i < dc->nf; ++i) if (dc->f[i].Lf == Lf) cached = 1;
    if (!cached) free(Lf);
    return 0;
}

int orc_solve_shifted(const orc_mono* m, int method, double g, const double* b, double* x)
{
    if (method == ORC_SOLVE_DCT) return solve_dct(m, g, b, x);
    if (method == ORC_SOLVE_CG) return solve_cg(m, g, b, x);
    if (method == ORC_SOLVE_DENSE) return solve_dense((orc_mono*)m, 0, g, b, x);
    return -1;
}

int orc_solve_A(const orc_mono* m, int method, double g, const double* b, double* x)
{
    if (!is_layered(m) && !is_field(m)) return orc_solve_shifted(m, method, g * m->sigma, b, x);
    if (method == ORC_SOLVE_DENSE) return solve_dense((orc_mono*)m, 1, g, b, x);
    return solve_cg_op(m, 1, g, b, x);
}

void orc_mono_free(orc_mono* m)
{
    dense_cache* dc = m->work;
    if (dc) {
        for (int i = 0; i < dc->nf; ++i) free(dc->f[i].Lf);
        free(dc);
    }
    m->work = NULL;
}
