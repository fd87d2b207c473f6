/*
 * esdc.h -- C ABI of the GB300 (sm_103a) HSDC / ES-SDC library for the
 * semi-discrete monodomain equation
 *
 *     y' = f_I(t,y) + f_E(t,y) + f_e(t,y),   f_e = Lambda(y) (y - y_inf(y))
 *
 * (arXiv 2405.19994, Sec. 1 eq. (1) and Sec. 2.2 eqs. (sd_sys), (def_f_IE),
 * (def_Lambda)).  One call of esdc_sweep advances one time step with the
 * hybrid SDC method: K sweeps of the preconditioned Picard iteration
 * P(y^{k+1}) = (P - C)(y^k) + 1 (x) y_n (Sec. 3.1.3, eq. (prec_picard)) with
 * the IMEX Rush-Larsen preconditioner P of eq. (def_P) and the exponential
 * collocation operator C of eq. (def_C), on M Radau IIA nodes.
 *
 * Conventions for every entry point:
 *   - Return value: ESDC_OK (0) on success, a negative ESDC_ERR_* code on
 *     failure.  No C++ exception crosses the ABI.  After a failure,
 *     esdc_last_error() returns a one-line description owned by the handle.
 *   - "device" pointers are CUDA device pointers on the device that was current
 *     when esdc_create was called; "host" pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it in order; calls that return data
 *     to host memory synchronise that stream before returning.
 *   - The caller owns every buffer it passes.  The handle owns its workspace,
 *     allocated once in esdc_create (sized for M <= options.M_max) and freed in
 *     esdc_destroy.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - State layout ("SoA"): y[s * ld + p] holds state s (0 = V_m [mV], then the
 *     m_1 auxiliary variables, then the m_2 gating variables) at mesh node
 *     p = ix + nx*(iy + ny*iz).  ld >= n_nodes is the row pitch returned by
 *     esdc_state_size (a multiple of 32 doubles); columns p >= n_nodes are
 *     ignored and left unchanged.
 *   - Units: mm, ms, mV, mS/mm (sigma), 1/mm (chi), uF/mm^2 (C_m), uA/mm^2.
 */
#ifndef ESDC_H
#define ESDC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESDC_OK                     0
#define ESDC_ERR_INVALID_ARG       -1   /* a null pointer, size or value out of range */
#define ESDC_ERR_CUDA              -2   /* a CUDA runtime call failed                  */
#define ESDC_ERR_CG_NOT_CONVERGED  -3   /* a diffusion solve hit cg_maxit              */
#define ESDC_ERR_NONFINITE         -4   /* NaN/Inf in the residual or the state        */
#define ESDC_ERR_DEVICE_TIMEOUT    -5   /* a bounded device-side wait gave up          */
#define ESDC_ERR_UNSUPPORTED       -6   /* valid but not implemented combination       */
#define ESDC_ERR_NO_MEMORY         -7   /* device allocation failed                    */
#define ESDC_ERR_TOO_LARGE         -8   /* mesh exceeds esdc_diffusion_solve_static's fixed scratch */

/* Ionic models (Sec. 5).  Parameters are passed explicitly to esdc_create:
 *  ESDC_MODEL_HH1952: Hodgkin-Huxley 1952, states (V, m, h, n) (m_1 = 0,
 *    m_2 = 3), 7 parameters [gNa, gK, gL, ENa, EK, EL, Vrest] (mS/mm^2, mV).
 *  ESDC_MODEL_SYN19: 19-state synthetic stiff model with the shape of ten
 *    Tusscher-Panfilov 2006 (m_1 = 6, m_2 = 12), 88 parameters: 12 gates x
 *    (Vh, k, r, ln rho, Vr, sr), then [G_f, E_f, G_s, E_s, G_K, E_K, G_K1,
 *    G_b, E_b, c_K6], then tau_1..tau_6. */
#define ESDC_MODEL_HH1952 0
#define ESDC_MODEL_SYN19  1

typedef struct esdc_handle esdc_handle;

/* Uniform cell-centred mesh of the rectangle/box Omega (Sec. 2.2, Sec. 5):
 * dim in {1,2,3}; extents nx, ny, nz >= 1 (ny = nz = 1 in 1D, nz = 1 in 2D);
 * h > 0 the mesh size.  A = sigma * L with L the 3/5/7-point Laplacian with
 * mirrored ghost nodes (zero normal flux, the boundary condition of
 * eq. (monodomain)). */
typedef struct {
    int    dim;
    int    nx, ny, nz;
    double h;
} esdc_mesh;

typedef struct {
    int    M_max;      /* largest M that esdc_sweep will be called with, 1..8      */
    double tol_cg;     /* relative 2-norm stop ||r|| <= tol_cg ||b|| of each solve */
    int    cg_maxit;   /* iteration cap of each solve (>= 1)                       */
    int    precond;    /* 1 = Jacobi-preconditioned CG, 0 = plain CG               */
    int    precision;  /* 0 = FP64 throughout; 1 = precision form: the ionic model
                          (f_E, Lambda, y_inf) evaluated in FP32, and each diffusion
                          solve done by iterative refinement (FP64 residuals
                          r = b - A x, FP32 inner solve of A e = r, x += e) to the
                          same tol_cg; state, coefficient tables, quadrature and
                          residual stay FP64                                       */
    int    solver;     /* diffusion solves of the sweep and esdc_diffusion_solve:
                          0 = automatic: with precision 0, the scalar sigma and
                          cheap transforms (esdc_get_solver) the DCT-II direct
                          solve of 2 (exact; the handle holds its tables from
                          esdc_create on), otherwise as 3;
                          3 = the Chebyshev semi-iteration on an
                          interval holding the spectrum of the operator of
                          esdc_diffusion_solve: for the scalar sigma exactly
                          [1, 1 + (g/h^2) sum_axes 4 sin^2(pi (n-1)/(2n))] (the
                          cosine modes are its eigenvectors) or the fourth-order
                          stencil's [1, 1 + (g/(12 h^2)) sum_axes (30 + 2 cos 2t
                          - 32 cos t)], t = pi (n-1)/n; for layers and a field
                          [1, 1 + g G] with G the Gershgorin bound of -A.  The
                          Jacobi-PCG runs only when g is too small for the
                          interval to have width in FP64.  With precision 1 and
                          nx a multiple of 4 the refinement's FP32 inner solves
                          are a fixed number of Chebyshev iterations
                          (2 q^k <= 1e-5), else PCG;
                          1 = the (Jacobi-P)CG always;
                          2 = the DCT-II direct solve, the paper's solver (Sec. 5):
                          x = C^T diag(1/(1 - g mu)) C b with C the orthonormal
                          3D DCT-II and mu the eigenvalues of the second- or
                          fourth-order stencil, computed by this library's own
                          kernels: a fast transform (FFT of pairs of lines,
                          O(n log n)) along axes of power-of-two length, a dense
                          product along other axes, and for the second-order
                          stencil a direct tridiagonal solve along z instead of
                          the z transform; exact, no iteration (iters reports 1).
                          Scalar sigma and precision 0 only (esdc_create returns
                          ESDC_ERR_UNSUPPORTED with precision 1; the conductivity
                          setters return it for layers or a field); holds the
                          axes' tables (dense axes: 2 n^2 doubles) and the
                          z-solve factors of up to M_max values of g (16 bytes
                          per node each).
                          Batches take 0, 1 or 3 (0 and 3 alike: Chebyshev).
                          1 and 3 stop at the same ||r|| <= tol_cg ||b||.  The
                          paper solves these systems with the DCT-II.            */
    int    fuse_node1; /* 1: node 1 of each sweep (its explicit rows need no
                          stencil) runs inside the launch (batches' persistent
                          step: the phase) before it, the set-up or the
                          previous sweep's final evaluation, for M >= 2 and not
                          while the adjoint records a step; 0: its own launch.
                          The results are the same bit for bit.                  */
} esdc_options;

/* Fills *opt with the defaults: M_max 8, tol_cg 1e-14, cg_maxit 200, precond 1,
 * precision 0, solver 0, fuse_node1 1. */
void esdc_default_options(esdc_options* opt);

/*
 * Creates a solver for the semi-discrete monodomain equation eq. (sd_sys) on
 * `mesh` with conductivity `sigma`, surface-to-volume ratio `chi` and membrane
 * capacitance `Cm` (eq. (monodomain)), and the ionic model `model` with
 * `n_params` host doubles `params` (copied).  `opt` may be NULL for defaults.
 * Allocates all device workspace on the current device.
 * Errors: INVALID_ARG (bad sizes/values/model/param count), NO_MEMORY, CUDA.
 * On failure *out is set to NULL.
 */
int esdc_create(const esdc_mesh* mesh, double sigma, double chi, double Cm,
                int model, const double* params, int n_params,
                const esdc_options* opt, esdc_handle** out);

/* Frees the handle and its device workspace (NULL is a no-op). */
void esdc_destroy(esdc_handle* h);

/* One-line description of the last error on this handle ("" if none). */
const char* esdc_last_error(const esdc_handle* h);

/*
 * Stimulus I_stim(t, x) of eq. (monodomain): a sum of boxes.  Box b adds
 * amp[b] uA/mm^2 at nodes ix in [box[6b], box[6b+1]), iy in [box[6b+2],
 * box[6b+3]), iz in [box[6b+4], box[6b+5]) while t_on[b] <= t < t_off[b].
 * All arrays are host memory, copied.  nbox = 0 removes the stimulus.
 * At most 16 boxes.  Errors: INVALID_ARG.
 */
int esdc_set_stimulus(esdc_handle* h, int nbox, const int* box, const double* amp,
                      const double* t_on, const double* t_off);

/*
 * Layered anisotropic conductivity: per z-layer tensor entries sigma_xx[k],
 * sigma_yy[k], sigma_xy[k], sigma_zz[k] (host arrays of length nz, mS/mm,
 * copied; sigma_xz = sigma_yz = 0, i.e. fibres in the xy-plane, e.g. rotating
 * through the depth).  Replaces the scalar sigma of esdc_create in f_I and in
 * the diffusion solves: A = div(sigma grad) in flux form, with the in-plane
 * cross term on the four diagonal neighbours (weight a b sigma_xy/(2h^2)) and
 * zero flux through boundary faces; z faces use the mean of the two layers'
 * sigma_zz.  Every layer must be positive definite.  All four pointers NULL
 * return to the scalar sigma.  Synchronises the device.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA.
 */
/*
 * Order of the Laplacian of f_I and of the diffusion solves: 2 (the default
 * 3-/5-/7-point cell-centred stencil) or 4, the fourth-order differences of
 * the paper's experiments (Sec. 5): along every axis
 * (-v_{i-2} + 16 v_{i-1} - 30 v_i + 16 v_{i+1} - v_{i+2}) / (12 h^2), ghost cells
 * mirrored about the boundary faces (zero flux; the operator stays symmetric
 * and is diagonalised by DCT-II).  Order 4 needs the scalar sigma and the FP64
 * path; its solves are the ones options.solver selects (DCT-II and Chebyshev
 * on the exact fourth-order spectrum; the CG with Jacobi weights from the
 * operator's diagonal).  Synchronises the device.
 * Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA.
 */
int esdc_set_stencil_order(esdc_handle* h, int order);

/*
 * The diffusion solver the handle's solves take now (options.solver resolved
 * against the mesh, the conductivity and the stencil order): *solver = 2 for
 * the DCT-II direct solve, 3 for the Chebyshev semi-iteration (with its CG
 * fallback when g is too small for the interval, and the precision form's
 * refinement), 1 for the CG.  The automatic choice (0) takes the DCT-II with
 * precision 0 and the scalar sigma while its transforms are cheap: every
 * transformed axis (x and y; z too for the fourth order) has power-of-two
 * length, except dense axes of total length at most 32.  Host only.
 * Errors: INVALID_ARG (null h or solver).
 */
int esdc_get_solver(const esdc_handle* h, int* solver);

/*
 * Heterogeneous isotropic conductivity: sigma[p] (host array of N values,
 * mS/mm, copied, all positive) at every mesh node.  Replaces the scalar sigma
 * (and any layers) in f_I and in the diffusion solves:
 *   (A v)_p = (1/h^2) sum_{q in nbr(p)} (sigma_p + sigma_q)/2 (v_q - v_p),
 * zero flux through boundary faces.  sigma = NULL returns to the scalar sigma.
 * FP64 path only (options.precision = 0).  Synchronises the device.
 * Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA.
 */
int esdc_set_conductivity_field(esdc_handle* h, const double* sigma);

int esdc_set_conductivity_layers(esdc_handle* h, const double* sxx, const double* syy,
                                 const double* sxy, const double* szz);

/* Reports the number of states per node (1 + m_1 + m_2), the number of mesh
 * nodes and the row pitch ld (in doubles) of a state buffer. */
int esdc_state_size(const esdc_handle* h, int* n_state, int64_t* n_nodes, int64_t* ld);

/*
 * Writes a resting state into the device buffer y [n_state][ld]: V = V0,
 * gates at w_inf(V0) (eq. monodomain_g_lambda), auxiliaries at the model's
 * V0 steady state.  Enqueued on `stream`.
 */
int esdc_init_state(esdc_handle* h, double* y, double V0, void* stream);

/*
 * One HSDC time step [t, t + dt] (Sec. 3.1): y (device [n_state][ld]) holds
 * y_n on entry and y_{n+1} = y_{n,M}^K on return (eq. (sys_erk_aij), c_M = 1).
 *   Lambda_n = Lambda(y_n) is frozen for the step (eq. (def_ode_esdc));
 *   the gate coefficients a_ij(dt Lambda_n) follow App. A eq.
 *   (def_aij_computable); y^0 = 1 (x) y_n; each sweep visits the nodes
 *   i = 1..M in order and solves (I - dt d_i (chi C_m)^{-1} A) V_i = rhs (the
 *   implicit f_I row of P) with the solver options.solver selects
 *   (esdc_get_solver); K >= 0 sweeps are taken.
 * After the sweeps the residual r_i = y_n + dt sum_j a_ij G_j - y_i of
 * eq. (def_C) is formed on the device (see esdc_residual).
 * 1 <= M <= M_max, dt > 0.  Work is enqueued on `stream`; the call does not
 * synchronise, except the first step with a new (M, dt): it builds the table
 * of the set-up's coefficients dt S_ij(z), dt d_i phi_1(d_i z) for them on the
 * host (cached per process) and synchronises the device once to upload it (a
 * handle keeps four such tables; a fifth (M, dt) replaces the oldest).  A
 * handle builds at most 16 tables: later new (M, dt), as with step sizes that
 * keep changing, and steps while `stream` is being captured into a CUDA graph
 * without the table, evaluate the coefficients directly (the same values
 * within a few units of 1e-16 dt).  Errors: INVALID_ARG, CUDA.  Convergence failures of the
 * solves are recorded on the device and reported by esdc_residual/esdc_stats.
 */
int esdc_sweep(esdc_handle* h, double* y, double t, double dt, int M, int K, void* stream);

/*
 * Same step with y in HOST memory (pitch ld_host >= n_nodes, layout as
 * above): copies y to the device, steps, and copies y_{n+1} back, all on
 * `stream`, then synchronises it.  For callers that keep the state on the host.
 */
int esdc_sweep_host(esdc_handle* h, double* y_host, int64_t ld_host, double t, double dt,
                    int M, int K, void* stream);

/*
 * Residual of the most recent esdc_sweep (Algorithm 1 stop test, Sec. 3.2):
 * res_inf = max_{i,s,p} |r_i|, y_inf = max over y_n and y_1..y_M of |y|
 * (the paper leaves the norm unnamed; this library uses the max norm).
 * res_state (host, optional, length n_state) receives the per-state maxima.
 * Synchronises the stream of that sweep.  Returns ESDC_ERR_NONFINITE if the
 * residual or the state is not finite, ESDC_ERR_CG_NOT_CONVERGED if a solve of
 * that step hit cg_maxit (the values are still written).
 */
int esdc_residual(esdc_handle* h, double* res_inf, double* y_inf, double* res_state);

/*
 * Iteration counts of the diffusion solves of the most recent esdc_sweep:
 * cg_iters (host, length >= K*M) receives the count of solve (k, i) at
 * index k*M + (i-1).  n = length of cg_iters.  Synchronises that stream.
 */
int esdc_stats(esdc_handle* h, int* cg_iters, int n);

/*
 * Copies the collocation iterate y_{n,1..M}^K of the most recent esdc_sweep
 * (device [M][n_state][ld]) and, if r_out != NULL, the residual vectors
 * r_1..r_M of eq. (def_C) (device [M][n_state][ld]; requires
 * esdc_keep_residual(h, 1) before that sweep) into caller buffers.
 */
int esdc_collocation(esdc_handle* h, double* y_out, double* r_out, void* stream);

/*
 * Kernel timing.  enable != 0 makes every later esdc_sweep record a CUDA event
 * pair on its stream around each launch of the four kernel classes of the step:
 * 0 = step set-up (Lambda_n, a_ij(dt Lambda_n), spread), 1 = sweep node kernel
 * (ionic model + quadrature), 2 = diffusion solve (CG), 3 = residual.
 * esdc_profile_read returns, per class, the summed milliseconds ms[4] and the
 * number of launches launches[4] since the last read, then resets them; it
 * synchronises the recorded events.  Not part of the method; no effect on results.
 */
int esdc_profile(esdc_handle* h, int enable);
int esdc_profile_read(esdc_handle* h, double* ms, long long* launches);

/*
 * keep != 0 makes every later esdc_sweep also store the residual vectors
 * r_1..r_M (allocates M_max*n_state*ld doubles); keep = 0 frees them.
 */
int esdc_keep_residual(esdc_handle* h, int keep);

/*
 * Exponential collocation coefficients (App. A eq. (def_aij_computable)):
 * for n values z (device), writes a[(i*M + j)*n + e] = a_{i+1,j+1}(z[e])
 * (device [M*M][n]) for the M Radau IIA nodes.  Enqueued on `stream`.
 */
int esdc_coefficients(esdc_handle* h, const double* z, int64_t n, int M, double* a, void* stream);

/*
 * Diffusion solve (I - g L) x = b on the handle's mesh (the implicit step of
 * eq. (def_P) with g = dt d_i sigma/(chi C_m)); with a layered conductivity,
 * (I - g A) x = b with g = dt d_i/(chi C_m).  b, x device [n_nodes]; x holds
 * the initial guess on entry and the solution on return.  iters (host,
 * optional) receives the iteration count; synchronises `stream`.  Returns
 * ESDC_ERR_CG_NOT_CONVERGED if cg_maxit was reached.  The solver is the one
 * options.solver selects.  With precision = 1 the solve is the refinement of
 * the precision form and iters counts the inner (FP32) iterations.
 */
int esdc_diffusion_solve(esdc_handle* h, double g, const double* b, double* x, int* iters,
                         void* stream);

/*
 * Pointwise ionic model at every node of y (device [n_state][ld]): writes
 * fE = (-I_ion, h_a, 0), lam = (0, 0, Lambda_g(V)), yinf = (0, 0, w_g,inf(V))
 * (eq. monodomain_g_lambda; device [n_state][ld] each).
 */
int esdc_ionic(esdc_handle* h, const double* y, double* fE, double* lam, double* yinf,
               void* stream);

/*
 * Diagnostic: the library's FP64 exponential and reciprocal, used by the
 * synthetic ionic model (table-driven exp after Tang 1989; Newton reciprocal
 * from the FP32 one), elementwise on device arrays of length n:
 * ex[e] = e^{x[e]}, rc[e] = 1/x[e].  Not part of the method.
 */
int esdc_math_check(const double* x, int64_t n, double* ex, double* rc, void* stream);

/*
 * FMA throughput probe (not part of the method; it measures the ceiling the
 * FP64 kernels are compared with): 4 blocks of 256 threads per SM, each thread
 * running 8 independent chains of n dependent FMAs in FP64 (fp32 = 0) or FP32
 * (fp32 = 1).  *ms (host) receives the CUDA-event time of the launch on
 * `stream`, *flops (host) the flop count (an FMA counts 2).  Synchronises.
 * Errors: INVALID_ARG (n < 1, null outputs), NO_MEMORY, CUDA.
 */
int esdc_fma_probe(int fp32, int64_t n, double* ms, double* flops, void* stream);

/*
 * The build-time errors of the two tables the kernels evaluate in place of
 * transcendental functions (host only: no device work, no handle).  For the
 * ionic model `model` with its parameters (as for esdc_create) the gate table
 * in V: err[0] = the largest error of the FP64 evaluation of b = -Lambda w_inf
 * over |Lambda| (i.e. of w_inf), err[1] = the largest relative error of
 * Lambda.  For M (1..8) and dt > 0 the set-up's coefficient table in z:
 * err[2] = the largest error of dt S_ij and dt d_i phi_1 in units of dt.  All
 * against long-double evaluations of the same functions, as checked when a
 * handle builds them (a table above 4e-15 is refused and the kernels evaluate
 * directly).  Not part of the method.  Errors: INVALID_ARG (unknown model,
 * wrong parameter count, M or dt out of range, null err).
 */
int esdc_table_errors(int model, const double* params, int n_params, int M, double dt, double* err);

/*
 * Allocation-free diffusion solve (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, e.g. code that
 * runs inside a memory-pool or allocator callback, in a process whose device
 * memory another framework has reserved up front, or in a loop that must not
 * enter the allocator after start-up; such callers cannot call esdc_create).
 *
 * Solves (I - g L) x = b on `mesh` like esdc_diffusion_solve with
 * options.solver = 1 (the same CG kernel, Jacobi-preconditioned when
 * precond != 0, stop at ||r|| <= tol ||b||, at most
 * maxit iterations; x holds the initial guess on entry), but needs no handle and
 * allocates nothing: its scratch (CG vectors, block partial sums, barrier
 * counter) lives in one fixed array compiled into the library, of
 * ESDC_STATIC_SCRATCH_BYTES bytes, which every GPU that loads the library holds
 * until the process exits.  b and x are caller-owned device arrays of
 * nx*ny*nz doubles.  iters (host, optional) receives the iteration count; the
 * call synchronises `stream`.
 * Limits and rules:
 *   - meshes with more than ESDC_STATIC_MAX_NODES nodes return ESDC_ERR_TOO_LARGE;
 *   - all calls share the scratch array: calls whose GPU work overlaps (other
 *     streams, other host threads) race on it and must be serialised;
 *   - the first call on each device looks up the array's device address with
 *     cudaGetSymbolAddress, so make it before any stream capture begins.
 * Returns ESDC_OK, ESDC_ERR_INVALID_ARG, ESDC_ERR_TOO_LARGE, ESDC_ERR_CUDA,
 * ESDC_ERR_CG_NOT_CONVERGED, ESDC_ERR_NONFINITE or ESDC_ERR_DEVICE_TIMEOUT.
 */
/*
 * Failure-path check: makes the grid-barrier waits of the handle's iterative
 * solves run out on purpose, so that the error path (ESDC_ERR_DEVICE_TIMEOUT)
 * can be exercised without a hang or a GPU fault.  With skip_block >= 0, block
 * `skip_block` of each cooperative solve kernel does not arrive at the
 * kernel's first grid barrier; every block then waits there until limit_us
 * microseconds (0: the normal 1 s) have passed, raises the TIMEOUT flag and
 * returns.  The solve's result, and the state of a sweep that ran such solves,
 * are then undefined, and esdc_diffusion_solve / esdc_residual return
 * ESDC_ERR_DEVICE_TIMEOUT.  skip_block < 0 restores normal operation.  Only the
 * Chebyshev and CG solves have grid barriers (options.solver 1 and 3, and 0
 * where it does not take the DCT).  Synchronises the device.  Returns
 * ESDC_OK, ESDC_ERR_INVALID_ARG (null handle, limit_us above 1e6) or
 * ESDC_ERR_CUDA.
 */
int esdc_debug_barrier(esdc_handle* h, int skip_block, unsigned limit_us);

#define ESDC_STATIC_MAX_NODES 262144
#define ESDC_STATIC_SCRATCH_BYTES ((4LL * ESDC_STATIC_MAX_NODES + 8 * 1024 + 32) * 8)
int esdc_diffusion_solve_static(const esdc_mesh* mesh, double g, const double* b, double* x,
                                double tol, int maxit, int precond, int* iters, void* stream);

/* ------------------------------------------------------------------------
 * Differentiation: the discrete adjoint of the step.
 *
 * The adjoint is the reverse-mode derivative of exactly the arithmetic of
 * esdc_sweep (the sweep of eq. def_P with the tables of App. A), written by
 * hand: sweeps and nodes in reverse order, one adjoint CG solve per implicit
 * row (the operator is symmetric), analytic Hodgkin-Huxley derivatives, and
 * phi_k' = phi_k - k phi_{k+1} for the Lambda_n-dependence of the tables.
 * Supported: Hodgkin-Huxley, FP64 path, a per-node conductivity field
 * (esdc_set_conductivity_field), M <= 7.  The paper has no adjoint; this is
 * the library's own use of its step.
 * ------------------------------------------------------------------------ */

/* Replaces the ionic-model parameters (same count and rules as esdc_create),
 * e.g. to perturb g_Na and g_K.  Errors: INVALID_ARG. */
int esdc_set_params(esdc_handle* h, const double* params, int n_params);

/* Forward run of nsteps steps from y (device [n_state][ld], in: y_0 at t0,
 * out: y_nsteps) keeping a checkpoint of every step's input in ckpt (device,
 * caller-owned, [nsteps][n_state][ld]) and, after every step n, V at the
 * nsens sensor nodes sens (device int [nsens]) in traces (device
 * [nsteps][nsens]).  Stream-ordered.  Errors: INVALID_ARG, UNSUPPORTED, and
 * those of esdc_sweep. */
int esdc_adjoint_forward(esdc_handle* h, double* y, double t0, double dt, int M, int K, int nsteps, int nsens,
                         const int* sens, double* traces, double* ckpt, void* stream);

/* Gradients of a loss L through its derivative dtraces = dL/dtraces (device
 * [nsteps][nsens]) and, optionally, dy_final = dL/dy_nsteps (device
 * [n_state][ld] or NULL): gsig (device [N]) = dL/dsigma per node, gpar (host
 * [2]) = dL/d(g_Na, g_K), gy0 (device [n_state][ld] or NULL) = dL/dy_0.
 * Recomputes every step from ckpt (esdc_adjoint_forward with the same
 * arguments and parameters) and reverses it.  Allocates its workspace and
 * synchronises the stream.  Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA,
 * CG_NOT_CONVERGED, NONFINITE, DEVICE_TIMEOUT. */
int esdc_adjoint_backward(esdc_handle* h, const double* ckpt, double t0, double dt, int M, int K, int nsteps,
                          int nsens, const int* sens, const double* dtraces, const double* dy_final, double* gy0,
                          double* gsig, double* gpar, void* stream);

/* ------------------------------------------------------------------------
 * Ragged batches (many tissues per launch).
 *
 * A batch holds n tissues that share the ionic model, its parameters, chi,
 * C_m and the options, but each has its own mesh (any dim/size), scalar
 * conductivity sigma[b], stimulus and start time.  One esdc_batch_sweep
 * advances every tissue by one HSDC step (the same method and arithmetic as
 * esdc_sweep, Sec. 3.1) with the launches of a single step: the node kernels
 * cover all tissues, and each diffusion solve is one cooperative launch that
 * runs all tissues' CG iterations side by side, each with its own step sizes
 * and stop test.  The launches of a step are recorded once in a CUDA graph and
 * replayed.  Every reduction is fixed per 512-node tile and per tissue, so a
 * tissue's results are identical bit for bit whatever the rest of the batch and
 * whatever launch shape the autotuner picks.  The paper batches its
 * time-parallel slices across processors (Sec. 3.2); batching tissues is this
 * library's own use of the same step.
 *
 * State layout: one device array y[n_state][ld] for the whole batch; tissue b
 * occupies columns [offset_b, offset_b + N_b), offset_b a multiple of 512
 * (esdc_batch_layout); the padding columns are never read as mesh nodes.
 * Batches run the FP64 path (options.precision must be 0) with scalar
 * conductivities.  All tissues' diffusion solves run in one cooperative
 * launch: the Chebyshev semi-iteration, each tissue on its own exactly known
 * spectrum, with options.solver = 0 (the default), the Jacobi-PCG with
 * solver = 1.
 * ------------------------------------------------------------------------ */
typedef struct esdc_batch esdc_batch;

/* meshes[n], sigma[n] (mS/mm) are host arrays, copied.  Errors as esdc_create;
 * ESDC_ERR_UNSUPPORTED for precision != 0 or more tissues than one CG block
 * can track (about 19,000 single-tile tissues on 152 SMs). */
int esdc_batch_create(int n, const esdc_mesh* meshes, const double* sigma, double chi, double Cm, int model,
                      const double* params, int n_params, const esdc_options* opt, esdc_batch** out);
void esdc_batch_destroy(esdc_batch* b);
const char* esdc_batch_last_error(const esdc_batch* b);

/* Stimulus of tissue `tissue` (0-based), in the form of esdc_set_stimulus.
 * Synchronises the device.  Errors: INVALID_ARG, CUDA. */
int esdc_batch_set_stimulus(esdc_batch* b, int tissue, int nbox, const int* box, const double* amp,
                            const double* t_on, const double* t_off);

/* n_state, the row pitch ld of the batch state, and (optional, host [n]) the
 * first column of every tissue. */
int esdc_batch_layout(const esdc_batch* b, int* n_state, int64_t* ld, int64_t* offsets);

/* Every column of y (device, [n_state][ld]) at the model's rest state at V0. */
int esdc_batch_init_state(esdc_batch* b, double* y, double V0, void* stream);

/* One HSDC step of every tissue, in place on y (device, [n_state][ld]).
 * t (host, [n]) holds each tissue's t_n; dt, M (<= M_max) and K are shared.
 * Stream-ordered, no synchronisation, except the first step with a new
 * (M, dt), which builds and uploads the set-up's coefficient table as
 * esdc_sweep does (before any recording).  The first call for a given
 * (y, M, K, dt) records the step's launches in a CUDA graph on a stream of
 * the batch's own and later calls launch that graph on `stream` (falling back
 * to direct launches if the CUDA runtime cannot record them); a refilled
 * table slot makes the next call record again.  Errors: INVALID_ARG, CUDA. */
int esdc_batch_sweep(esdc_batch* b, double* y, const double* t, double dt, int M, int K, void* stream);

/* As esdc_batch_sweep with a separate output: y_n from y_in, y_{n+1} of every
 * tissue to y_out (both device [n_state][ld]; they may be the same array).
 * from_iterate != 0 starts the sweeps not from y^0 = 1 (x) y_n but from the
 * collocation iterate y_{n,1..M} that the previous call (same M) left in the
 * batch, with y_{n,0} = y_n now taken from y_in: G and f_I are evaluated on
 * that iterate with Lambda_n = Lambda(y_n).  This is one Q^par sweep
 * (eq. def_Q): the paper's parallel preconditioner applies the single-step
 * sweep to every time slice at once.  Errors: INVALID_ARG, CUDA. */
int esdc_batch_sweep_from(esdc_batch* b, const double* y_in, double* y_out, const double* t, double dt, int M, int K,
                          int from_iterate, void* stream);

/* `iters` iterations of Q^par (eq. prec_picard_seq with Q = Q^par, eq. def_Q)
 * over P = n consecutive time steps, the tissues of the batch being the time
 * slices (they must share mesh and conductivity).  On entry slice 0 of y_in
 * holds y0 at time t0; slice p covers [t0 + p dt, t0 + (p+1) dt].  The first
 * iteration starts every slice from z^0 = 1 (x) y0; iteration k+1 runs one
 * sweep in every slice from its iterate with y_{p,0} = y_{p-1,M} of iteration
 * k (y_{0,0} = y0).  On return y_out slice p holds y_{p,M}; y_in slices 1..P-1
 * are overwritten (y_{p,0} of a next iteration).  Stream-ordered.
 * Errors: INVALID_ARG, CUDA. */
int esdc_batch_qpar(esdc_batch* b, double* y_in, double* y_out, double t0, double dt, int M, int iters, void* stream);

/* The general form of esdc_batch_sweep_from: tau (device [M][n_state][ld] or
 * NULL) is the FAS correction of Algorithm HSDC (Sec. 3.2), added to the
 * right-hand side 1 (x) y_n of every tissue's collocation system; K = 0 (with
 * from_iterate) only evaluates the residual at the iterate; want_residual
 * keeps the residual vectors r_i = y_n + tau_i + dt sum_j a_ij G_j - y_i
 * (esdc_batch_iterate).  Errors: INVALID_ARG, NO_MEMORY, CUDA. */
int esdc_batch_sweep_ex(esdc_batch* b, const double* y_in, double* y_out, const double* tau, const double* t, double dt,
                        int M, int K, int from_iterate, int want_residual, void* stream);

/* Device pointers, owned by the batch, of its collocation iterate
 * y_{n,1..M} ([M_max][n_state][ld], node j at row block j-1) and of the kept
 * residual vectors (same layout; NULL until a call asked for them).  Writing
 * the iterate sets the starting point of the next from_iterate sweep. */
int esdc_batch_iterate(esdc_batch* b, double** Y, double** R);

/* dst_i = beta dst_i + sum_j W[i][j] src_j for the collocation rows i < Md,
 * j < Ms of every state and of the first n_cols columns (src [Ms][n_state]
 * [src_ld], dst [Md][n_state][dst_ld], both device, distinct; W host
 * [Md][Ms]).  With W the Lagrange matrix between two node sets this is the
 * interpolator I_l of Sec. 3.2 (restriction and prolongation in M).
 * Stream-ordered.  Errors: INVALID_ARG, CUDA. */
int esdc_interp(const double* src, int Ms, int64_t src_ld, double* dst, int Md, int64_t dst_ld, int n_state,
                int64_t n_cols, const double* W, double beta, void* stream);

/* Algorithm HSDC (Sec. 3.2) with two levels M = M1, M2 (M2 < M1) over the
 * P = n tissues of `fine` as consecutive time slices (shared mesh and
 * conductivity), without Burn-in (z^0 = 1 (x) y0).  coarse[p] (p < P) are
 * single-tissue batches of the same mesh with M_max >= M2 (the coarse level,
 * swept one slice after another by Q^seq).  The restriction S and the
 * prolongation T are the Lagrange interpolators between the two levels' Radau
 * nodes c_1..c_M.  One iteration: tau = S R_1(z) - R_2(S z) per
 * slice, one Q^seq sweep with tau on the coarse level, the coarse-grid
 * correction z += T (z_2 - S z), one Q^par sweep on the fine level.  y_in
 * slice 0 holds y0 at t0 on entry; on return the fine iterate is in
 * esdc_batch_iterate(fine) and y_out slice p holds y_{p,M1}.  Synchronises.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA and those of the sweeps. */
int esdc_hsdc2(esdc_batch* fine, esdc_batch* const* coarse, double* y_in, double* y_out, double t0, double dt, int M1,
               int M2, int iters, void* stream);

/* Algorithm HSDC (Sec. 3.2) with L >= 2 levels, M[0] > M[1] > ... > M[L-1]
 * Radau nodes (host array), over the P tissues of levels[0] as consecutive
 * time slices, without Burn-in.  levels[0..L-2] are P-tissue batches of the
 * same slices (same meshes, so the same layout; M_max >= M[l]) swept by Q^par;
 * coarse[p] (p < P) are single-tissue batches of the slice mesh with
 * M_max >= M[L-1], swept one slice after another by Q^seq.  Restriction and
 * prolongation between consecutive levels are the Lagrange interpolators
 * through the source level's nodes c_1..c_M.  One iteration: going down,
 * tau_l = S R_{l-1}(z_{l-1}; tau_{l-1}) - R_l(S z_{l-1}) (the paper's
 * D_l(S z) - S D_{l-1}(z) + S tau_{l-1}) and, above the coarsest level, one
 * Q^par sweep from S z_{l-1} with tau_l; one Q^seq sweep with tau on the
 * coarsest level; going up, the coarse-grid correction z_l += T (z_{l+1} -
 * S z_l) and one Q^par sweep with tau_l on each level.  A Q^par sweep starts
 * slice p from the end value of slice p-1 of the iterate it sweeps.  y_in
 * slice 0 holds y0 at t0 on entry; on return the finest iterate is in
 * esdc_batch_iterate(levels[0]) and y_out slice p holds y_{p,M[0]}.  With
 * L = 2 this is esdc_hsdc2.  Allocates its scratch (per level above the
 * coarsest: 2 M_l + 1 state arrays).  Synchronises.  Errors: INVALID_ARG,
 * NO_MEMORY, CUDA and those of the sweeps. */
int esdc_hsdc(esdc_batch* const* levels, esdc_batch* const* coarse, const int* M, int L, double* y_in,
              double* y_out, double t0, double dt, int iters, void* stream);

/* Per tissue (host [n], optional): max |r| of the collocation residual and
 * max |y| of the last step.  Synchronises that step's stream.  Returns
 * NONFINITE, CG_NOT_CONVERGED or DEVICE_TIMEOUT if any tissue raised it. */
int esdc_batch_residual(esdc_batch* b, double* res_inf, double* y_inf);

/* CG iterations of the last step, [K*M][n] (solve-major), at most n_entries. */
int esdc_batch_stats(esdc_batch* b, int* cg_iters, int n_entries);

/* Graph recording on (default) or off. */
int esdc_batch_set_graph(esdc_batch* b, int on);
/* 1 if the last step ran from a recorded graph. */
int esdc_batch_graph_active(const esdc_batch* b);
/* Why recording failed ("" if it did not). */
const char* esdc_batch_graph_error(const esdc_batch* b);

/* Launch shape: node-kernel grid in waves of the resident capacity (1..8), CG
 * block size (256 or 512) and CG blocks per SM (1..4, within occupancy).  No
 * effect on results. */
int esdc_batch_set_shape(esdc_batch* b, int node_waves, int cg_threads, int cg_blocks_per_sm);
int esdc_batch_get_shape(const esdc_batch* b, int* node_waves, int* cg_threads, int* cg_blocks);

/* One persistent launch per step (on = 1; batches with options.solver 0 or 3,
 * the Chebyshev solves): the set-up, the K (M+1) node phases, the K M solves
 * of all tissues and the residual run in one cooperative kernel whose phases
 * meet at the bounded grid barrier (the step is still recorded in a CUDA graph
 * when graphs are on).  threads: block size (256 or 512); tile: the consecutive
 * nodes a warp takes at a time in the node phases (a multiple of 32, at most
 * 2048).  on = 0 returns to the launch sequence.  Results are bit for bit those
 * of the launch sequence.  Synchronises.  Errors: INVALID_ARG, UNSUPPORTED
 * (the CG solver), CUDA. */
int esdc_batch_set_persistent(esdc_batch* b, int on, int threads, int tile);
int esdc_batch_get_persistent(const esdc_batch* b, int* on, int* threads, int* tile);

/* Autotuner: times `reps` steps of the batch itself (from rest at V0, time t,
 * on the caller's scratch state y_scratch of the batch's layout) for each
 * candidate and keeps the fastest: the launch sequence with each launch shape
 * (node waves, solve block size, solve blocks per SM), and with the Chebyshev
 * solves the persistent launch with block sizes 256 and 512 and node tiles of
 * 32 to 512 nodes.  Synchronises. */
int esdc_batch_tune(esdc_batch* b, double* y_scratch, double V0, double t, double dt, int M, int K, int reps,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif
