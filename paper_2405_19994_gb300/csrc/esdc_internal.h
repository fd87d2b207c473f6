// Internal declarations of the HSDC library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/esdc.h"

#define ESDC_MMAX 8        // collocation nodes
#define ESDC_NSMAX 19      // states per mesh node
#define ESDC_NGMAX 12      // gating variables per mesh node
#define ESDC_NPMAX 160     // ionic-model parameters (+ derived constants)
#define ESDC_MAXBOX 16     // stimulus boxes
#define ESDC_NSER 48       // reciprocal table length for the phi_k series
#define ESDC_PROF_CLASSES 4  // esdc_profile kernel classes
#ifndef ESDC_CG_THREADS
#define ESDC_CG_THREADS 512    // threads per CG block (one block per SM)
#endif

// Collocation data of one M (Sec. 3.1.2, App. A), computed on the host once.
struct ColloData {
    double c[ESDC_MMAX + 1];                       // c_0 = 0 < c_1 < ... < c_M = 1 (Radau IIA)
    double d[ESDC_MMAX + 1];                       // d_i = c_i - c_{i-1}
    // B[i-1][j-1][k-1] = c_i^k w_j^{k-1}: a_ij(z) = sum_k B_ijk phi_k(c_i z)   (App. A)
    double B[ESDC_MMAX][ESDC_MMAX][ESDC_MMAX];
    double A0[ESDC_MMAX][ESDC_MMAX];               // a_ij(0) (collocation matrix)
    double S0[ESDC_MMAX][ESDC_MMAX];               // a_ij(0) - a_{i-1,j}(0), a_0j = 0
    double X1;                                     // series / recurrence switch for phi_k
    int nser;                                      // terms of the phi_M series
    // ser[m] = 1/((M-1)! m! (m+M)): phi_M(x) = e^x sum_m ser[m] (-x)^m
    double ser[ESDC_NSER];
    // shorter series for smaller |x|: |x| <= xb[l] needs nb[l] terms (l = 0..4)
    double xb[5];
    int nb[5];
};

struct ModelDev;
struct ModelDevF;

// Fills ColloData for 1 <= M <= 8.  Returns 0 on success.
int esdc_colloc_build(int M, ColloData* out);

// Uniform cell-centred mesh as seen by the kernels.
struct MeshDev {
    int nx, ny, nz;
    int N;            // nx*ny*nz
    int64_t ld;       // row pitch of state arrays (doubles)
    double ih2;       // 1/h^2
    // Layered anisotropic conductivity (nullptr: scalar sigma, plain stencil):
    // lay[0..nz) sxx/h^2, [nz..2nz) syy/h^2, [2nz..3nz) sxy/(2h^2),
    // [3nz..4nz) face sigma_zz/h^2 between layers k and k+1.
    const double* lay = nullptr;
    const double* wdiag = nullptr;   // [N] -diag(A) (Jacobi weights), layered or field case
    const float* layf = nullptr;     // FP32 copy of lay (precision form)
    // Heterogeneous isotropic conductivity (nullptr: scalar sigma): sigma per
    // node [N] (mS/mm); a face carries the mean of its two nodes.
    const double* sig = nullptr;
    // Order of the Laplacian (scalar sigma only): 2 (3/5/7-point) or 4 (the
    // fourth-order five-point difference per axis with mirrored ghost cells).
    int order = 2;
    // Layered operator: an upper bound of the spectrum of -A (Gershgorin, set
    // on the host with the layers; 0 otherwise).  The spectrum of I - g A is
    // then inside [1, 1 + g lam_bound] (A is symmetric negative semi-definite
    // with the constants as null space).
    double lam_bound = 0.0;
};

// Mirror image of index j on an axis of n cells (reflection about the outer
// faces, repeated while outside: axes shorter than the stencil).
__host__ __device__ inline int esdc_mirror(int j, int n)
{
    while (j < 0 || j >= n) j = j < 0 ? -j - 1 : 2 * n - 1 - j;
    return j;
}

struct StimDev {
    int nbox;
    int box[ESDC_MAXBOX][6];
    double amp[ESDC_MAXBOX], t_on[ESDC_MAXBOX], t_off[ESDC_MAXBOX];
};

// The gate functions tabulated in V (esdc_vtab.cpp; SYN19 and HH1952): ESDC_VTAB_N
// intervals of ESDC_VTAB_W mV from ESDC_VTAB_VLO, a polynomial of degree
// ESDC_VTAB_NC - 1 in t = V - V_mid per function and interval; a row holds
// V_mid and a pad (16-byte alignment), then per gate the coefficient pairs
// (b, Lambda) of t^0, t^1, ..., b = -Lambda w_inf, so that one 16-byte load feeds both
// Horner recurrences.
#define ESDC_VTAB_VLO (-140.0)
#ifndef ESDC_VTAB_W
#define ESDC_VTAB_W 0.0078125      // interval width (mV): 1/128, a power of two
#endif
#ifndef ESDC_VTAB_NC
#define ESDC_VTAB_NC 4             // coefficients per function (degree 3)
#endif
#define ESDC_VTAB_N ((int)(240.0 / ESDC_VTAB_W))
#define ESDC_VTAB_ROW (2 + 2 * ESDC_NGMAX * ESDC_VTAB_NC)
#define ESDC_VTAB_TOL 4e-15        // refuse a table whose FP64 evaluation misses by more
struct ModelDev {
    double p[ESDC_NPMAX];
    const double* vtab = nullptr;  // the gate table, or nullptr: direct evaluation
};

struct ModelDevF {            // FP32 copy of the parameters (precision form)
    float p[ESDC_NPMAX];
};

// Ragged batches: meshes concatenated in the state arrays, each starting on a
// tile boundary; tiles are also the unit of every deterministic reduction.
#define ESDC_TILE_SHIFT 9
#define ESDC_TILE (1 << ESDC_TILE_SHIFT)   // 512 nodes

struct TissueDev {
    int nx, ny, nz, N;
    int off;                 // first node in the concatenated arrays (multiple of ESDC_TILE)
    int tile0, ntile;        // its tiles
    double ih2, D;           // 1/h^2, sigma / (chi C_m)
    double wspec;            // sum over axes with n > 1 of 4 sin^2(pi (n-1)/(2n)): the spectrum
                             // of I - g L is [1, 1 + g ih2 wspec]
    StimDev st;
};

// Direct DCT-II solve (options.solver = 2), per axis: the FFT tables (powers
// of two: twiddles e^{-2 pi i k/n}, and (cos, sin)(pi k/(2n)) whole and halved
// for the inverse and forward post-processing) or the two dense cosine
// matrices (other lengths).
struct DctAxisDev {
    int n = 1, logn = -1;
    const double2* tw = nullptr;
    const double2* cs = nullptr;
    const double2* csh = nullptr;
    const double* fwd = nullptr;
    const double* inv = nullptr;
};
#define ESDC_DCT_SLOTS ESDC_MMAX
// The axes' tables, the eigenvalues of the 1D difference operators per mode
// (1/h^2 included), and the factor tables of the z-direction tridiagonal
// solves of the second-order stencil: per slot [2][N] (A then C) for the
// value gkey of g (a slot is refilled, round robin, when a new g comes).
struct DctDev {
    DctAxisDev ax, ay, az;
    double *ex = nullptr, *ey = nullptr, *ez = nullptr;
    double* ztab = nullptr;
    int nslot = 0, next_slot = 0;
    double gkey[ESDC_DCT_SLOTS] = {};
    bool used[ESDC_DCT_SLOTS] = {};
    bool cheap = false;             // esdc_dct_cheap for the current stencil order (the automatic choice)
    bool yzy = false;               // second order: y transforms and z solves in one kernel (k_dct_yzy)
    int yzy_threads = 0;
    size_t yzy_smem = 0;
};

// CG solve on the handle's mesh: (I - g L) x = b (Jacobi-preconditioned).
struct CgWork {
    double *r, *p, *q, *z;          // [ld] each
    float *r32, *p32, *q32, *z32, *e32;   // [ld] each, precision form only (else null)
    double* part;                   // [8 * max_blocks] block partial sums
    unsigned* bar;                  // [4] grid barrier: arrival count, spare, and two test words (grid_barrier)
    int* status;                    // [2]: iterations of the last solve, flag bits
    int max_blocks;
    int threads;
    DctDev* dct = nullptr;          // set when options.solver = 2
};

// Whether the DCT solve costs less than an iterative one on this mesh for the
// given stencil order: every transformed axis (x and y; z for the fourth
// order) is of power-of-two length (FFT, about 13 FP64 operations per value
// and pass) or dense, and the dense axes together cost at most 32 FMAs per
// value and pass (a dense axis of length n costs n).  The automatic solver
// choice takes the DCT only then.
bool esdc_dct_cheap(const MeshDev& m, int order);
// Whether the DCT solve takes this mesh (every axis length does, up to the
// shared-memory size of a dense tile).
bool esdc_dct_supported(const MeshDev& m);
// Tables for the mesh, with nslot (1..ESDC_DCT_SLOTS) cached values of g.
cudaError_t esdc_dct_create(const MeshDev& m, int nslot, DctDev* d);
cudaError_t esdc_dct_set_order(const MeshDev& m, DctDev* d);   // eigenvalues for m.order
void esdc_dct_destroy(DctDev* d);
// x = (I - g L)^{-1} b by the DCT-II (scalar sigma); uses w.r and w.p as work vectors
// (b may alias x, not w.r or w.p).
cudaError_t esdc_dct_launch(const MeshDev& m, const CgWork& w, double g, const double* b, double* x,
                            int* iter_log, int* flags, cudaStream_t s);

// The gate table of a model (SYN19, HH1952): rows [ESDC_VTAB_N][ESDC_VTAB_ROW] and
// the largest errors of its FP64 evaluation against the direct functions
// (absolute for w_inf, relative for Lambda).  0: built; -1: no table for this
// model; -2: an error above ESDC_VTAB_TOL (rows cleared).
int esdc_vtab_build(int model, const double* params, std::vector<double>& rows, double* err_winf, double* err_lam);

// The set-up's exponential coefficients tabulated in y = 1 - z, z = dt Lambda
// (esdc_ztab.cpp): ESDC_ZTAB_OCT octaves of y, 2^ESDC_ZTAB_SUB intervals each,
// a polynomial of degree ESDC_ZTAB_NC - 1 per function and interval; a row
// holds y_mid, a pad, then for i = 0..M-1 the coefficients of dt d_{i+1}
// phi_1(d_{i+1} z) and of dt S_{i+1,j}(z), j = 0..M-1.
#define ESDC_ZTAB_OCT 12
#ifndef ESDC_ZTAB_SUB
#define ESDC_ZTAB_SUB 10           // 1024 intervals per octave of y
#endif
#ifndef ESDC_ZTAB_NC
#define ESDC_ZTAB_NC 4             // coefficients per function (degree 3)
#endif
#define ESDC_ZTAB_ROW(M) (2 + (M) * ((M) + 1) * ESDC_ZTAB_NC)
#define ESDC_ZTAB_TOL 4e-15         // refuse a table whose FP64 evaluation misses by more (units of dt)
// Builds (or takes from this process's cache) the table for (M, dt, C);
// returns 0, -1 (bad arguments) or -2 (error above ESDC_ZTAB_TOL, rows
// cleared); *err: the largest error, in units of dt.
int esdc_ztab_build(int M, double dt, const ColloData& C, std::vector<double>& rows, double* err);
// Device copies of the set-up tables of a handle or batch for a few (M, dt).
#define ESDC_ZTAB_SLOTS 4
struct ZtabSlots {
    int M[ESDC_ZTAB_SLOTS] = {};
    double dt[ESDC_ZTAB_SLOTS] = {};
    double* dev[ESDC_ZTAB_SLOTS] = {};
    size_t n[ESDC_ZTAB_SLOTS] = {};      // doubles allocated
    int next = 0;
    unsigned gen = 0;                    // counts slot fills (recorded graphs check it)
    int builds = 0;                      // tables built so far (at most ESDC_ZTAB_BUILDS)
};
#define ESDC_ZTAB_BUILDS 16
// The device table for (M, dt): built and uploaded on first use (which
// synchronises the device once), or nullptr for the direct evaluation (no
// table within ESDC_ZTAB_TOL, a CUDA error, the stream is being captured and
// the table is not there yet, or ESDC_ZTAB_BUILDS tables were built already:
// step sizes that keep changing do not pay for a table each).
const double* esdc_ztab_device(ZtabSlots& z, int M, double dt, const ColloData& C, cudaStream_t s);
void esdc_ztab_free(ZtabSlots& z);

// Validates ionic-model parameters and fills the device parameter blocks;
// returns ESDC_OK or ESDC_ERR_INVALID_ARG.
int esdc_model_setup(int model, const double* params, int n_params, ModelDev* mp, ModelDevF* mpf, int* NS, int* NG);

#define ESDC_FLAG_CG_MAXIT   1
#define ESDC_FLAG_TIMEOUT    2
#define ESDC_FLAG_NONFINITE  4

// Enqueue one solve of (I - g A) x = b; iter_log (device, optional) receives the
// iteration count, flags (device) accumulates ESDC_FLAG_* bits.  solver 0 takes
// the Chebyshev semi-iteration where esdc_cheb_eligible holds and g > 0, the
// (Jacobi-P)CG otherwise; solver 1 always the CG; solver 2 the DCT-II direct
// solve (w.dct must be set).  Returns a cudaError_t.
cudaError_t esdc_cg_launch(const MeshDev& mesh, const CgWork& w, double g, const double* b,
                           double* x, double tol, int maxit, int precond, int solver, int* iter_log,
                           int* flags, cudaStream_t s);
// Precision form: FP32 inner PCG with FP64 iterative refinement (same contract;
// iter_log receives the number of inner iterations).
cudaError_t esdc_cg_mixed_launch(const MeshDev& mesh, const CgWork& w, double g, const double* b,
                                 double* x, double tol, int maxit, int precond, int solver, int* iter_log,
                                 int* flags, cudaStream_t s);
// Blocks to use for a cooperative CG launch on this device.
int esdc_cg_blocks(const MeshDev& mesh, int threads);

// Quad form of the solves (four x-consecutive nodes per thread, diagonal and
// Jacobi tables in shared memory): used when nx is a multiple of 4, b and x are
// 16-byte aligned and the layered operator has at most ESDC_CG4_MAX_LAYERS
// layers; esdc_cg_launch and esdc_cg_mixed_launch dispatch to it.
#define ESDC_CG4_MAX_LAYERS 256
struct CgArgsHost {
    MeshDev mesh;
    CgWork w;
    double g;
    const double* b;
    double* x;
    double tol;
    int maxit, precond;
    int* iter_log;
    int* flags;
};
bool esdc_cg4_eligible(const MeshDev& m, const void* b, const void* x);
cudaError_t esdc_cg4_launch(const CgArgsHost& h, bool mixed, cudaStream_t s);
// Chebyshev semi-iteration: 1/theta, q = (sqrt(kappa) - 1)/(sqrt(kappa) + 1),
// log q, and the recurrence coefficients ca[k] = rho_{k+1} rho_k and
// cb[k] = 2 rho_{k+1}/delta (the last entry serves beyond the table).
#define ESDC_CHEB_TAB 64
struct ChebArgs {
    double inv_theta, q, log_q;
    double ca[ESDC_CHEB_TAB];
    double cb[ESDC_CHEB_TAB];
};
// The interval [1, 1 + g w] holding the spectrum of I - g A (or I - g L) of the
// mesh's operator, and the coefficients on it.  w: exactly
// (1/h^2) sum_axes 4 sin^2(pi (n-1)/(2n)) for the scalar second-order stencil,
// exactly (1/(12 h^2)) sum_axes (30 + 2 cos 2t - 32 cos t), t = pi (n-1)/n, for
// the fourth-order one, and the host's Gershgorin bound lam_bound for the
// layered operator and the conductivity field.  False when the interval has no
// width in FP64 (g below rounding) or no bound is known.
bool esdc_cheb_interval(const MeshDev& m, double g, ChebArgs& c);
// Chebyshev semi-iteration, quad layout (no dot products inside the iteration).
bool esdc_cheb_eligible(const MeshDev& m, const void* b, const void* x);
cudaError_t esdc_cheb_launch(const CgArgsHost& h, cudaStream_t s);
// The precision form's refinement with Chebyshev inner solves (same eligibility).
cudaError_t esdc_cheb_mixed_launch(const CgArgsHost& h, cudaStream_t s);
