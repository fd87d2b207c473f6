// HSDC time step on the device: step set-up, the fused per-node sweep kernel,
// the final evaluation and the collocation residual (Sec. 3.1).
//
// The sweep implements the preconditioned Picard iteration of eq. (prec_picard)
// with P from eq. (def_P) and C from eq. (def_C).  Subtracting row i-1 from row i
// gives the recursive form used here (for i = 1 the y_{n,0} terms cancel, as
// noted after eq. (def_P)):
//
//   y_i^{k+1} - dt d_i f_I(y_i^{k+1}) = y_{i-1}^{k+1} + dt sum_j S_ij G_j^k
//        + dt d_i [ -f_I(y_i^k) + Delta f_E + phi_1(d_i dt Lambda_n) Delta h ]
//
// with S_ij = a_ij - a_{i-1,j} (a_0j = 0), G_j^k = g_n(y_j^k) (eq. def_g) and
// Delta(.) = (.)(y_{i-1}^{k+1}) - (.)(y_{i-1}^k), h(y) = f_e(y) + Lambda_n (y_n - y).
// V and the auxiliaries see Lambda_n = 0 (a_ij = standard collocation weights),
// the gates see the exponential weights a_ij(dt Lambda_n) (Sec. 3.1.2).
//
// Data layout (all FP64, SoA rows of pitch ld):
//   y (caller)   [NS][ld]        y_n in, y_{n+1} out
//   Y            [M][NS][ld]     collocation iterate y_1..y_M
//   G[2]         [M][NS][ld]     g_n(y_j) of the previous / current sweep
//   FI           [M][ld]         f_I(y_j) (V row only)
//   S            [M][M][NG][ld]  S_ij(dt Lambda_n) per gate
//   PHI          [M][NG][ld]     phi_1(d_i dt Lambda_n)
//   LAMN         [NG][ld]        Lambda_n
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "esdc_internal.h"
#include "esdc_models.cuh"

namespace {

__constant__ ColloData c_col[ESDC_MMAX];     // index M-1
__constant__ double c_inv[ESDC_NSER];        // c_inv[m] = 1/m (c_inv[0] unused)
__constant__ double c_invfact[ESDC_MMAX + 2];

struct StepArgs {
    MeshDev m;
    StimDev st;
    ModelDev mp;
    int i;                 // collocation node 1..M (k_node), M+1: evaluate G at node M only
    int k;                 // sweep index (0-based)
    double rho;            // warm-start extrapolation weight for node i
    double* Vprev;         // [ld] V_{i-1}^k, saved before node i-1 was solved
    double dt, t_n, D, inv_Cm;
    double dS0[ESDC_MMAX][ESDC_MMAX];   // dt * (a_ij(0) - a_{i-1,j}(0))
    double dtd[ESDC_MMAX + 1];          // dt * d_i
    unsigned stim_on[ESDC_MMAX + 1];    // boxes active at t_{n,j}, j = 0..M (bit b = box b)
    const double* yn;
    double* yout;          // residual kernel: destination of y_{n+1}
    double* Y;
    const double* Gold;
    double* Gnew;
    double* FI;
    double* S;
    double* PHI;
    double* LAMN;
    double* rhs;
    double* R;             // residual vectors (optional)
    unsigned long long* rmax;   // [NS] per-state max |r| (as ordered bits), [NS] max |y|
    int* flags;
};

__device__ __forceinline__ void node_xyz(const MeshDev& m, int p, int& ix, int& iy, int& iz)
{
    int r = p / m.nx;
    ix = p - r * m.nx;
    iz = r / m.ny;
    iy = r - iz * m.ny;
}

// L v at node p: (1/h^2) sum over in-domain neighbours of (v_q - v_p).
__device__ __forceinline__ double lap(const MeshDev& m, const double* __restrict__ v, int p,
                                      int ix, int iy, int iz)
{
    const double vp = v[p];
    const int sxy = m.nx * m.ny;
    double s = 0.0;
    if (ix > 0)        s += v[p - 1] - vp;
    if (ix < m.nx - 1) s += v[p + 1] - vp;
    if (iy > 0)        s += v[p - m.nx] - vp;
    if (iy < m.ny - 1) s += v[p + m.nx] - vp;
    if (iz > 0)        s += v[p - sxy] - vp;
    if (iz < m.nz - 1) s += v[p + sxy] - vp;
    return s * m.ih2;
}

// I_stim at a node for the boxes whose time window contains the node's time
// (the window test t_on <= t < t_off is made once on the host: bit b of `on`).
__device__ __forceinline__ double stim_at(const StimDev& st, unsigned on, int ix, int iy, int iz)
{
    double s = 0.0;
    for (int b = 0; b < st.nbox; ++b) {
        if (((on >> b) & 1u) && ix >= st.box[b][0] && ix < st.box[b][1] &&
            iy >= st.box[b][2] && iy < st.box[b][3] && iz >= st.box[b][4] && iz < st.box[b][5])
            s += st.amp[b];
    }
    return s;
}

// phi_1..phi_M at x <= 0 (App. A eq. def_phik).  Two regimes:
//  |x| >  X1: phi_1 = (e^x - 1)/x (no cancellation there: X1 > 1.4 for M >= 2),
//             then phi_{k+1} = (phi_k - 1/k!)/x;
//  |x| <= X1: phi_M = e^x/(M-1)! sum_m (-x)^m/(m! (m+M)) (all terms >= 0,
//             Horner form with host coefficients; the number of terms steps
//             down with |x|), then phi_k = x phi_{k+1} + 1/k!.
// X1 balances the rounding growth of the two recurrences (set on the host).
// M = 1: phi_1 = expm1(x)/x.
template <int M>
__device__ __forceinline__ void phi_all(double x, double (&ph)[M])
{
    const ColloData& C = c_col[M - 1];
    if (M == 1) {
        ph[0] = (x == 0.0) ? 1.0 : expm1(x) / x;
    } else if (-x > C.X1) {
        const double rx = esdc::esdc_rcp(x);
        ph[0] = (esdc::esdc_exp(x) - 1.0) * rx;
#pragma unroll
        for (int k = 1; k < M; ++k) ph[k] = (ph[k - 1] - c_invfact[k]) * rx;
    } else {
        const double nx = -x;
        const int n = nx <= C.xb[0] ? C.nb[0] : nx <= C.xb[1] ? C.nb[1] : nx <= C.xb[2] ? C.nb[2]
                    : nx <= C.xb[3] ? C.nb[3] : C.nb[4];
        double acc = C.ser[n];
        for (int m = n - 1; m >= 0; --m) acc = fma(acc, nx, C.ser[m]);
        ph[M - 1] = esdc::esdc_exp(x) * acc;
#pragma unroll
        for (int k = M - 1; k >= 1; --k) ph[k - 1] = fma(x, ph[k], c_invfact[k]);
    }
}

// phi_1(y) = (e^y - 1)/y for y <= 0.
__device__ __forceinline__ double phi1(double y)
{
    if (y < -1.0) return (esdc::esdc_exp(y) - 1.0) * esdc::esdc_rcp(y);
    return (y == 0.0) ? 1.0 : expm1(y) / y;
}

// ------------------------------------------------------------------ set-up
// Lambda_n, dt S_ij(dt Lambda_n), dt d_i phi_1(d_i dt Lambda_n) (tables carry the
// step size); y^0 = 1 (x) y_n; G_j^0 = g_n(t_{n,j}, y_n); FI_j^0 = f_I(y_n).
template <class Model, int M>
__global__ void __launch_bounds__(128) k_setup(StepArgs a)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const MeshDev& m = a.m;
    const ColloData& C = c_col[M - 1];
    const int64_t ld = m.ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(m, p, ix, iy, iz);
        double u[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) u[s] = a.yn[s * ld + p];
        const double fi = a.D * lap(m, a.yn, p, ix, iy, iz);
        double mI, ha[NA > 0 ? NA : 1], lam[NG], yinf[NG];
        Model::eval(a.mp.p, u, mI, NA > 0 ? ha : nullptr, lam, yinf);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            double* Yj = a.Y + (int64_t)j * NS * ld;
            double* Gj = a.Gnew + (int64_t)j * NS * ld;
            Gj[p] = fi + (stim_at(a.st, a.stim_on[j + 1], ix, iy, iz) + mI) * a.inv_Cm;
            Yj[p] = u[0];
#pragma unroll
            for (int s = 1; s <= NA; ++s) { Gj[s * ld + p] = ha[s - 1]; Yj[s * ld + p] = u[s]; }
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int s = 1 + NA + g;
                Gj[s * ld + p] = lam[g] * (u[s] - yinf[g]);
                Yj[s * ld + p] = u[s];
            }
            a.FI[(int64_t)j * ld + p] = fi;
        }
#pragma unroll 1
        for (int g = 0; g < NG; ++g) {
            const double z = a.dt * lam[g];
            a.LAMN[(int64_t)g * ld + p] = lam[g];
            double aprev[M];
#pragma unroll
            for (int j = 0; j < M; ++j) aprev[j] = 0.0;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                double ph[M];
                phi_all<M>(C.c[i + 1] * z, ph);
                const double p1 = (i == 0) ? ph[0] : phi1(C.d[i + 1] * z);
                a.PHI[((int64_t)i * NG + g) * ld + p] = a.dtd[i + 1] * p1;      // dt d_i phi_1
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    double aij = 0.0;
#pragma unroll
                    for (int k = 0; k < M; ++k) aij = fma(C.B[i][j][k], ph[k], aij);
                    aij *= a.dt;                                                 // dt a_ij
                    a.S[(((int64_t)i * M + j) * NG + g) * ld + p] = aij - aprev[j];
                    aprev[j] = aij;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ sweep node i
// i in 1..M: ionic evaluation at y_{i-1}^{k+1} (i >= 2), G_{i-1}^{k+1}, FI_{i-1}^{k+1},
// explicit rows (auxiliaries, gates) of y_i^{k+1} and the right-hand side of the
// V row.  i == M+1: only the evaluation at y_M^{k+1}.  Each gate's rate is used
// as soon as it is computed (its G, Delta and update), which keeps few values live.
#ifndef ESDC_NODE_MINBLOCKS
#define ESDC_NODE_MINBLOCKS 5      // 5 x 128 threads per SM: at most 102 registers
#endif
template <class Model, int M>
__global__ void __launch_bounds__(128, ESDC_NODE_MINBLOCKS) k_node(StepArgs a)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const MeshDev& m = a.m;
    const int64_t ld = m.ld;
    const int i = a.i;
    const bool eval = i >= 2;                 // G at y_{i-1}^{k+1}
    const bool quad = i <= M;                 // explicit rows of y_i^{k+1}
    const int jm = i - 2;                     // 0-based index of node i-1
    const int ii = i - 1;                     // 0-based index of node i
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(m, p, ix, iy, iz);
        const double* src = eval ? a.Y + (int64_t)jm * NS * ld : a.yn;   // y_{i-1}^{k+1}
        double u[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) u[s] = src[s * ld + p];
        const double* Gp = a.Gold + (int64_t)jm * NS * ld;               // G_{i-1}^k
        double* Gq = a.Gnew + (int64_t)jm * NS * ld;                     // G_{i-1}^{k+1}
        double* Yi = a.Y + (int64_t)ii * NS * ld;
        const double dtd = quad ? a.dtd[i] : 0.0;

        // ---- V row and auxiliaries
        double dlt0 = 0.0, ha[NA > 0 ? NA : 1];
        if (eval) {
            const double fi = a.D * lap(m, src, p, ix, iy, iz);
            double mI;
            Model::currents(a.mp.p, u, mI, ha);
            const double fE = (stim_at(a.st, a.stim_on[i - 1], ix, iy, iz) + mI) * a.inv_Cm;
            const double fi_old = a.FI[(int64_t)jm * ld + p];
            a.FI[(int64_t)jm * ld + p] = fi;
            Gq[p] = fi + fE;
            dlt0 = fE - (Gp[p] - fi_old);
#pragma unroll
            for (int s = 1; s <= NA; ++s) Gq[s * ld + p] = ha[s - 1];
        }
        if (quad) {
            // Initial guess of the V_i solve: V_i^k moved by the change the previous
            // node just received, V_i^k + rho (V_{i-1}^{k+1} - V_{i-1}^k).  Only the
            // starting point of CG changes; the solution is the same.
            const double vik = Yi[p];
            if (eval) Yi[p] = fma(a.rho, u[0] - a.Vprev[p], vik);
            a.Vprev[p] = vik;
            double q = u[0];
#pragma unroll
            for (int j = 0; j < M; ++j) q = fma(a.dS0[ii][j], a.Gold[(int64_t)j * NS * ld + p], q);
            a.rhs[p] = fma(dtd, dlt0 - a.FI[(int64_t)ii * ld + p], q);
#pragma unroll
            for (int s = 1; s <= NA; ++s) {
                const double dl = eval ? ha[s - 1] - Gp[s * ld + p] : 0.0;
                double qa = u[s];
#pragma unroll
                for (int j = 0; j < M; ++j) qa = fma(a.dS0[ii][j], a.Gold[((int64_t)j * NS + s) * ld + p], qa);
                Yi[s * ld + p] = fma(dtd, dl, qa);
            }
        }
        // ---- gates, one at a time
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + NA + g;
            double dl = 0.0;
            if (eval) {
                double lam, yinf;
                Model::gate(a.mp.p, g, u[0], lam, yinf);
                const double gn = lam * (u[s] - yinf) + a.LAMN[(int64_t)g * ld + p] * (a.yn[s * ld + p] - u[s]);
                Gq[s * ld + p] = gn;
                dl = gn - Gp[s * ld + p];
            }
            if (quad) {
                double qg = u[s];
#pragma unroll
                for (int j = 0; j < M; ++j)
                    qg = fma(a.S[(((int64_t)ii * M + j) * NG + g) * ld + p],
                             a.Gold[((int64_t)j * NS + s) * ld + p], qg);
                Yi[s * ld + p] = fma(a.PHI[((int64_t)ii * NG + g) * ld + p], dl, qg);
            }
        }
    }
}

// ------------------------------------------------------------------ residual + output
// r_i = y_n + dt sum_j a_ij G_j - y_i (eq. def_C), accumulated over i from the row
// differences dt S_ij = dt (a_ij - a_{i-1,j});
// per-state max |r| and max |y|; y_{n+1} = y_M.
template <class Model, int M>
__global__ void __launch_bounds__(128) k_residual(StepArgs a)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const MeshDev& m = a.m;
    const ColloData& C = c_col[M - 1];
    const int64_t ld = m.ld;
    __shared__ double smax[2 * ESDC_NSMAX];
    for (int s = threadIdx.x; s < 2 * NS; s += blockDim.x) smax[s] = 0.0;
    __syncthreads();
    bool bad = false;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            const int g = s - 1 - NA;
            const double yns = a.yn[s * ld + p];
            double ymax = fabs(yns), rmax = 0.0;
            // r_i = r_{i-1} + sum_j dt S_ij G_j - (y_i - y_{i-1}), r_0 = 0 (y_0 = y_n)
            double r = 0.0, yprev = yns;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                double q = 0.0;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const double sij = (g >= 0) ? a.S[(((int64_t)i * M + j) * NG + g) * ld + p] : a.dS0[i][j];
                    q = fma(sij, a.Gold[((int64_t)j * NS + s) * ld + p], q);
                }
                const double yi = a.Y[((int64_t)i * NS + s) * ld + p];
                r += q - (yi - yprev);
                yprev = yi;
                if (a.R) a.R[((int64_t)i * NS + s) * ld + p] = r;
                bad |= !isfinite(r) || !isfinite(yi);
                rmax = fmax(rmax, fabs(r));
                ymax = fmax(ymax, fabs(yi));
            }
            // y_{n+1} = y_{n,M} (c_M = 1); y_n was read above by this thread only.
            a.yout[s * ld + p] = a.Y[((int64_t)(M - 1) * NS + s) * ld + p];
            // shared-memory max of non-negative doubles through their bit patterns
            atomicMax((unsigned long long*)&smax[s], (unsigned long long)__double_as_longlong(rmax));
            atomicMax((unsigned long long*)&smax[NS + s], (unsigned long long)__double_as_longlong(ymax));
        }
    }
    if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
    __syncthreads();
    for (int s = threadIdx.x; s < 2 * NS; s += blockDim.x)
        atomicMax(a.rmax + s, (unsigned long long)__double_as_longlong(smax[s]));
}

template <class Model>
__global__ void k_init(MeshDev m, ModelDev mp, double V0, double* y)
{
    constexpr int NS = Model::NS;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
        double u[NS];
        Model::rest(mp.p, V0, u);
        for (int s = 0; s < NS; ++s) y[s * m.ld + p] = u[s];
    }
}

template <class Model>
__global__ void k_ionic(MeshDev m, ModelDev mp, const double* y, double* fE, double* lam, double* yinf)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
        double u[NS], mI, ha[NA > 0 ? NA : 1], l[NG], yi[NG];
        for (int s = 0; s < NS; ++s) u[s] = y[s * m.ld + p];
        Model::eval(mp.p, u, mI, NA > 0 ? ha : nullptr, l, yi);
        fE[p] = mI; lam[p] = 0.0; yinf[p] = 0.0;
        for (int s = 1; s <= NA; ++s) { fE[s * m.ld + p] = ha[s - 1]; lam[s * m.ld + p] = 0.0; yinf[s * m.ld + p] = 0.0; }
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + NA + g;
            fE[s * m.ld + p] = 0.0; lam[s * m.ld + p] = l[g]; yinf[s * m.ld + p] = yi[g];
        }
    }
}

__global__ void k_math(const double* x, int64_t n, double* ex, double* rc)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        ex[e] = esdc::esdc_exp(x[e]);
        rc[e] = esdc::esdc_rcp(x[e]);
    }
}

template <int M>
__global__ void k_coef(const double* z, int64_t n, double* out)
{
    const ColloData& C = c_col[M - 1];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < M; ++i) {
            double ph[M];
            phi_all<M>(C.c[i + 1] * z[e], ph);
            for (int j = 0; j < M; ++j) {
                double aij = 0.0;
                for (int k = 0; k < M; ++k) aij = fma(C.B[i][j][k], ph[k], aij);
                out[((int64_t)i * M + j) * n + e] = aij;
            }
        }
    }
}

}  // namespace

// ====================================================================== host side

struct esdc_handle {
    int device = 0, sms = 152;
    int model = 0, NS = 0, NA = 0, NG = 0;
    ColloData col[ESDC_MMAX];
    MeshDev mesh{};
    StimDev stim{};
    ModelDev mp{};
    double sigma = 0, chi = 0, Cm = 0, D = 0;
    esdc_options opt{};
    // workspace
    double *Y = nullptr, *G0 = nullptr, *G1 = nullptr, *FI = nullptr, *S = nullptr, *PHI = nullptr,
           *LAMN = nullptr, *rhs = nullptr, *R = nullptr, *ydev = nullptr, *Vprev = nullptr;
    CgWork cg{};
    unsigned long long* rmax = nullptr;   // [2*NS]
    int* flags = nullptr;                 // [1]
    int* cg_log = nullptr;                // [K_log] iteration counts of the last step
    int cg_log_len = 0;
    // state of the most recent sweep
    int last_M = 0, last_K = 0;
    double last_dt = 0.0;
    const double* last_Gfinal = nullptr;
    cudaStream_t last_stream = nullptr;
    // kernel-class timing (esdc_profile): event pairs around each launch
    bool prof_on = false;
    cudaEvent_t prof_ev[2 * 512] = {};
    int prof_cls[512] = {};
    int prof_used = 0;
    double prof_ms[ESDC_PROF_CLASSES] = {};
    long long prof_cnt[ESDC_PROF_CLASSES] = {};
    char err[256] = {0};
};

namespace {

// Folds the recorded event pairs into the per-class totals (synchronises them).
cudaError_t prof_flush(esdc_handle* h)
{
    for (int k = 0; k < h->prof_used; ++k) {
        cudaError_t e = cudaEventSynchronize(h->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return e;
        h->prof_ms[h->prof_cls[k]] += ms;
        h->prof_cnt[h->prof_cls[k]] += 1;
    }
    h->prof_used = 0;
    return cudaSuccess;
}

inline void prof_begin(esdc_handle* h, int cls, cudaStream_t s)
{
    if (!h->prof_on) return;
    if (h->prof_used == 512) prof_flush(h);
    h->prof_cls[h->prof_used] = cls;
    cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
}

inline void prof_end(esdc_handle* h, cudaStream_t s)
{
    if (!h->prof_on) return;
    cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
    h->prof_used++;
}

std::mutex g_const_mu;
bool g_const_done[64] = {false};

int set_err(esdc_handle* h, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int set_err(esdc_handle* h, int code, const char* fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CUDA_TRY(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_err((h), e_ == cudaErrorMemoryAllocation ? ESDC_ERR_NO_MEMORY : ESDC_ERR_CUDA, \
                           "%s: %s", #call, cudaGetErrorString(e_));                           \
    } while (0)

int upload_constants(esdc_handle* h, int dev)
{
    std::lock_guard<std::mutex> lk(g_const_mu);
    if (dev >= 0 && dev < 64 && g_const_done[dev]) return ESDC_OK;
    ColloData col[ESDC_MMAX];
    for (int M = 1; M <= ESDC_MMAX; ++M)
        if (esdc_colloc_build(M, &col[M - 1]))
            return set_err(h, ESDC_ERR_CUDA, "collocation data for M=%d failed", M);
    double inv[ESDC_NSER], invf[ESDC_MMAX + 2];
    inv[0] = 0.0;
    for (int k = 1; k < ESDC_NSER; ++k) inv[k] = 1.0 / k;
    invf[0] = 1.0;
    for (int k = 1; k < ESDC_MMAX + 2; ++k) invf[k] = invf[k - 1] / k;
    CUDA_TRY(h, cudaMemcpyToSymbol(c_col, col, sizeof col));
    CUDA_TRY(h, cudaMemcpyToSymbol(c_inv, inv, sizeof inv));
    CUDA_TRY(h, cudaMemcpyToSymbol(c_invfact, invf, sizeof invf));
    if (dev >= 0 && dev < 64) g_const_done[dev] = true;
    return ESDC_OK;
}

int grid_for(const esdc_handle* h, int threads)
{
    long long need = ((long long)h->mesh.N + threads - 1) / threads;
    long long cap = (long long)h->sms * 16;
    return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

// Grid of a per-node kernel: the resident capacity of the device (blocks per SM
// from the occupancy calculator x SMs), so that the grid-stride loop spreads the
// nodes evenly over all SMs in one wave; smaller meshes use one block per 128 nodes.
template <class F>
int blocks_per_sm(F kernel, int threads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm;
}

int resident_grid(const esdc_handle* h, int per_sm, int threads)
{
    long long cap = (long long)h->sms * per_sm;
    long long need = ((long long)h->mesh.N + threads - 1) / threads;
    return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

template <class Model, int M>
cudaError_t launch_step_kernels(esdc_handle* h, StepArgs& a, double* y, int K, cudaStream_t s)
{
    const int T = 128;
    static int occ_setup = 0, occ_node = 0, occ_res = 0;    // blocks/SM per (model, M) instantiation
    if (!occ_setup) {
        occ_node = blocks_per_sm(k_node<Model, M>, T);
        occ_res = blocks_per_sm(k_residual<Model, M>, T);
        occ_setup = blocks_per_sm(k_setup<Model, M>, T);
    }
    const int nb_setup = resident_grid(h, occ_setup, T);
    const int nb_node = resident_grid(h, occ_node, T);
    const int nb_res = resident_grid(h, occ_res, T);
    const double g0 = h->D;   // operator scale: (I - dt d_i D L)
    const ColloData* C = &h->col[M - 1];

    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) a.dS0[i][j] = a.dt * C->S0[i][j];
    for (int i = 0; i <= M; ++i) {
        a.dtd[i] = a.dt * C->d[i];
        const double tj = a.t_n + C->c[i] * a.dt;
        unsigned on = 0;
        for (int b = 0; b < h->stim.nbox; ++b)
            if (tj >= h->stim.t_on[b] && tj < h->stim.t_off[b]) on |= 1u << b;
        a.stim_on[i] = on;
    }
    a.Gnew = h->G0;
    a.Gold = h->G0;
    prof_begin(h, 0, s);
    k_setup<Model, M><<<nb_setup, T, 0, s>>>(a);
    prof_end(h, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* Gold = h->G0;
    double* Gnew = h->G1;
    for (int k = 0; k < K; ++k) {
        a.Gold = Gold;
        a.Gnew = Gnew;
        for (int i = 1; i <= M + 1; ++i) {
            a.i = i;
            a.k = k;
            // first sweep: y^0 = y_n, so the change grows with the node time c_i
            a.rho = (i >= 2 && i <= M) ? (k == 0 ? C->c[i] / C->c[i - 1] : 1.0) : 0.0;
            prof_begin(h, 1, s);
            k_node<Model, M><<<nb_node, T, 0, s>>>(a);
            prof_end(h, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (i <= M) {
                double* Vi = h->Y + (int64_t)(i - 1) * h->NS * h->mesh.ld;
                const double g = a.dt * C->d[i] * g0;
                int* log = (k * M + (i - 1) < h->cg_log_len) ? h->cg_log + k * M + (i - 1) : nullptr;
                prof_begin(h, 2, s);
                e = esdc_cg_launch(h->mesh, h->cg, g, h->rhs, Vi, h->opt.tol_cg, h->opt.cg_maxit,
                                   h->opt.precond, log, h->flags, s);
                prof_end(h, s);
                if (e != cudaSuccess) return e;
            }
        }
        double* t = Gold; Gold = Gnew; Gnew = t;
    }
    a.Gold = Gold;
    a.yout = y;
    prof_begin(h, 3, s);
    k_residual<Model, M><<<nb_res, T, 0, s>>>(a);
    prof_end(h, s);
    h->last_Gfinal = Gold;
    return cudaGetLastError();
}

template <class Model>
cudaError_t dispatch_M(esdc_handle* h, StepArgs& a, double* y, int M, int K, cudaStream_t s)
{
    switch (M) {
        case 1: return launch_step_kernels<Model, 1>(h, a, y, K, s);
        case 2: return launch_step_kernels<Model, 2>(h, a, y, K, s);
        case 3: return launch_step_kernels<Model, 3>(h, a, y, K, s);
        case 4: return launch_step_kernels<Model, 4>(h, a, y, K, s);
        case 5: return launch_step_kernels<Model, 5>(h, a, y, K, s);
        case 6: return launch_step_kernels<Model, 6>(h, a, y, K, s);
        case 7: return launch_step_kernels<Model, 7>(h, a, y, K, s);
        case 8: return launch_step_kernels<Model, 8>(h, a, y, K, s);
        default: return cudaErrorInvalidValue;
    }
}

void free_all(esdc_handle* h)
{
    for (auto& e : h->prof_ev)
        if (e) cudaEventDestroy(e);
    void* ptrs[] = {h->Y, h->G0, h->G1, h->FI, h->S, h->PHI, h->LAMN, h->rhs, h->R, h->ydev, h->Vprev,
                    h->cg.r, h->cg.p, h->cg.q, h->cg.z, h->cg.part, h->cg.bar, h->cg.status,
                    h->rmax, h->flags, h->cg_log};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

void esdc_default_options(esdc_options* opt)
{
    if (!opt) return;
    opt->M_max = 8;
    opt->tol_cg = 1e-14;
    opt->cg_maxit = 200;
    opt->precond = 1;
}

int esdc_create(const esdc_mesh* mesh, double sigma, double chi, double Cm, int model,
                const double* params, int n_params, const esdc_options* opt, esdc_handle** out)
{
    if (!out) return ESDC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mesh || !params) return ESDC_ERR_INVALID_ARG;
    if (mesh->dim < 1 || mesh->dim > 3 || mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1)
        return ESDC_ERR_INVALID_ARG;
    if ((mesh->dim < 3 && mesh->nz != 1) || (mesh->dim < 2 && mesh->ny != 1)) return ESDC_ERR_INVALID_ARG;
    if (!(mesh->h > 0.0) || !std::isfinite(mesh->h)) return ESDC_ERR_INVALID_ARG;
    long long N = (long long)mesh->nx * mesh->ny * mesh->nz;
    if (N > 0x7fffffffLL - 64) return ESDC_ERR_INVALID_ARG;
    if (!(sigma >= 0.0) || !(chi > 0.0) || !(Cm > 0.0) || !std::isfinite(sigma) || !std::isfinite(chi) ||
        !std::isfinite(Cm))
        return ESDC_ERR_INVALID_ARG;
    int need = model == ESDC_MODEL_HH1952 ? 7 : model == ESDC_MODEL_SYN19 ? 88 : -1;
    if (need < 0 || n_params != need) return ESDC_ERR_INVALID_ARG;
    for (int k = 0; k < n_params; ++k)
        if (!std::isfinite(params[k])) return ESDC_ERR_INVALID_ARG;
    if (model == ESDC_MODEL_SYN19) {
        for (int q = 0; q < 12; ++q)
            if (params[6 * q + 1] == 0.0 || params[6 * q + 5] == 0.0 || !(params[6 * q + 2] > 0.0))
                return ESDC_ERR_INVALID_ARG;
        for (int l = 0; l < 6; ++l)
            if (!(params[82 + l] > 0.0)) return ESDC_ERR_INVALID_ARG;
    }
    esdc_options o;
    esdc_default_options(&o);
    if (opt) o = *opt;
    if (o.M_max < 1 || o.M_max > ESDC_MMAX || !(o.tol_cg >= 0.0) || o.cg_maxit < 1) return ESDC_ERR_INVALID_ARG;

    esdc_handle* h = new (std::nothrow) esdc_handle();
    if (!h) return ESDC_ERR_NO_MEMORY;
    h->opt = o;
    h->model = model;
    h->NS = model == ESDC_MODEL_HH1952 ? 4 : 19;
    h->NG = model == ESDC_MODEL_HH1952 ? 3 : 12;
    h->NA = h->NS - 1 - h->NG;
    h->sigma = sigma; h->chi = chi; h->Cm = Cm;
    h->D = sigma / (chi * Cm);
    h->mesh.nx = mesh->nx; h->mesh.ny = mesh->ny; h->mesh.nz = mesh->nz;
    h->mesh.N = (int)N;
    h->mesh.ld = (N + 31) / 32 * 32;
    h->mesh.ih2 = 1.0 / (mesh->h * mesh->h);
    for (int k = 0; k < n_params; ++k) h->mp.p[k] = params[k];
    if (model == ESDC_MODEL_SYN19) {             // reciprocals of the constant divisors
        for (int q = 0; q < 12; ++q) {
            h->mp.p[88 + q] = 1.0 / params[6 * q + 1];
            h->mp.p[100 + q] = 1.0 / params[6 * q + 5];
        }
        for (int l = 0; l < 6; ++l) h->mp.p[112 + l] = 1.0 / params[82 + l];
    }

    int rc = ESDC_OK;
    auto fail = [&](int code) { free_all(h); delete h; return code; };
    for (int M = 1; M <= ESDC_MMAX; ++M)
        if (esdc_colloc_build(M, &h->col[M - 1])) return fail(ESDC_ERR_CUDA);
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(ESDC_ERR_CUDA);
    if ((rc = upload_constants(h, h->device)) != ESDC_OK) return fail(rc);

    const int64_t ld = h->mesh.ld, NS = h->NS, NG = h->NG, Mx = o.M_max;
    struct { double** p; int64_t n; } bufs[] = {
        {&h->Y, Mx * NS * ld}, {&h->G0, Mx * NS * ld}, {&h->G1, Mx * NS * ld}, {&h->FI, Mx * ld},
        {&h->S, Mx * Mx * NG * ld}, {&h->PHI, Mx * NG * ld}, {&h->LAMN, NG * ld}, {&h->rhs, ld},
        {&h->Vprev, ld},
        {&h->cg.r, ld}, {&h->cg.p, ld}, {&h->cg.q, ld}, {&h->cg.z, ld}};
    for (auto& b : bufs) {
        cudaError_t e = cudaMalloc((void**)b.p, sizeof(double) * b.n);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? ESDC_ERR_NO_MEMORY : ESDC_ERR_CUDA);
        cudaMemset(*b.p, 0, sizeof(double) * b.n);
    }
    h->cg.threads = ESDC_CG_THREADS;
    h->cg.max_blocks = esdc_cg_blocks(h->mesh, h->cg.threads);
    if (h->cg.max_blocks < 1) return fail(ESDC_ERR_CUDA);
    if (cudaMalloc((void**)&h->cg.part, sizeof(double) * 6 * h->cg.max_blocks) != cudaSuccess ||
        cudaMalloc((void**)&h->cg.bar, sizeof(unsigned) * 2) != cudaSuccess ||
        cudaMalloc((void**)&h->cg.status, sizeof(int) * 2) != cudaSuccess ||
        cudaMalloc((void**)&h->rmax, sizeof(unsigned long long) * 2 * ESDC_NSMAX) != cudaSuccess ||
        cudaMalloc((void**)&h->flags, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&h->cg_log, sizeof(int) * 64 * ESDC_MMAX) != cudaSuccess)
        return fail(ESDC_ERR_NO_MEMORY);
    h->cg_log_len = 64 * ESDC_MMAX;
    cudaMemset(h->cg.bar, 0, sizeof(unsigned) * 2);
    cudaMemset(h->cg.status, 0, sizeof(int) * 2);
    cudaMemset(h->flags, 0, sizeof(int));
    cudaMemset(h->cg_log, 0, sizeof(int) * h->cg_log_len);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(ESDC_ERR_CUDA);
    *out = h;
    return ESDC_OK;
}

void esdc_destroy(esdc_handle* h)
{
    if (!h) return;
    free_all(h);
    delete h;
}

const char* esdc_last_error(const esdc_handle* h) { return h ? h->err : "null handle"; }

int esdc_set_stimulus(esdc_handle* h, int nbox, const int* box, const double* amp,
                      const double* t_on, const double* t_off)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (nbox < 0 || nbox > ESDC_MAXBOX) return set_err(h, ESDC_ERR_INVALID_ARG, "nbox out of range");
    if (nbox > 0 && (!box || !amp || !t_on || !t_off)) return set_err(h, ESDC_ERR_INVALID_ARG, "null stimulus array");
    StimDev st{};
    st.nbox = nbox;
    for (int b = 0; b < nbox; ++b) {
        for (int k = 0; k < 6; ++k) st.box[b][k] = box[6 * b + k];
        if (!std::isfinite(amp[b]) || std::isnan(t_on[b]) || std::isnan(t_off[b]))
            return set_err(h, ESDC_ERR_INVALID_ARG, "non-finite stimulus value");
        st.amp[b] = amp[b]; st.t_on[b] = t_on[b]; st.t_off[b] = t_off[b];
    }
    h->stim = st;
    return ESDC_OK;
}

int esdc_state_size(const esdc_handle* h, int* n_state, int64_t* n_nodes, int64_t* ld)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (n_state) *n_state = h->NS;
    if (n_nodes) *n_nodes = h->mesh.N;
    if (ld) *ld = h->mesh.ld;
    return ESDC_OK;
}

int esdc_init_state(esdc_handle* h, double* y, double V0, void* stream)
{
    if (!h || !y || !std::isfinite(V0)) return ESDC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = grid_for(h, 128);
    if (h->model == ESDC_MODEL_HH1952) k_init<esdc::HH1952><<<nb, 128, 0, s>>>(h->mesh, h->mp, V0, y);
    else k_init<esdc::SYN19><<<nb, 128, 0, s>>>(h->mesh, h->mp, V0, y);
    CUDA_TRY(h, cudaGetLastError());
    return ESDC_OK;
}

int esdc_sweep(esdc_handle* h, double* y, double t, double dt, int M, int K, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!y) return set_err(h, ESDC_ERR_INVALID_ARG, "y is null");
    if (M < 1 || M > h->opt.M_max) return set_err(h, ESDC_ERR_INVALID_ARG, "M=%d outside 1..%d", M, h->opt.M_max);
    if (K < 0 || K > 64) return set_err(h, ESDC_ERR_INVALID_ARG, "K=%d outside 0..64", K);
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t)) return set_err(h, ESDC_ERR_INVALID_ARG, "bad t/dt");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(h, cudaMemsetAsync(h->rmax, 0, sizeof(unsigned long long) * 2 * ESDC_NSMAX, s));
    CUDA_TRY(h, cudaMemsetAsync(h->flags, 0, sizeof(int), s));
    CUDA_TRY(h, cudaMemsetAsync(h->cg_log, 0, sizeof(int) * h->cg_log_len, s));
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.m = h->mesh; a.st = h->stim; a.mp = h->mp;
    a.dt = dt; a.t_n = t; a.D = h->D; a.inv_Cm = 1.0 / h->Cm;
    a.yn = y; a.Y = h->Y; a.FI = h->FI; a.S = h->S; a.PHI = h->PHI; a.LAMN = h->LAMN; a.rhs = h->rhs;
    a.R = h->R; a.rmax = h->rmax; a.flags = h->flags; a.Vprev = h->Vprev;
    cudaError_t e = h->model == ESDC_MODEL_HH1952 ? dispatch_M<esdc::HH1952>(h, a, y, M, K, s)
                                                  : dispatch_M<esdc::SYN19>(h, a, y, M, K, s);
    if (e != cudaSuccess) return set_err(h, ESDC_ERR_CUDA, "step launch: %s", cudaGetErrorString(e));
    h->last_M = M; h->last_K = K; h->last_dt = dt; h->last_stream = s;
    return ESDC_OK;
}

int esdc_sweep_host(esdc_handle* h, double* y_host, int64_t ld_host, double t, double dt, int M, int K,
                    void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!y_host || ld_host < h->mesh.N) return set_err(h, ESDC_ERR_INVALID_ARG, "bad host buffer");
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->ydev) CUDA_TRY(h, cudaMalloc((void**)&h->ydev, sizeof(double) * h->NS * h->mesh.ld));
    const size_t row = sizeof(double) * h->mesh.N;
    CUDA_TRY(h, cudaMemcpy2DAsync(h->ydev, sizeof(double) * h->mesh.ld, y_host, sizeof(double) * ld_host, row,
                                  h->NS, cudaMemcpyHostToDevice, s));
    int rc = esdc_sweep(h, h->ydev, t, dt, M, K, stream);
    if (rc) return rc;
    CUDA_TRY(h, cudaMemcpy2DAsync(y_host, sizeof(double) * ld_host, h->ydev, sizeof(double) * h->mesh.ld, row,
                                  h->NS, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return ESDC_OK;
}

int esdc_residual(esdc_handle* h, double* res_inf, double* y_inf, double* res_state)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!h->last_M) return set_err(h, ESDC_ERR_INVALID_ARG, "no sweep yet");
    CUDA_TRY(h, cudaStreamSynchronize(h->last_stream));
    unsigned long long bits[2 * ESDC_NSMAX];
    int flags = 0;
    CUDA_TRY(h, cudaMemcpy(bits, h->rmax, sizeof bits, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(&flags, h->flags, sizeof flags, cudaMemcpyDeviceToHost));
    double rmax = 0.0, ymax = 0.0;
    for (int s = 0; s < h->NS; ++s) {
        double r, yv;
        std::memcpy(&r, &bits[s], 8);
        std::memcpy(&yv, &bits[h->NS + s], 8);
        if (res_state) res_state[s] = r;
        rmax = std::fmax(rmax, r);
        ymax = std::fmax(ymax, yv);
    }
    if (res_inf) *res_inf = rmax;
    if (y_inf) *y_inf = ymax;
    if (flags & ESDC_FLAG_TIMEOUT) return set_err(h, ESDC_ERR_DEVICE_TIMEOUT, "a device-side wait timed out");
    if (flags & ESDC_FLAG_NONFINITE) return set_err(h, ESDC_ERR_NONFINITE, "non-finite residual or state");
    if (flags & ESDC_FLAG_CG_MAXIT) return set_err(h, ESDC_ERR_CG_NOT_CONVERGED, "a diffusion solve hit cg_maxit");
    return ESDC_OK;
}

int esdc_stats(esdc_handle* h, int* cg_iters, int n)
{
    if (!h || !cg_iters || n < 0) return ESDC_ERR_INVALID_ARG;
    if (!h->last_M) return set_err(h, ESDC_ERR_INVALID_ARG, "no sweep yet");
    CUDA_TRY(h, cudaStreamSynchronize(h->last_stream));
    int cnt = h->last_K * h->last_M;
    if (cnt > h->cg_log_len) cnt = h->cg_log_len;
    if (n < cnt) cnt = n;
    CUDA_TRY(h, cudaMemcpy(cg_iters, h->cg_log, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
    return ESDC_OK;
}

int esdc_collocation(esdc_handle* h, double* y_out, double* r_out, void* stream)
{
    if (!h || !y_out) return ESDC_ERR_INVALID_ARG;
    if (!h->last_M) return set_err(h, ESDC_ERR_INVALID_ARG, "no sweep yet");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * h->last_M * h->NS * h->mesh.ld;
    CUDA_TRY(h, cudaMemcpyAsync(y_out, h->Y, bytes, cudaMemcpyDeviceToDevice, s));
    if (r_out) {
        if (!h->R) return set_err(h, ESDC_ERR_INVALID_ARG, "residual vectors were not kept; call esdc_keep_residual first");
        CUDA_TRY(h, cudaMemcpyAsync(r_out, h->R, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return ESDC_OK;
}

int esdc_coefficients(esdc_handle* h, const double* z, int64_t n, int M, double* a, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!z || !a || n < 0 || M < 1 || M > ESDC_MMAX) return set_err(h, ESDC_ERR_INVALID_ARG, "bad coefficient args");
    if (n == 0) return ESDC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long nb = (n + 127) / 128;
    if (nb > 152 * 16) nb = 152 * 16;
    switch (M) {
        case 1: k_coef<1><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 2: k_coef<2><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 3: k_coef<3><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 4: k_coef<4><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 5: k_coef<5><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 6: k_coef<6><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 7: k_coef<7><<<(int)nb, 128, 0, s>>>(z, n, a); break;
        case 8: k_coef<8><<<(int)nb, 128, 0, s>>>(z, n, a); break;
    }
    CUDA_TRY(h, cudaGetLastError());
    return ESDC_OK;
}

int esdc_diffusion_solve(esdc_handle* h, double g, const double* b, double* x, int* iters, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!b || !x || !(g >= 0.0) || !std::isfinite(g)) return set_err(h, ESDC_ERR_INVALID_ARG, "bad solve args");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(h, cudaMemsetAsync(h->flags, 0, sizeof(int), s));
    CUDA_TRY(h, esdc_cg_launch(h->mesh, h->cg, g, b, x, h->opt.tol_cg, h->opt.cg_maxit, h->opt.precond,
                               nullptr, h->flags, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    int st[2] = {0, 0}, flags = 0;
    CUDA_TRY(h, cudaMemcpy(st, h->cg.status, sizeof st, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(&flags, h->flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (iters) *iters = st[0];
    if (flags & ESDC_FLAG_TIMEOUT) return set_err(h, ESDC_ERR_DEVICE_TIMEOUT, "CG grid barrier timed out");
    if (flags & ESDC_FLAG_NONFINITE) return set_err(h, ESDC_ERR_NONFINITE, "non-finite CG residual");
    if (flags & ESDC_FLAG_CG_MAXIT) return set_err(h, ESDC_ERR_CG_NOT_CONVERGED, "CG hit cg_maxit");
    return ESDC_OK;
}

int esdc_ionic(esdc_handle* h, const double* y, double* fE, double* lam, double* yinf, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!y || !fE || !lam || !yinf) return set_err(h, ESDC_ERR_INVALID_ARG, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = grid_for(h, 128);
    if (h->model == ESDC_MODEL_HH1952) k_ionic<esdc::HH1952><<<nb, 128, 0, s>>>(h->mesh, h->mp, y, fE, lam, yinf);
    else k_ionic<esdc::SYN19><<<nb, 128, 0, s>>>(h->mesh, h->mp, y, fE, lam, yinf);
    CUDA_TRY(h, cudaGetLastError());
    return ESDC_OK;
}

int esdc_math_check(const double* x, int64_t n, double* ex, double* rc, void* stream)
{
    if (!x || !ex || !rc || n < 0) return ESDC_ERR_INVALID_ARG;
    if (n == 0) return ESDC_OK;
    long long nb = (n + 255) / 256;
    if (nb > 4096) nb = 4096;
    k_math<<<(int)nb, 256, 0, (cudaStream_t)stream>>>(x, n, ex, rc);
    return cudaGetLastError() == cudaSuccess ? ESDC_OK : ESDC_ERR_CUDA;
}

int esdc_profile(esdc_handle* h, int enable)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (enable && !h->prof_ev[0])
        for (auto& e : h->prof_ev) CUDA_TRY(h, cudaEventCreate(&e));
    if (!enable && h->prof_on) CUDA_TRY(h, prof_flush(h));
    h->prof_on = enable != 0;
    return ESDC_OK;
}

int esdc_profile_read(esdc_handle* h, double* ms, long long* launches)
{
    if (!h || !ms || !launches) return ESDC_ERR_INVALID_ARG;
    CUDA_TRY(h, prof_flush(h));
    for (int c = 0; c < ESDC_PROF_CLASSES; ++c) {
        ms[c] = h->prof_ms[c];
        launches[c] = h->prof_cnt[c];
        h->prof_ms[c] = 0.0;
        h->prof_cnt[c] = 0;
    }
    return ESDC_OK;
}

int esdc_keep_residual(esdc_handle* h, int keep)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (keep && !h->R) {
        CUDA_TRY(h, cudaMalloc((void**)&h->R, sizeof(double) * h->opt.M_max * h->NS * h->mesh.ld));
    } else if (!keep && h->R) {
        cudaFree(h->R);
        h->R = nullptr;
    }
    return ESDC_OK;
}

}  // extern "C"
