// Device side of the HSDC step, shared by the translation units that
// instantiate it (esdc_step.cu: FP64; esdc_step_mixed.cu: precision form).
#pragma once
#include <cmath>

#include "esdc_handle.h"
#include "esdc_models.cuh"

namespace {

// Each translation unit that includes this header owns a copy of these
// constants and uploads it with upload_constants_local().
static __constant__ ColloData c_col[ESDC_MMAX];     // index M-1
static __constant__ double c_inv[ESDC_NSER];        // c_inv[m] = 1/m (c_inv[0] unused)
static __constant__ double c_invfact[ESDC_MMAX + 2];



__device__ __forceinline__ void node_xyz(const MeshDev& m, int p, int& ix, int& iy, int& iz)
{
    int r = p / m.nx;
    ix = p - r * m.nx;
    iz = r / m.ny;
    iy = r - iz * m.ny;
}

// The fourth-order difference of the paper's experiments (Sec. 5) along one
// axis, (-v_{i-2} + 16 v_{i-1} - 30 v_i + 16 v_{i+1} - v_{i+2}), mirrored ghost
// cells; an axis of one cell contributes nothing.
__device__ __forceinline__ double axis4(const double* v, int p, int i, int n, int stride)
{
    if (n == 1) return 0.0;
    const double a = v[p + (esdc_mirror(i - 2, n) - i) * stride], b = v[p + (esdc_mirror(i - 1, n) - i) * stride];
    const double c = v[p + (esdc_mirror(i + 1, n) - i) * stride], d = v[p + (esdc_mirror(i + 2, n) - i) * stride];
    return fma(16.0, b + c, -(a + d)) - 30.0 * v[p];
}

// Sum over the axes of axis4 (times 1/(12 h^2) it is the fourth-order Laplacian).
__device__ __forceinline__ double lap4(const double* v, int p, int ix, int iy, int iz, int nx, int ny, int nz)
{
    return axis4(v, p, ix, nx, 1) + axis4(v, p, iy, ny, nx) + axis4(v, p, iz, nz, nx * ny);
}

// L v at node p: (1/h^2) sum over in-domain neighbours of (v_q - v_p); with a
// layered conductivity, A v (the coefficients then include sigma and 1/h^2,
// and the in-plane diagonal neighbours carry the sigma_xy cross term); with a
// per-node conductivity field, A v with face conductivities (sigma_p + sigma_q)/2.
__device__ __forceinline__ double lap(const MeshDev& m, const double* __restrict__ v, int p,
                                      int ix, int iy, int iz)
{
    const double vp = v[p];
    const int sxy = m.nx * m.ny;
    if (m.sig) {                       // (A v)_p = (1/h^2) sum_q (sigma_p + sigma_q)/2 (v_q - v_p)
        const double sp = __ldg(m.sig + p);
        double s = 0.0;
        if (ix > 0)        s = fma(sp + __ldg(m.sig + p - 1), v[p - 1] - vp, s);
        if (ix < m.nx - 1) s = fma(sp + __ldg(m.sig + p + 1), v[p + 1] - vp, s);
        if (iy > 0)        s = fma(sp + __ldg(m.sig + p - m.nx), v[p - m.nx] - vp, s);
        if (iy < m.ny - 1) s = fma(sp + __ldg(m.sig + p + m.nx), v[p + m.nx] - vp, s);
        if (iz > 0)        s = fma(sp + __ldg(m.sig + p - sxy), v[p - sxy] - vp, s);
        if (iz < m.nz - 1) s = fma(sp + __ldg(m.sig + p + sxy), v[p + sxy] - vp, s);
        return 0.5 * m.ih2 * s;
    }
    if (m.lay) {
        const double cxx = __ldg(m.lay + iz), cyy = __ldg(m.lay + m.nz + iz), cd = __ldg(m.lay + 2 * m.nz + iz);
        double s = 0.0;
        if (ix > 0)        s = fma(cxx, v[p - 1] - vp, s);
        if (ix < m.nx - 1) s = fma(cxx, v[p + 1] - vp, s);
        if (iy > 0)        s = fma(cyy, v[p - m.nx] - vp, s);
        if (iy < m.ny - 1) s = fma(cyy, v[p + m.nx] - vp, s);
        if (iz > 0)        s = fma(__ldg(m.lay + 3 * m.nz + iz - 1), v[p - sxy] - vp, s);
        if (iz < m.nz - 1) s = fma(__ldg(m.lay + 3 * m.nz + iz), v[p + sxy] - vp, s);
        const bool xm = ix > 0, xp = ix < m.nx - 1, ym = iy > 0, yp = iy < m.ny - 1;
        double c = 0.0;
        if (xp && yp) c += v[p + 1 + m.nx] - vp;
        if (xm && ym) c += v[p - 1 - m.nx] - vp;
        if (xp && ym) c -= v[p + 1 - m.nx] - vp;
        if (xm && yp) c -= v[p - 1 + m.nx] - vp;
        return fma(cd, c, s);
    }
    if (m.order == 4) return lap4(v, p, ix, iy, iz, m.nx, m.ny, m.nz) * (m.ih2 * (1.0 / 12.0));
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

// Order tests of non-negative doubles on their bit patterns: for a, b >= 0 (or
// -0), a <= b exactly when the patterns compare so as signed 64-bit integers.
// Integer compares run on the ALU pipe; the FP64 pipe is the scarce unit.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }

// phi_1(y) = (e^y - 1)/y for y <= 0: below -1/2 directly (e^y - 1 keeps at least
// 1 - e^{-1/2} of its magnitude, so about 3 ulp); above, the reciprocal of
// x/(e^x - 1) from its Bernoulli series.
__device__ __forceinline__ double phi1(double y)
{
    if (dbits(-y) > dbits(0.5)) return (esdc::esdc_exp(y) - 1.0) * esdc::esdc_rcp(y);   // y < -1/2
    return (dbits(y) << 1) == 0 ? 1.0 : esdc::esdc_rcp(esdc::x_over_expm1(y));          // y = +-0
}

// phi_1..phi_M at x <= 0 (App. A eq. def_phik).  Two regimes:
//  |x| >  X1: phi_1 = (e^x - 1)/x (no cancellation there: X1 > 1.4 for M >= 2),
//             then phi_{k+1} = (phi_k - 1/k!)/x;
//  |x| <= X1: phi_M = e^x/(M-1)! sum_m (-x)^m/(m! (m+M)) (all terms >= 0,
//             Horner form with host coefficients; the number of terms steps
//             down with |x|), then phi_k = x phi_{k+1} + 1/k!.
// X1 balances the rounding growth of the two recurrences (set on the host).
// M = 1: phi_1 as in phi1().
template <int M>
__device__ __forceinline__ void phi_all(double x, double (&ph)[M])
{
    const ColloData& C = c_col[M - 1];
    const double nx = -x;
    const long long nbits = dbits(nx);
    if (M == 1) {
        ph[0] = phi1(x);
    } else if (nbits > dbits(C.X1)) {                     // -x > X1
        const double rx = esdc::esdc_rcp(x);
        ph[0] = (esdc::esdc_exp(x) - 1.0) * rx;
#pragma unroll
        for (int k = 1; k < M; ++k) ph[k] = (ph[k - 1] - c_invfact[k]) * rx;
    } else {
        const int n = nbits <= dbits(C.xb[0]) ? C.nb[0] : nbits <= dbits(C.xb[1]) ? C.nb[1]
                    : nbits <= dbits(C.xb[2]) ? C.nb[2] : nbits <= dbits(C.xb[3]) ? C.nb[3] : C.nb[4];
        double acc = C.ser[n];
        for (int m = n - 1; m >= 0; --m) acc = fma(acc, nx, C.ser[m]);
        ph[M - 1] = esdc::esdc_exp(x) * acc;
#pragma unroll
        for (int k = M - 1; k >= 1; --k) ph[k - 1] = fma(x, ph[k], c_invfact[k]);
    }
}


// ------------------------------------------------------------------ set-up
// Lambda_n, dt S_ij(dt Lambda_n), dt d_i phi_1(d_i dt Lambda_n) (tables carry the
// step size); y^0 = 1 (x) y_n; G_j^0 = g_n(t_{n,j}, y_n); FI_j^0 = f_I(y_n).
// Batched form: nodes of a ragged batch of meshes, concatenated in ESDC_TILE-node
// tiles; the tissue of a node is found from its tile.
struct BatchNode {
    MeshDev m;               // the node's own mesh (ld: the pitch of the concatenated arrays)
    const TissueDev* T;
    const unsigned* on;      // stimulus window bits of the tissue, per collocation time
    int ix, iy, iz;
};

__device__ __forceinline__ bool batch_node(const StepArgs& a, int p, BatchNode& n)
{
    const int b = __ldg(a.tile_tissue + (p >> ESDC_TILE_SHIFT));
    const TissueDev* T = a.tis + b;
    const int q = p - (int)T->off;
    if (q >= T->N) return false;              // padding at the end of the tissue's last tile
    n.m = a.m;
    n.m.nx = T->nx; n.m.ny = T->ny; n.m.nz = T->nz; n.m.N = T->N; n.m.ih2 = T->ih2;
    n.m.lay = nullptr; n.m.wdiag = nullptr; n.m.layf = nullptr;
    n.T = T;
    n.on = a.tis_on + (size_t)b * (ESDC_MMAX + 1);
    node_xyz(n.m, q, n.ix, n.iy, n.iz);
    return true;
}

// The values that change from one launch of a step's sequence to the next:
// the collocation node i of a node launch, its warm-start weight, the sweep's
// G buffers (G^k read, G^{k+1} written) and the residual's output.  The
// launch-sequence kernels take them from their StepArgs; the persistent step
// kernel of the batches passes its own for each phase.
struct PhaseArgs {
    int i;
    double rho;
    const double* Gold;
    double* Gnew;
    double* yout;
};
__device__ __forceinline__ PhaseArgs phase_of(const StepArgs& a) { return PhaseArgs{a.i, a.rho, a.Gold, a.Gnew, a.yout}; }

// One function of the set-up table (esdc_ztab.cpp) at t: Horner's rule on its
// ESDC_ZTAB_NC coefficients.
__device__ __forceinline__ double ztab_poly(const double* __restrict__ c, double t)
{
    double r = __ldg(c + ESDC_ZTAB_NC - 1);
#pragma unroll
    for (int k = ESDC_ZTAB_NC - 2; k >= 0; --k) r = fma(r, t, __ldg(c + k));
    return r;
}

// Per-step tables of gate g at node p: Lambda_n, dt d_i phi_1(d_i dt Lambda_n)
// and dt S_ij(dt Lambda_n) (App. A).  From the set-up table when there is one
// and z = dt Lambda_n lies in its range (1 <= y = 1 - z < 2^ESDC_ZTAB_OCT: the
// interval is y's exponent and leading mantissa bits), else directly.
template <int M>
__device__ __forceinline__ void gate_tables(const StepArgs& a, int g, int NG, double lam, int p)
{
    const ColloData& C = c_col[M - 1];
    const int64_t ld = a.m.ld;
    const double z = a.dt * lam;
    a.LAMN[(int64_t)g * ld + p] = lam;
    if (a.ztab) {
        const double y = 1.0 - z;
        const long long bits = __double_as_longlong(y);
        const int e = (int)(bits >> 52) - 1023;             // NaN, Inf and y < 1 fall outside
        if (e >= 0 && e < ESDC_ZTAB_OCT) {
            const int r = (e << ESDC_ZTAB_SUB) + (int)((bits >> (52 - ESDC_ZTAB_SUB)) & ((1 << ESDC_ZTAB_SUB) - 1));
            const double* row = a.ztab + (size_t)r * ESDC_ZTAB_ROW(M);
            const double t = y - __ldg(row);
            const double* c = row + 2;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                a.PHI[((int64_t)i * NG + g) * ld + p] = ztab_poly(c + (i * (M + 1)) * ESDC_ZTAB_NC, t);
#pragma unroll
                for (int j = 0; j < M; ++j)
                    a.S[(((int64_t)i * M + j) * NG + g) * ld + p] =
                        ztab_poly(c + (i * (M + 1) + 1 + j) * ESDC_ZTAB_NC, t);
            }
            return;
        }
    }
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
            double aij = 0.0;                                            // dt a_ij
#pragma unroll
            for (int k = 0; k < M; ++k) aij = fma(a.dtB[i][j][k], ph[k], aij);
            a.S[(((int64_t)i * M + j) * NG + g) * ld + p] = aij - aprev[j];
            aprev[j] = aij;
        }
    }
}

// Set-up from a given iterate (the Q^par iteration of Sec. 3.2): y_{n,0} = y_n
// is new, y_{n,1..M} are the iterate in Y.  Lambda_n = Lambda(y_n) and the
// tables as in the plain set-up; G_j = g_n(t_{n,j}, y_j) and FI_j = f_I(y_j) on
// the iterate (the plain set-up's G^0 with y_j in place of y_n).
template <class Model, int M>
__device__ __forceinline__ void setup_iter_body(const StepArgs& a, const PhaseArgs& ph, const MeshDev& m,
                                                const StimDev& st, const unsigned* on, double D, int p, int ix,
                                                int iy, int iz)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const int64_t ld = a.m.ld;
    const double vn = a.yn[p];
    const typename Model::VCtx vcn = Model::vctx(a.mp, vn);
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
        double lam, b;
        Model::gate_lb(a.mp.p, vcn, g, vn, lam, b);
        gate_tables<M>(a, g, NG, lam, p);
    }
#pragma unroll 1
    for (int j = 0; j < M; ++j) {
        const double* Yj = a.Y + (int64_t)j * NS * ld;
        double* Gj = ph.Gnew + (int64_t)j * NS * ld;
        double u[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) u[s] = Yj[s * ld + p];
        const double fi = D * lap(m, Yj, p, ix, iy, iz);
        double mI, ha[NA > 0 ? NA : 1];
        Model::currents(a.mp.p, u, mI, ha);
        Gj[p] = fi + (stim_at(st, on[j + 1], ix, iy, iz) + mI) * a.inv_Cm;
#pragma unroll
        for (int s = 1; s <= NA; ++s) Gj[s * ld + p] = ha[s - 1];
        a.FI[(int64_t)j * ld + p] = fi;
        const typename Model::VCtx vc = Model::vctx(a.mp, u[0]);
#pragma unroll 1
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + NA + g;
            double lam, b;
            Model::gate_lb(a.mp.p, vc, g, u[0], lam, b);
            Gj[s * ld + p] = fma(a.LAMN[(int64_t)g * ld + p], a.yn[s * ld + p] - u[s], fma(lam, u[s], b));
        }
    }
}

template <class Model, int M, bool MIXED>
__device__ __forceinline__ void setup_body(const StepArgs& a, const PhaseArgs& ph, const MeshDev& m,
                                           const StimDev& st, const unsigned* on, double D, int p, int ix, int iy,
                                           int iz)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const int64_t ld = a.m.ld;
    double u[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) u[s] = a.yn[s * ld + p];
    const double fi = D * lap(m, a.yn, p, ix, iy, iz);
    double mI, ha[NA > 0 ? NA : 1];
    float uf[NS];
    if (MIXED) {
#pragma unroll
        for (int s = 0; s < NS; ++s) uf[s] = (float)u[s];
        float mIf, haf[NA > 0 ? NA : 1];
        Model::currents_f(a.mpf.p, uf, mIf, haf);
        mI = mIf;
#pragma unroll
        for (int s = 0; s < NA; ++s) ha[s] = haf[s];
    } else {
        Model::currents(a.mp.p, u, mI, ha);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double* Yj = a.Y + (int64_t)j * NS * ld;
        double* Gj = ph.Gnew + (int64_t)j * NS * ld;
        Gj[p] = fi + (stim_at(st, on[j + 1], ix, iy, iz) + mI) * a.inv_Cm;
        Yj[p] = u[0];
#pragma unroll
        for (int s = 1; s <= NA; ++s) { Gj[s * ld + p] = ha[s - 1]; Yj[s * ld + p] = u[s]; }
        a.FI[(int64_t)j * ld + p] = fi;
    }
    const typename Model::VCtx vc = Model::vctx(a.mp, u[0]);
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
        const int s = 1 + NA + g;
        const double us = a.yn[s * ld + p];
        double lam, g0;                          // g0 = Lambda (u - w_inf) = Lambda u + b
        if (MIXED) {
            float lf, yf;
            Model::gate_f(a.mpf.p, g, uf[0], lf, yf);
            lam = lf;
            g0 = lam * (us - (double)yf);
        } else {
            double b;
            Model::gate_lb(a.mp.p, vc, g, u[0], lam, b);
            g0 = fma(lam, us, b);
        }
#pragma unroll
        for (int j = 0; j < M; ++j) {
            ph.Gnew[((int64_t)j * NS + s) * ld + p] = g0;
            a.Y[((int64_t)j * NS + s) * ld + p] = us;
        }
        gate_tables<M>(a, g, NG, lam, p);
    }
}

#ifndef ESDC_SETUP_MINBLOCKS
#define ESDC_SETUP_MINBLOCKS 5     // blocks of 128 threads per SM the register budget must allow (96 registers)
#endif
// ------------------------------------------------------------------ sweep node i
// i in 1..M: ionic evaluation at y_{i-1}^{k+1} (i >= 2), G_{i-1}^{k+1}, FI_{i-1}^{k+1},
// explicit rows (auxiliaries, gates) of y_i^{k+1} and the right-hand side of the
// V row.  i == M+1: only the evaluation at y_M^{k+1}.  Each gate's rate is used
// as soon as it is computed (its G, Delta and update), which keeps few values live.
#ifndef ESDC_NODE_MINBLOCKS
#define ESDC_NODE_MINBLOCKS 6      // 6 x 128 threads per SM: at most 85 registers (SYN19: 80, a
                                   // 76-byte spill; the kernel waits on memory more than on FP64,
                                   // and 6 blocks beat 5, 7 and 8 on the headline slab)
#endif
// TAU: batched kernels may add the FAS correction tau (a.tau, rows 1..M; the
// recursive form adds tau_i - tau_{i-1}, tau_0 = 0, to every row of node i).
template <class Model, int M, bool MIXED, bool TAU = false>
__device__ __forceinline__ void node_body(const StepArgs& a, const PhaseArgs& ph, const MeshDev& m,
                                          const StimDev& st, const unsigned* on, double D, int p, int ix, int iy,
                                          int iz)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const int64_t ld = a.m.ld;
    const int i = ph.i;
    const bool eval = i >= 2;                 // G at y_{i-1}^{k+1}
    const bool quad = i <= M;                 // explicit rows of y_i^{k+1}
    const int jm = i - 2;                     // 0-based index of node i-1
    const int ii = i - 1;                     // 0-based index of node i
    auto dtau = [&](int s) -> double {
        if (!TAU || !a.tau) return 0.0;
        const double t1 = a.tau[((int64_t)ii * NS + s) * ld + p];
        return ii > 0 ? t1 - a.tau[((int64_t)(ii - 1) * NS + s) * ld + p] : t1;
    };
    const double* src = eval ? a.Y + (int64_t)jm * NS * ld : a.yn;   // y_{i-1}^{k+1}
    double u[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) u[s] = src[s * ld + p];
    const double* Gp = ph.Gold + (int64_t)jm * NS * ld;               // G_{i-1}^k
    double* Gq = ph.Gnew + (int64_t)jm * NS * ld;                     // G_{i-1}^{k+1}
    double* Yi = a.Y + (int64_t)ii * NS * ld;
    const double dtd = quad ? a.dtd[i] : 0.0;

    // ---- V row and auxiliaries
    double dlt0 = 0.0, ha[NA > 0 ? NA : 1];
    float uf[NS];
    if (eval) {
        const double fi = D * lap(m, src, p, ix, iy, iz);
        double mI;
        if (MIXED) {                      // precision form: the ionic model in FP32
#pragma unroll
            for (int s = 0; s < NS; ++s) uf[s] = (float)u[s];
            float mIf, haf[NA > 0 ? NA : 1];
            Model::currents_f(a.mpf.p, uf, mIf, haf);
            mI = mIf;
#pragma unroll
            for (int s = 0; s < NA; ++s) ha[s] = haf[s];
        } else {
            Model::currents(a.mp.p, u, mI, ha);
        }
        const double fE = (stim_at(st, on[i - 1], ix, iy, iz) + mI) * a.inv_Cm;
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
        if (eval) Yi[p] = fma(ph.rho, u[0] - a.Vprev[p], vik);
        a.Vprev[p] = vik;
        double q = u[0];
#pragma unroll
        for (int j = 0; j < M; ++j) q = fma(a.dS0[ii][j], ph.Gold[(int64_t)j * NS * ld + p], q);
        double rv = fma(dtd, dlt0 - a.FI[(int64_t)ii * ld + p], q);
        if (TAU) rv += dtau(0);                // (x + 0.0 is not x in IEEE arithmetic: no add without TAU)
        a.rhs[p] = rv;
#pragma unroll
        for (int s = 1; s <= NA; ++s) {
            const double dl = eval ? ha[s - 1] - Gp[s * ld + p] : 0.0;
            double qa = u[s];
#pragma unroll
            for (int j = 0; j < M; ++j) qa = fma(a.dS0[ii][j], ph.Gold[((int64_t)j * NS + s) * ld + p], qa);
            double ya = fma(dtd, dl, qa);
            if (TAU) ya += dtau(s);
            Yi[s * ld + p] = ya;
        }
    }
    // ---- gates, one at a time
    typename Model::VCtx vc{};
    if (eval && !MIXED) vc = Model::vctx(a.mp, u[0]);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int s = 1 + NA + g;
        double dl = 0.0;
        if (eval) {
            // g_n = Lambda(V) u + b(V) + Lambda_n (u_n - u), b = -Lambda w_inf
            const double ln = a.LAMN[(int64_t)g * ld + p], du = a.yn[s * ld + p] - u[s];
            double gn;
            if (MIXED) {
                float lf, yf;
                Model::gate_f(a.mpf.p, g, uf[0], lf, yf);
                gn = (double)lf * (u[s] - (double)yf) + ln * du;
            } else {
                double lam, b;
                Model::gate_lb(a.mp.p, vc, g, u[0], lam, b);
                gn = fma(ln, du, fma(lam, u[s], b));
            }
            Gq[s * ld + p] = gn;
            dl = gn - Gp[s * ld + p];
        }
        if (quad) {
            double qg = u[s];
#pragma unroll
            for (int j = 0; j < M; ++j)
                qg = fma(a.S[(((int64_t)ii * M + j) * NG + g) * ld + p],
                         ph.Gold[((int64_t)j * NS + s) * ld + p], qg);
            double yg = fma(a.PHI[((int64_t)ii * NG + g) * ld + p], dl, qg);
            if (TAU) yg += dtau(s);
            Yi[s * ld + p] = yg;
        }
    }
}

// Node 1 of the next sweep fused into a launch (a.fuse1, M >= 2): the explicit
// rows of y_1 from the G this thread has just written, at the same node.  It
// reads only this node's values (no stencil), and for M >= 2 it writes rows
// (y_1's) that no stencil of the launch reads, so the fused launch computes
// exactly what the two launches compute.
__device__ __forceinline__ PhaseArgs next_node1(const StepArgs& a) { return PhaseArgs{1, 0.0, a.Gnew, a.Gnew, nullptr}; }

template <class Model, int M, bool MIXED, bool BATCH>
__global__ void __launch_bounds__(128, ESDC_NODE_MINBLOCKS) k_node(StepArgs a)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        if (!BATCH) {
            int ix, iy, iz;
            node_xyz(a.m, p, ix, iy, iz);
            node_body<Model, M, MIXED>(a, phase_of(a), a.m, a.st, a.stim_on, a.D, p, ix, iy, iz);
            if (M >= 2 && a.fuse1) node_body<Model, M, MIXED>(a, next_node1(a), a.m, a.st, a.stim_on, a.D, p, ix, iy, iz);
        } else {
            BatchNode n;
            if (!batch_node(a, p, n)) continue;
            node_body<Model, M, MIXED, true>(a, phase_of(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
            if (M >= 2 && a.fuse1)
                node_body<Model, M, MIXED, true>(a, next_node1(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
        }
    }
}

template <class Model, int M, bool MIXED, bool BATCH>
__global__ void __launch_bounds__(128, ESDC_SETUP_MINBLOCKS) k_setup(StepArgs a)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        if (!BATCH) {
            int ix, iy, iz;
            node_xyz(a.m, p, ix, iy, iz);
            setup_body<Model, M, MIXED>(a, phase_of(a), a.m, a.st, a.stim_on, a.D, p, ix, iy, iz);
            if (M >= 2 && a.fuse1) node_body<Model, M, MIXED>(a, next_node1(a), a.m, a.st, a.stim_on, a.D, p, ix, iy, iz);
        } else {
            BatchNode n;
            if (!batch_node(a, p, n)) continue;
            setup_body<Model, M, MIXED>(a, phase_of(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
            if (M >= 2 && a.fuse1)
                node_body<Model, M, MIXED, true>(a, next_node1(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
        }
    }
}


// ------------------------------------------------------------------ residual + output
// r_i = y_n + dt sum_j a_ij G_j - y_i (eq. def_C), accumulated over i from the row
// differences dt S_ij = dt (a_ij - a_{i-1,j});
// per-state max |r| and max |y|; y_{n+1} = y_M.
// One state s of one node: the residuals of the M nodes, the largest |r_i|
// and |y| (y_n included), and y_{n+1} = y_{n,M} (c_M = 1).
// Returns false if a residual or iterate is not finite.
// The maxima are taken on the bit patterns of |r| and |y| with integer
// operations: for non-negative doubles the patterns order like the values, and
// Inf and NaN have the largest patterns (>= 0x7ff0...), so one test at the end
// finds them.  This keeps the comparisons off the FP64 pipe, the scarce unit.
__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

template <class Model, int M, bool TAU = false>
__device__ __forceinline__ bool residual_state(const StepArgs& a, const PhaseArgs& ph, int p, int s, double& rmax,
                                               double& ymax)
{
    constexpr int NS = Model::NS, NA = Model::NA, NG = Model::NG;
    const int64_t ld = a.m.ld;
    const int g = s - 1 - NA;
    const double yns = a.yn[s * ld + p];
    unsigned long long rb = 0ULL, yb = abs_bits(yns);
    // r_i = y_n + dt sum_j a_ij G_j - y_i (eq. def_C; the batches' FAS form adds
    // tau_i): the row sums of dt S are dt a_ij, so A_i = y_n + sum_{l <= i}
    // sum_j dt S_lj G_j is carried through the FMAs and r_i = A_i - y_i.
    double A = yns;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const double sij = (g >= 0) ? a.S[(((int64_t)i * M + j) * NG + g) * ld + p] : a.dS0[i][j];
            A = fma(sij, ph.Gold[((int64_t)j * NS + s) * ld + p], A);
        }
        const double yi = a.Y[((int64_t)i * NS + s) * ld + p];
        double r = A - yi;
        if (TAU && a.tau) r += a.tau[((int64_t)i * NS + s) * ld + p];
        if (a.R) a.R[((int64_t)i * NS + s) * ld + p] = r;
        rb = max(rb, abs_bits(r));
        yb = max(yb, abs_bits(yi));
    }
    // y_n was read above by this thread only, so y may alias y_{n+1}.
    ph.yout[s * ld + p] = a.Y[((int64_t)(M - 1) * NS + s) * ld + p];
    rmax = __longlong_as_double((long long)rb);
    ymax = __longlong_as_double((long long)yb);
    return rb < 0x7ff0000000000000ULL && yb < 0x7ff0000000000000ULL;
}

template <class Model, int M>
__global__ void __launch_bounds__(128) k_residual(StepArgs a)
{
    constexpr int NS = Model::NS;
    __shared__ double smax[2 * ESDC_NSMAX];
    for (int s = threadIdx.x; s < 2 * NS; s += blockDim.x) smax[s] = 0.0;
    __syncthreads();
    bool bad = false;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            double rmax, ymax;
            bad |= !residual_state<Model, M>(a, phase_of(a), p, s, rmax, ymax);
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



// Uploads this translation unit's copy of the collocation constants to the
// current device (once per device).
inline cudaError_t upload_constants_local(bool* done, int dev)
{
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    ColloData col[ESDC_MMAX];
    for (int M = 1; M <= ESDC_MMAX; ++M)
        if (esdc_colloc_build(M, &col[M - 1])) return cudaErrorInvalidValue;
    double inv[ESDC_NSER], invf[ESDC_MMAX + 2];
    inv[0] = 0.0;
    for (int k = 1; k < ESDC_NSER; ++k) inv[k] = 1.0 / k;
    invf[0] = 1.0;
    for (int k = 1; k < ESDC_MMAX + 2; ++k) invf[k] = invf[k - 1] / k;
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_col, col, sizeof col)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_inv, inv, sizeof inv)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_invfact, invf, sizeof invf)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// Grid of a per-node kernel: the resident capacity of the device (blocks per SM
// from the occupancy calculator x SMs), so that the grid-stride loop spreads the
// nodes evenly over all SMs in one wave; smaller meshes use one block per 128 nodes.
template <class F>
inline int blocks_per_sm(F kernel, int threads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm;
}

inline int resident_grid(const esdc_handle* h, int per_sm, int threads)
{
    long long cap = (long long)h->sms * per_sm;
    long long need = ((long long)h->mesh.N + threads - 1) / threads;
    return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

template <class Model, int M, bool MIXED>
cudaError_t launch_step_kernels(esdc_handle* h, StepArgs& a, double* y, int K, cudaStream_t s)
{
    const int T = 128;
    static int occ_setup = 0, occ_node = 0, occ_res = 0;    // blocks/SM per (model, M) instantiation
    if (!occ_setup) {
        occ_node = blocks_per_sm(k_node<Model, M, MIXED, false>, T);
        occ_res = blocks_per_sm(k_residual<Model, M>, T);
        occ_setup = blocks_per_sm(k_setup<Model, M, MIXED, false>, T);
    }
    const int nb_setup = resident_grid(h, occ_setup, T);
    const int nb_node = resident_grid(h, occ_node, T);
    const int nb_res = resident_grid(h, occ_res, T);
    const double g0 = h->D;   // operator scale: (I - dt d_i D L)
    const ColloData* C = &h->col[M - 1];

    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            a.dS0[i][j] = a.dt * C->S0[i][j];
            for (int q = 0; q < M; ++q) a.dtB[i][j][q] = a.dt * C->B[i][j][q];
        }
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
    // Node 1 of each sweep runs inside the launch before it (the set-up, or the
    // previous sweep's final evaluation), except while the adjoint records the
    // iterate after every sweep (node 1 would already have overwritten y_1).
    const bool fuse = h->opt.fuse_node1 && M >= 2 && K >= 1 && !h->tapeY;
    a.fuse1 = fuse;
    a.ztab = esdc_ztab_device(h->zt, M, a.dt, *C, s);
    prof_begin(h, 0, s);
    k_setup<Model, M, MIXED, false><<<nb_setup, T, 0, s>>>(a);
    prof_end(h, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Adjoint recording (esdc_adjoint_*): G^0 and FI^0 after the set-up, and
    // Y^{k+1}, G^{k+1}, FI^{k+1} after every sweep.
    const int64_t tY = (int64_t)M * h->NS * h->mesh.ld, tF = (int64_t)M * h->mesh.ld;
    if (h->tapeY) {
        if ((e = cudaMemcpyAsync(h->tapeG, h->G0, sizeof(double) * tY, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h->tapeFI, h->FI, sizeof(double) * tF, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
    }
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
            a.fuse1 = fuse && i == M + 1 && k + 1 < K;
            if (!(fuse && i == 1)) {
                prof_begin(h, 1, s);
                k_node<Model, M, MIXED, false><<<nb_node, T, 0, s>>>(a);
                prof_end(h, s);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            if (i <= M) {
                double* Vi = h->Y + (int64_t)(i - 1) * h->NS * h->mesh.ld;
                const double g = a.dt * C->d[i] * g0;
                int* log = (k * M + (i - 1) < h->cg_log_len) ? h->cg_log + k * M + (i - 1) : nullptr;
                prof_begin(h, 2, s);
                e = MIXED ? esdc_cg_mixed_launch(h->mesh, h->cg, g, h->rhs, Vi, h->opt.tol_cg, h->opt.cg_maxit,
                                                 h->opt.precond, h->opt.solver, log, h->flags, s)
                          : esdc_cg_launch(h->mesh, h->cg, g, h->rhs, Vi, h->opt.tol_cg, h->opt.cg_maxit,
                                           h->opt.precond, h->opt.solver, log, h->flags, s);
                prof_end(h, s);
                if (e != cudaSuccess) return e;
            }
        }
        if (h->tapeY) {
            if ((e = cudaMemcpyAsync(h->tapeY + k * tY, h->Y, sizeof(double) * tY, cudaMemcpyDeviceToDevice, s)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(h->tapeG + (k + 1) * tY, Gnew, sizeof(double) * tY, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(h->tapeFI + (k + 1) * tF, h->FI, sizeof(double) * tF, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
                return e;
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

template <class Model, bool MIXED>
cudaError_t dispatch_M(esdc_handle* h, StepArgs& a, double* y, int M, int K, cudaStream_t s)
{
    switch (M) {
        case 1: return launch_step_kernels<Model, 1, MIXED>(h, a, y, K, s);
        case 2: return launch_step_kernels<Model, 2, MIXED>(h, a, y, K, s);
        case 3: return launch_step_kernels<Model, 3, MIXED>(h, a, y, K, s);
        case 4: return launch_step_kernels<Model, 4, MIXED>(h, a, y, K, s);
        case 5: return launch_step_kernels<Model, 5, MIXED>(h, a, y, K, s);
        case 6: return launch_step_kernels<Model, 6, MIXED>(h, a, y, K, s);
        case 7: return launch_step_kernels<Model, 7, MIXED>(h, a, y, K, s);
        case 8: return launch_step_kernels<Model, 8, MIXED>(h, a, y, K, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
