// Discrete adjoint of the HSDC step (the differentiation form).
//
// The forward map is exactly the GPU step of esdc_sweep: the recursive sweep
// of eq. def_P over the nodes i = 1..M, K times, after the set-up that
// freezes Lambda_n = Lambda(V_n) and tabulates dt S_ij(dt Lambda_n) and
// dt d_i phi_1(d_i dt Lambda_n) (App. A).  This file runs that map backwards
// (reverse-mode differentiation of the same arithmetic, by hand):
//
//   sweep k, node launch i (forward: evaluation at y_{i-1}^{k+1}, then the
//   explicit rows and the right-hand side of node i, then the implicit solve)
//   is reversed as: gate rows of node i, the adjoint solve (the operator
//   I - dt d_i D A is symmetric, so it is the same CG), the right-hand side,
//   then the evaluation at node i-1.  Launch i = M+1 (evaluation at node M
//   only) comes first, launch i = 1 last.  The set-up comes after sweep 0.
//
// The derivative of the coefficient tables in Lambda_n uses
// phi_k'(x) = phi_k(x) - k phi_{k+1}(x) (from the series of App. A), the
// Hodgkin-Huxley derivatives are analytic (esdc_models.cuh), and the
// conductivity derivative of lambda^T A v is, per node p,
//   -(1/(2h^2)) sum_{q in nbr(p)} (lambda_p - lambda_q)(v_p - v_q).
//
// Over many steps (esdc_adjoint_forward / esdc_adjoint_backward) the forward
// run keeps one checkpoint y_n per step; the backward run recomputes each
// step from its checkpoint, recording the sweep iterates (handle tape), and
// reverses it.  Outputs are the gradients of a loss through the adjoint of V
// at sensor nodes after every step, with respect to the per-node conductivity
// field, g_Na, g_K and the initial state.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "esdc_kernels.cuh"

namespace {

std::mutex g_aconst_mu;
bool g_aconst_done[64] = {false};

using HH = esdc::HH1952;
constexpr int NS = HH::NS, NG = HH::NG;

struct AdjArgs {
    MeshDev m;
    ModelDev mp;
    int64_t ld;
    double D, inv_Cm, dt;
    double dS0[ESDC_MMAX][ESDC_MMAX];
    double dtd[ESDC_MMAX + 1];
    const double* yn;          // y_n [NS][ld]
    const double* Yk1;         // Y^{k+1} [M][NS][ld]
    const double* Gk;          // G^k
    const double* Gk1;         // G^{k+1}
    const double* S;           // dt S_ij, [M][M][NG][ld]
    const double* PHI;         // dt d_i phi_1, [M][NG][ld]
    const double* LAMN;        // Lambda_n [NG][ld]
    double* bY;                // adjoint of Y^{k+1}
    double* byn;               // adjoint of y_n
    double* bGk;               // adjoint of G^k (accumulated here)
    const double* bGk1;        // adjoint of G^{k+1} (complete)
    double* bFIk;              // adjoint of FI^k [M][ld]
    const double* bFIk1;       // adjoint of FI^{k+1}
    double* bS;                // [M][M][NG][ld]
    double* bPHI;              // [M][NG][ld]
    double* bLAM;              // [NG][ld]
    double* bdlt0;             // [ld] adjoint of the f_E change of node i-1
    double* bdl;               // [NG][ld] adjoint of the gate changes of node i-1
    const double* brhs;        // [ld] adjoint of the V right-hand side (after the solve)
    double* tmp;               // [ld]
    double* gsig;              // [ld]
    double* gpar;              // [2][ld] d/d(g_Na, g_K) per node
    int i;                     // node launch 1..M+1
};

// lambda^T (dA/dsigma_p) v and (A w)_p for the field operator.
__device__ __forceinline__ void field_terms(const MeshDev& m, const double* lam, const double* v, const double* w,
                                            int p, int ix, int iy, int iz, double& dsig, double& aw)
{
    const int sxy = m.nx * m.ny;
    const double sp = m.sig[p], lp = lam[p], vp = v[p], wp = w[p];
    double g = 0.0, a = 0.0;
    auto face = [&](int q) {
        g += (lp - lam[q]) * (vp - v[q]);
        a += (sp + m.sig[q]) * (w[q] - wp);
    };
    if (ix > 0) face(p - 1);
    if (ix < m.nx - 1) face(p + 1);
    if (iy > 0) face(p - m.nx);
    if (iy < m.ny - 1) face(p + m.nx);
    if (iz > 0) face(p - sxy);
    if (iz < m.nz - 1) face(p + sxy);
    dsig = -0.5 * m.ih2 * g;
    aw = 0.5 * m.ih2 * a;
}

// Gate rows of node i (reverse of Y_{i,g} = u_g + sum_j dt S_ij G^k_{j,g} + PHI_i dl_g).
template <int M>
__global__ void k_adj_gates(AdjArgs a)
{
    const int64_t ld = a.ld;
    const int ii = a.i - 1;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        const double* bYi = a.bY + (int64_t)ii * NS * ld;
        double* bu = a.i == 1 ? a.byn : a.bY + (int64_t)(ii - 1) * NS * ld;
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + g;
            const double bw = bYi[s * ld + p];
            bu[s * ld + p] += bw;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int64_t sij = (((int64_t)ii * M + j) * NG + g) * ld + p;
                a.bGk[((int64_t)j * NS + s) * ld + p] += a.S[sij] * bw;
                a.bS[sij] += a.Gk[((int64_t)j * NS + s) * ld + p] * bw;
            }
            if (a.i >= 2) {
                const int64_t jm = ii - 1;
                const double dl = a.Gk1[(jm * NS + s) * ld + p] - a.Gk[(jm * NS + s) * ld + p];
                a.bPHI[((int64_t)ii * NG + g) * ld + p] += dl * bw;
                a.bdl[g * ld + p] = a.PHI[((int64_t)ii * NG + g) * ld + p] * bw;
            }
        }
    }
}

// The V right-hand side of node i, after the adjoint solve gave brhs:
// rhs = u_V + sum_j dt S^0_ij G^k_{j,V} + dt d_i (dlt0 - FI^k_i), and the
// conductivity term of the solve's operator.
template <int M>
__global__ void k_adj_rhs(AdjArgs a)
{
    const int64_t ld = a.ld;
    const int ii = a.i - 1;
    const double gam = a.dtd[a.i] * a.D;
    const double* Vi = a.Yk1 + (int64_t)ii * NS * ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        double* bu = a.i == 1 ? a.byn : a.bY + (int64_t)(ii - 1) * NS * ld;
        const double br = a.brhs[p];
        bu[p] += br;
#pragma unroll
        for (int j = 0; j < M; ++j) a.bGk[(int64_t)j * NS * ld + p] += a.dS0[ii][j] * br;
        a.bdlt0[p] = a.i >= 2 ? a.dtd[a.i] * br : 0.0;
        a.bFIk[(int64_t)ii * ld + p] -= a.dtd[a.i] * br;
        int ix, iy, iz;
        node_xyz(a.m, p, ix, iy, iz);
        double dsig, aw;
        field_terms(a.m, a.brhs, Vi, a.brhs, p, ix, iy, iz, dsig, aw);
        a.gsig[p] += gam * dsig;                 // F = (I - gam A) V - rhs: dL/dsigma = gam brhs^T dA/dsigma V
    }
}

// bFI^{k+1}_{i-1} + bG^{k+1}_{i-1,V}: the adjoint of FI at node i-1 (a
// stencil input), gathered before the evaluation kernel reads neighbours.
__global__ void k_adj_fisum(AdjArgs a, int jm)
{
    const int64_t ld = a.ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x)
        a.tmp[p] = a.bFIk1[(int64_t)jm * ld + p] + a.bGk1[(int64_t)jm * NS * ld + p];
}

// Evaluation at node i-1 = u (launch i >= 2; i = M+1: the final evaluation).
template <int M>
__global__ void k_adj_eval(AdjArgs a)
{
    const int64_t ld = a.ld;
    const int jm = a.i - 2;
    const bool quad = a.i <= M;
    const double* U = a.Yk1 + (int64_t)jm * NS * ld;
    double* bu = a.bY + (int64_t)jm * NS * ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(a.m, p, ix, iy, iz);
        double u[NS];
        for (int s = 0; s < NS; ++s) u[s] = U[s * ld + p];
        // FI = D A u_V
        double dsig, aw;
        field_terms(a.m, a.tmp, U, a.tmp, p, ix, iy, iz, dsig, aw);
        double buV = a.D * aw;
        a.gsig[p] += a.D * dsig;
        // f_E = (stim + mI(u)) / C_m enters G_V and dlt0
        const double bdlt0 = quad ? a.bdlt0[p] : 0.0;
        const double bmI = (a.bGk1[(int64_t)jm * NS * ld + p] + bdlt0) * a.inv_Cm;
        double dmI[NS], dpar[2];
        HH::currents_d(a.mp.p, u, dmI, dpar);
        buV += dmI[0] * bmI;
        double bus[NS];
        for (int s = 1; s < NS; ++s) bus[s] = dmI[s] * bmI;
        a.gpar[p] += dpar[0] * bmI;
        a.gpar[ld + p] += dpar[1] * bmI;
        if (quad) {                      // dlt0 = fE^{k+1} - (G^k_V - FI^k)
            a.bGk[(int64_t)jm * NS * ld + p] -= bdlt0;
            a.bFIk[(int64_t)jm * ld + p] += bdlt0;
        }
        // gates: G_g = lam(u_V)(u_g - yinf(u_V)) + Lambda_n (yn_g - u_g); dl_g = G_g - G^k_g
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + g;
            double lam, yinf, dlam, dyinf;
            HH::gate_d(a.mp.p, g, u[0], lam, yinf, dlam, dyinf);
            const double bdl = quad ? a.bdl[g * ld + p] : 0.0;
            const double bgn = a.bGk1[((int64_t)jm * NS + s) * ld + p] + bdl;
            if (quad) a.bGk[((int64_t)jm * NS + s) * ld + p] -= bdl;
            const double Ln = a.LAMN[(int64_t)g * ld + p];
            bus[s] += bgn * (lam - Ln);
            buV += bgn * (dlam * (u[s] - yinf) - lam * dyinf);
            a.bLAM[(int64_t)g * ld + p] += bgn * (a.yn[s * ld + p] - u[s]);
            a.byn[s * ld + p] += bgn * Ln;
        }
        bu[p] += buV;
        for (int s = 1; s < NS; ++s) bu[s * ld + p] += bus[s];
    }
}

// Set-up, part 1: tmp = sum_j (bFI^0_j + bG^0_{j,V}) (FI^0 = D A V_n feeds both).
template <int M>
__global__ void k_adj_setup_sum(AdjArgs a)
{
    const int64_t ld = a.ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int j = 0; j < M; ++j) t += a.bFIk[(int64_t)j * ld + p] + a.bGk[(int64_t)j * NS * ld + p];
        a.tmp[p] = t;
    }
}

// Set-up, part 2: G^0 = g_n(y_n) (no Lambda_n term at y = y_n), FI^0, and the
// tables' dependence on Lambda_n = lam(V_n).
template <int M>
__global__ void k_adj_setup(AdjArgs a)
{
    const ColloData& C = c_col[M - 1];
    const int64_t ld = a.ld;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(a.m, p, ix, iy, iz);
        double u[NS];
        for (int s = 0; s < NS; ++s) u[s] = a.yn[s * ld + p];
        double dsig, aw;
        field_terms(a.m, a.tmp, a.yn, a.tmp, p, ix, iy, iz, dsig, aw);
        double bV = a.D * aw;
        a.gsig[p] += a.D * dsig;
        double sGV = 0.0;
        for (int j = 0; j < M; ++j) sGV += a.bGk[(int64_t)j * NS * ld + p];
        const double bmI = sGV * a.inv_Cm;
        double dmI[NS], dpar[2];
        HH::currents_d(a.mp.p, u, dmI, dpar);
        bV += dmI[0] * bmI;
        double bus[NS];
        for (int s = 1; s < NS; ++s) bus[s] = dmI[s] * bmI;
        a.gpar[p] += dpar[0] * bmI;
        a.gpar[ld + p] += dpar[1] * bmI;
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + g;
            double lam, yinf, dlam, dyinf;
            HH::gate_d(a.mp.p, g, u[0], lam, yinf, dlam, dyinf);
            double sG = 0.0;
            for (int j = 0; j < M; ++j) sG += a.bGk[((int64_t)j * NS + s) * ld + p];
            bus[s] += sG * lam;
            bV += sG * (dlam * (u[s] - yinf) - lam * dyinf);
            // d/dLambda of the tables
            const double z = a.dt * lam;
            double bL = a.bLAM[(int64_t)g * ld + p];
            double daprev[M];
            for (int j = 0; j < M; ++j) daprev[j] = 0.0;
            for (int i = 0; i < M; ++i) {
                double ph[M + 1];
                phi_all<M + 1>(C.c[i + 1] * z, ph);
                double ph1[M + 1];
                phi_all<M + 1>(C.d[i + 1] * z, ph1);
                // PHI_i = dt d_i phi_1(d_i dt Lambda)
                bL += a.bPHI[((int64_t)i * NG + g) * ld + p] * a.dtd[i + 1] * (ph1[0] - ph1[1]) * C.d[i + 1] * a.dt;
                for (int j = 0; j < M; ++j) {
                    double da = 0.0;
                    for (int k = 0; k < M; ++k) da = fma(C.B[i][j][k], ph[k] - (k + 1) * ph[k + 1], da);
                    da *= a.dt * C.c[i + 1] * a.dt;               // d(dt a_ij)/dLambda
                    bL += a.bS[(((int64_t)i * M + j) * NG + g) * ld + p] * (da - daprev[j]);
                    daprev[j] = da;
                }
            }
            bV += dlam * bL;
        }
        a.byn[p] += bV;
        for (int s = 1; s < NS; ++s) a.byn[s * ld + p] += bus[s];
    }
}

__global__ void k_scatter_sensors(double* lamV, const int* sens, const double* d, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) atomicAdd(lamV + sens[k], d[k]);
}

__global__ void k_gather_sensors(const double* V, const int* sens, double* out, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) out[k] = V[sens[k]];
}

// Deterministic sums of the per-node parameter derivatives (one block, fixed order).
__global__ void k_sum2(const double* g, int64_t ld, int N, double* out)
{
    __shared__ double sh[2][256];
    for (int r = 0; r < 2; ++r) {
        double s = 0.0;
        for (int p = threadIdx.x; p < N; p += blockDim.x) s += g[r * ld + p];
        sh[r][threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) s += sh[threadIdx.x][t];
        out[threadIdx.x] = s;
    }
}

struct AdjWork {
    double *bY = nullptr, *byn = nullptr, *bG[2] = {nullptr, nullptr}, *bFI[2] = {nullptr, nullptr};
    double *bS = nullptr, *bPHI = nullptr, *bLAM = nullptr, *bdlt0 = nullptr, *bdl = nullptr, *brhs = nullptr,
           *tmp = nullptr, *gpar = nullptr, *yw = nullptr, *lam = nullptr, *sum2 = nullptr;
    double *tapeY = nullptr, *tapeG = nullptr, *tapeFI = nullptr;
    std::vector<void*> all;
    cudaError_t alloc(double** p, int64_t n)
    {
        cudaError_t e = cudaMalloc((void**)p, sizeof(double) * n);
        if (e == cudaSuccess) { all.push_back(*p); cudaMemset(*p, 0, sizeof(double) * n); }
        return e;
    }
    ~AdjWork()
    {
        for (void* p : all) cudaFree(p);
    }
};

int grid_of(const esdc_handle* h)
{
    long long need = (h->mesh.N + 127) / 128;
    long long cap = (long long)h->sms * 8;
    return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

template <int M>
cudaError_t reverse_step(esdc_handle* h, AdjWork& w, AdjArgs& a, int K, cudaStream_t s)
{
    const int64_t ld = h->mesh.ld, NSld = (int64_t)NS * ld, tY = (int64_t)M * NSld, tF = (int64_t)M * ld;
    const ColloData* C = &h->col[M - 1];
    const int nb = grid_of(h);
    cudaError_t e;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) a.dS0[i][j] = a.dt * C->S0[i][j];
    for (int i = 0; i <= M; ++i) a.dtd[i] = a.dt * C->d[i];
    // table adjoints, y_n adjoint
    if ((e = cudaMemsetAsync(w.bS, 0, sizeof(double) * M * M * NG * ld, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.bPHI, 0, sizeof(double) * M * NG * ld, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.bLAM, 0, sizeof(double) * NG * ld, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.byn, 0, sizeof(double) * NSld, s)) != cudaSuccess) return e;
    // adjoint of G^K, FI^K: nothing consumes them
    int cur = 0;
    if ((e = cudaMemsetAsync(w.bG[1], 0, sizeof(double) * tY, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.bFI[1], 0, sizeof(double) * tF, s)) != cudaSuccess) return e;
    for (int k = K - 1; k >= 0; --k) {
        // bY: adjoint of Y^{k+1}; only the last sweep's node M is an output
        if ((e = cudaMemsetAsync(w.bY, 0, sizeof(double) * tY, s)) != cudaSuccess) return e;
        if (k == K - 1 &&
            (e = cudaMemcpyAsync(w.bY + (int64_t)(M - 1) * NSld, w.lam, sizeof(double) * NSld,
                                 cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(w.bG[cur], 0, sizeof(double) * tY, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(w.bFI[cur], 0, sizeof(double) * tF, s)) != cudaSuccess) return e;
        a.Yk1 = w.tapeY + (int64_t)k * tY;
        a.Gk = w.tapeG + (int64_t)k * tY;
        a.Gk1 = w.tapeG + (int64_t)(k + 1) * tY;
        a.bGk = w.bG[cur];
        a.bGk1 = w.bG[1 - cur];
        a.bFIk = w.bFI[cur];
        a.bFIk1 = w.bFI[1 - cur];
        for (int i = M + 1; i >= 1; --i) {
            a.i = i;
            if (i <= M) {
                k_adj_gates<M><<<nb, 128, 0, s>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                // adjoint solve: (I - dt d_i D A) brhs = bY_{i,V}
                if ((e = cudaMemsetAsync(w.brhs, 0, sizeof(double) * ld, s)) != cudaSuccess) return e;
                e = esdc_cg_launch(h->mesh, h->cg, a.dt * C->d[i] * h->D, w.bY + (int64_t)(i - 1) * NSld, w.brhs,
                                   h->opt.tol_cg, h->opt.cg_maxit, h->opt.precond, h->opt.solver, nullptr,
                                   h->flags, s);
                if (e != cudaSuccess) return e;
                k_adj_rhs<M><<<nb, 128, 0, s>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            if (i >= 2) {
                k_adj_fisum<<<nb, 128, 0, s>>>(a, i - 2);
                k_adj_eval<M><<<nb, 128, 0, s>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
        cur = 1 - cur;
    }
    // set-up: bG^0, bFI^0 are in bG[1 - cur] after the last swap
    a.bGk = w.bG[1 - cur];
    a.bFIk = w.bFI[1 - cur];
    k_adj_setup_sum<M><<<nb, 128, 0, s>>>(a);
    k_adj_setup<M><<<nb, 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the adjoint of y_n becomes the output adjoint of the previous step
    return cudaMemcpyAsync(w.lam, w.byn, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s);
}

cudaError_t reverse_step_M(esdc_handle* h, AdjWork& w, AdjArgs& a, int M, int K, cudaStream_t s)
{
    switch (M) {
        case 1: return reverse_step<1>(h, w, a, K, s);
        case 2: return reverse_step<2>(h, w, a, K, s);
        case 3: return reverse_step<3>(h, w, a, K, s);
        case 4: return reverse_step<4>(h, w, a, K, s);
        case 5: return reverse_step<5>(h, w, a, K, s);
        case 6: return reverse_step<6>(h, w, a, K, s);
        case 7: return reverse_step<7>(h, w, a, K, s);
        default: return cudaErrorInvalidValue;
    }
}

int check_handle(esdc_handle* h, int M, int K, int nsteps, int nsens, const int* sens, double dt)
{
    if (h->model != ESDC_MODEL_HH1952) return set_err(h, ESDC_ERR_UNSUPPORTED, "the adjoint covers Hodgkin-Huxley");
    if (!h->mesh.sig) return set_err(h, ESDC_ERR_UNSUPPORTED, "the adjoint needs a conductivity field");
    if (h->opt.precision != 0) return set_err(h, ESDC_ERR_UNSUPPORTED, "the adjoint runs on the FP64 path");
    if (M < 1 || M > 7 || M > h->opt.M_max || K < 1 || K > 64 || nsteps < 1 || nsens < 0 || (nsens > 0 && !sens) ||
        !(dt > 0.0) || !std::isfinite(dt))
        return set_err(h, ESDC_ERR_INVALID_ARG, "bad adjoint arguments");
    if (nsens > 0) {                       // sensor indices are device data: check them before any kernel uses them
        std::vector<int> hs(nsens);
        if (cudaMemcpy(hs.data(), sens, sizeof(int) * nsens, cudaMemcpyDeviceToHost) != cudaSuccess)
            return set_err(h, ESDC_ERR_INVALID_ARG, "sensor indices must be device memory");
        for (int v : hs)
            if (v < 0 || v >= h->mesh.N) return set_err(h, ESDC_ERR_INVALID_ARG, "sensor index %d out of range", v);
    }
    return ESDC_OK;
}

}  // namespace

extern "C" {

int esdc_adjoint_forward(esdc_handle* h, double* y, double t0, double dt, int M, int K, int nsteps, int nsens,
                         const int* sens, double* traces, double* ckpt, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    int rc = check_handle(h, M, K, nsteps, nsens, sens, dt);
    if (rc != ESDC_OK) return rc;
    if (!y || !ckpt || (nsens > 0 && !traces)) return set_err(h, ESDC_ERR_INVALID_ARG, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t NSld = (int64_t)NS * h->mesh.ld;
    double t = t0;
    for (int n = 0; n < nsteps; ++n) {
        CUDA_TRY(h, cudaMemcpyAsync(ckpt + n * NSld, y, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s));
        if ((rc = esdc_sweep(h, y, t, dt, M, K, stream)) != ESDC_OK) return rc;
        if (nsens > 0) {
            k_gather_sensors<<<(nsens + 127) / 128, 128, 0, s>>>(y, sens, traces + (int64_t)n * nsens, nsens);
            CUDA_TRY(h, cudaGetLastError());
        }
        t = t0 + (n + 1) * dt;
    }
    return ESDC_OK;
}

int esdc_adjoint_backward(esdc_handle* h, const double* ckpt, double t0, double dt, int M, int K, int nsteps,
                          int nsens, const int* sens, const double* dtraces, const double* dy_final, double* gy0,
                          double* gsig, double* gpar, void* stream)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    int rc = check_handle(h, M, K, nsteps, nsens, sens, dt);
    if (rc != ESDC_OK) return rc;
    if (!ckpt || !gsig || !gpar || (nsens > 0 && !dtraces)) return set_err(h, ESDC_ERR_INVALID_ARG, "null buffer");
    {
        std::lock_guard<std::mutex> lk(g_aconst_mu);
        if (upload_constants_local(g_aconst_done, h->device) != cudaSuccess)
            return set_err(h, ESDC_ERR_CUDA, "constant upload failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ld = h->mesh.ld, NSld = (int64_t)NS * ld, tY = (int64_t)M * NSld, tF = (int64_t)M * ld;
    AdjWork w;
    if (w.alloc(&w.bY, tY) || w.alloc(&w.byn, NSld) || w.alloc(&w.bG[0], tY) || w.alloc(&w.bG[1], tY) ||
        w.alloc(&w.bFI[0], tF) || w.alloc(&w.bFI[1], tF) || w.alloc(&w.bS, (int64_t)M * M * NG * ld) ||
        w.alloc(&w.bPHI, (int64_t)M * NG * ld) || w.alloc(&w.bLAM, (int64_t)NG * ld) || w.alloc(&w.bdlt0, ld) ||
        w.alloc(&w.bdl, (int64_t)NG * ld) || w.alloc(&w.brhs, ld) || w.alloc(&w.tmp, ld) || w.alloc(&w.gpar, 2 * ld) ||
        w.alloc(&w.yw, NSld) || w.alloc(&w.lam, NSld) || w.alloc(&w.sum2, 2) || w.alloc(&w.tapeY, (int64_t)K * tY) ||
        w.alloc(&w.tapeG, (int64_t)(K + 1) * tY) || w.alloc(&w.tapeFI, (int64_t)(K + 1) * tF))
        return set_err(h, ESDC_ERR_NO_MEMORY, "adjoint workspace");
    CUDA_TRY(h, cudaMemsetAsync(gsig, 0, sizeof(double) * h->mesh.N, s));
    if (dy_final) CUDA_TRY(h, cudaMemcpyAsync(w.lam, dy_final, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s));
    // gsig is accumulated over the padded pitch in a private buffer, then copied
    double* gs = nullptr;
    if (w.alloc(&gs, ld)) return set_err(h, ESDC_ERR_NO_MEMORY, "adjoint workspace");

    AdjArgs a{};
    a.m = h->mesh;
    a.mp = h->mp;
    a.ld = ld;
    a.D = h->D;
    a.inv_Cm = 1.0 / h->Cm;
    a.dt = dt;
    a.yn = w.yw;
    a.S = h->S; a.PHI = h->PHI; a.LAMN = h->LAMN;
    a.bY = w.bY; a.byn = w.byn;
    a.bS = w.bS; a.bPHI = w.bPHI; a.bLAM = w.bLAM;
    a.bdlt0 = w.bdlt0; a.bdl = w.bdl; a.brhs = w.brhs; a.tmp = w.tmp;
    a.gsig = gs; a.gpar = w.gpar;

    // the step is recomputed with its sweeps recorded, on a copy of the checkpoint
    double* ystep = nullptr;
    if (w.alloc(&ystep, NSld)) return set_err(h, ESDC_ERR_NO_MEMORY, "adjoint workspace");
    h->tapeY = w.tapeY; h->tapeG = w.tapeG; h->tapeFI = w.tapeFI;
    struct Untape { esdc_handle* h; ~Untape() { h->tapeY = h->tapeG = h->tapeFI = nullptr; } } untape{h};
    for (int n = nsteps - 1; n >= 0; --n) {
        if (nsens > 0) {
            k_scatter_sensors<<<(nsens + 127) / 128, 128, 0, s>>>(w.lam, sens, dtraces + (int64_t)n * nsens, nsens);
            CUDA_TRY(h, cudaGetLastError());
        }
        CUDA_TRY(h, cudaMemcpyAsync(w.yw, ckpt + n * NSld, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(ystep, w.yw, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s));
        if ((rc = esdc_sweep(h, ystep, t0 + n * dt, dt, M, K, stream)) != ESDC_OK) return rc;
        cudaError_t e = reverse_step_M(h, w, a, M, K, s);
        if (e != cudaSuccess) return set_err(h, ESDC_ERR_CUDA, "adjoint step: %s", cudaGetErrorString(e));
    }
    k_sum2<<<1, 256, 0, s>>>(w.gpar, ld, h->mesh.N, w.sum2);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaMemcpyAsync(gsig, gs, sizeof(double) * h->mesh.N, cudaMemcpyDeviceToDevice, s));
    if (gy0) CUDA_TRY(h, cudaMemcpyAsync(gy0, w.lam, sizeof(double) * NSld, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(gpar, w.sum2, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    int flags = 0;
    CUDA_TRY(h, cudaMemcpy(&flags, h->flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags & ESDC_FLAG_TIMEOUT) return set_err(h, ESDC_ERR_DEVICE_TIMEOUT, "CG grid barrier timed out");
    if (flags & ESDC_FLAG_NONFINITE) return set_err(h, ESDC_ERR_NONFINITE, "non-finite value in the adjoint");
    if (flags & ESDC_FLAG_CG_MAXIT) return set_err(h, ESDC_ERR_CG_NOT_CONVERGED, "CG hit cg_maxit");
    return ESDC_OK;
}

int esdc_set_params(esdc_handle* h, const double* params, int n_params)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    ModelDev mp{};
    ModelDevF mpf{};
    int ns = 0, ng = 0;
    const int rc = esdc_model_setup(h->model, params, n_params, &mp, &mpf, &ns, &ng);
    if (rc != ESDC_OK) return set_err(h, rc, "invalid model parameters");
    h->mp = mp;
    h->mpf = mpf;
    if (esdc_vtab_upload(h) != cudaSuccess) return set_err(h, ESDC_ERR_CUDA, "gate table upload failed");
    return ESDC_OK;
}

}  // extern "C"
