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
#include <vector>

#include "esdc_internal.h"
#include "esdc_kernels.cuh"

namespace {

std::mutex g_const_mu;
bool g_const_done[64] = {false};

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
        Model::eval(mp, u, mI, NA > 0 ? ha : nullptr, l, yi);
        fE[p] = mI; lam[p] = 0.0; yinf[p] = 0.0;
        for (int s = 1; s <= NA; ++s) { fE[s * m.ld + p] = ha[s - 1]; lam[s * m.ld + p] = 0.0; yinf[s * m.ld + p] = 0.0; }
        for (int g = 0; g < NG; ++g) {
            const int s = 1 + NA + g;
            fE[s * m.ld + p] = 0.0; lam[s * m.ld + p] = l[g]; yinf[s * m.ld + p] = yi[g];
        }
    }
}

// FMA throughput probe: ESDC_FMA_CHAINS independent dependent-FMA chains per
// thread, n FMAs each; the result is stored only if it hits an impossible
// value, so the chains stay live without memory traffic.
#define ESDC_FMA_CHAINS 8
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(double* sink, int64_t n, T a, T b)
{
    T x[ESDC_FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < ESDC_FMA_CHAINS; ++c) x[c] = (T)(threadIdx.x + 1) * (T)(c + 1) * (T)1e-3;
    for (int64_t k = 0; k < n; ++k) {
#pragma unroll
        for (int c = 0; c < ESDC_FMA_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T sum = 0;
#pragma unroll
    for (int c = 0; c < ESDC_FMA_CHAINS; ++c) sum += x[c];
    if (sum == (T)-1.0) *sink = (double)sum;
}

__global__ void k_math(const double* x, int64_t n, double* ex, double* rc)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        ex[e] = esdc::esdc_exp(x[e]);
        rc[e] = esdc::esdc_rcp(x[e]);
    }
}

// -diag(A) of the layered operator: sum of the coefficients of the present
// neighbours (faces, and a b sigma_xy/(2h^2) for the in-plane diagonals); of
// the field operator: sum over present faces of (sigma_p + sigma_q)/(2h^2).
__global__ void k_wdiag(MeshDev m, double* w)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m.N; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(m, p, ix, iy, iz);
        if (m.order == 4) {                 // -diag of the fourth-order Laplacian: 30 less the ghosts that mirror onto p
            const int idx[3] = {ix, iy, iz}, nn[3] = {m.nx, m.ny, m.nz};
            double d = 0.0;
            for (int a = 0; a < 3; ++a) {
                if (nn[a] == 1) continue;
                const int i = idx[a], n = nn[a];
                double c = -30.0;
                if (esdc_mirror(i - 1, n) == i) c += 16.0;
                if (esdc_mirror(i + 1, n) == i) c += 16.0;
                if (esdc_mirror(i - 2, n) == i) c -= 1.0;
                if (esdc_mirror(i + 2, n) == i) c -= 1.0;
                d += c;
            }
            w[p] = -d * m.ih2 / 12.0;
            continue;
        }
        if (m.sig) {
            const int sxy = m.nx * m.ny;
            const double sp = m.sig[p];
            double s = 0.0;
            if (ix > 0) s += sp + m.sig[p - 1];
            if (ix < m.nx - 1) s += sp + m.sig[p + 1];
            if (iy > 0) s += sp + m.sig[p - m.nx];
            if (iy < m.ny - 1) s += sp + m.sig[p + m.nx];
            if (iz > 0) s += sp + m.sig[p - sxy];
            if (iz < m.nz - 1) s += sp + m.sig[p + sxy];
            w[p] = 0.5 * m.ih2 * s;
            continue;
        }
        const double cxx = m.lay[iz], cyy = m.lay[m.nz + iz], cd = m.lay[2 * m.nz + iz];
        double s = 0.0;
        if (ix > 0) s += cxx;
        if (ix < m.nx - 1) s += cxx;
        if (iy > 0) s += cyy;
        if (iy < m.ny - 1) s += cyy;
        if (iz > 0) s += m.lay[3 * m.nz + iz - 1];
        if (iz < m.nz - 1) s += m.lay[3 * m.nz + iz];
        const bool xm = ix > 0, xp = ix < m.nx - 1, ym = iy > 0, yp = iy < m.ny - 1;
        double c = 0.0;
        if (xp && yp) c += 1.0;
        if (xm && ym) c += 1.0;
        if (xp && ym) c -= 1.0;
        if (xm && yp) c -= 1.0;
        w[p] = s + cd * c;
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

namespace {

int grid_for(const esdc_handle* h, int threads)
{
    long long need = ((long long)h->mesh.N + threads - 1) / threads;
    long long cap = (long long)h->sms * 16;
    return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

void free_all(esdc_handle* h)
{
    for (auto& e : h->prof_ev)
        if (e) cudaEventDestroy(e);
    esdc_dct_destroy(&h->dct);
    if (h->lay) cudaFree(h->lay);
    if (h->layf) cudaFree(h->layf);
    if (h->wdiag) cudaFree(h->wdiag);
    if (h->sigf) cudaFree(h->sigf);
    if (h->vtab) cudaFree(h->vtab);
    esdc_ztab_free(h->zt);
    void* ptrs[] = {h->Y, h->G0, h->G1, h->FI, h->S, h->PHI, h->LAMN, h->rhs, h->R, h->ydev, h->Vprev,
                    h->cg.r, h->cg.p, h->cg.q, h->cg.z, h->cg.r32, h->cg.p32, h->cg.q32, h->cg.z32,
                    h->cg.e32, h->cg.part, h->cg.bar, h->cg.status,
                    h->rmax, h->flags, h->cg_log};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

const double* esdc_ztab_device(ZtabSlots& z, int M, double dt, const ColloData& C, cudaStream_t s)
{
    for (int k = 0; k < ESDC_ZTAB_SLOTS; ++k)
        if (z.dev[k] && z.M[k] == M && z.dt[k] == dt) return z.dev[k];
    if (z.builds >= ESDC_ZTAB_BUILDS) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    std::vector<double> rows;
    double err = 0.0;
    if (esdc_ztab_build(M, dt, C, rows, &err) != 0) return nullptr;
    const int k = z.next;
    z.next = (z.next + 1) % ESDC_ZTAB_SLOTS;
    // the slot may hold a table that kernels in flight read
    if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
    if (z.n[k] < rows.size()) {
        if (z.dev[k]) cudaFree(z.dev[k]);
        z.dev[k] = nullptr;
        z.n[k] = 0;
        if (cudaMalloc((void**)&z.dev[k], sizeof(double) * rows.size()) != cudaSuccess) {
            z.dev[k] = nullptr;
            return nullptr;
        }
        z.n[k] = rows.size();
    }
    z.M[k] = 0;
    if (cudaMemcpy(z.dev[k], rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return nullptr;
    z.M[k] = M;
    z.dt[k] = dt;
    ++z.gen;
    ++z.builds;
    return z.dev[k];
}

void esdc_ztab_free(ZtabSlots& z)
{
    for (int k = 0; k < ESDC_ZTAB_SLOTS; ++k)
        if (z.dev[k]) cudaFree(z.dev[k]);
    z = ZtabSlots{};
}

// The gate table of the handle's model for the parameters in h->mp (built on
// the host, copied into h->vtab, allocated on first use); h->mp.vtab points
// to it, or stays nullptr (direct evaluation) for models without a table or a
// table that missed its accuracy check.  Synchronises the device before it
// overwrites a table that kernels in flight may read.
cudaError_t esdc_vtab_upload(esdc_handle* h)
{
    std::vector<double> rows;
    h->mp.vtab = nullptr;
    if (esdc_vtab_build(h->model, h->mp.p, rows, &h->vtab_err[0], &h->vtab_err[1]) != 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!h->vtab) e = cudaMalloc((void**)&h->vtab, sizeof(double) * rows.size());
    else e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h->vtab, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) h->mp.vtab = h->vtab;
    return e;
}

// Validates the ionic-model parameters and fills the device parameter blocks
// (FP64, with host reciprocals of the constant divisors of SYN19, and FP32).
int esdc_model_setup(int model, const double* params, int n_params, ModelDev* mp, ModelDevF* mpf, int* NS, int* NG)
{
    const int need = model == ESDC_MODEL_HH1952 ? 7 : model == ESDC_MODEL_SYN19 ? 88 : -1;
    if (need < 0 || !params || n_params != need) return ESDC_ERR_INVALID_ARG;
    for (int k = 0; k < n_params; ++k)
        if (!std::isfinite(params[k])) return ESDC_ERR_INVALID_ARG;
    if (model == ESDC_MODEL_SYN19) {
        for (int q = 0; q < 12; ++q)
            if (params[6 * q + 1] == 0.0 || params[6 * q + 5] == 0.0 || !(params[6 * q + 2] > 0.0))
                return ESDC_ERR_INVALID_ARG;
        for (int l = 0; l < 6; ++l)
            if (!(params[82 + l] > 0.0)) return ESDC_ERR_INVALID_ARG;
    }
    *mp = ModelDev{};
    for (int k = 0; k < n_params; ++k) mp->p[k] = params[k];
    if (model == ESDC_MODEL_SYN19) {
        for (int q = 0; q < 12; ++q) {
            mp->p[88 + q] = 1.0 / params[6 * q + 1];
            mp->p[100 + q] = 1.0 / params[6 * q + 5];
            mp->p[118 + q] = params[6 * q] / params[6 * q + 1];
            mp->p[130 + q] = params[6 * q + 4] / params[6 * q + 5];
            mp->p[142 + q] = std::log(params[6 * q + 2]);
        }
        for (int l = 0; l < 6; ++l) mp->p[112 + l] = 1.0 / params[82 + l];
    }
    for (int k = 0; k < ESDC_NPMAX; ++k) mpf->p[k] = (float)mp->p[k];
    *NS = model == ESDC_MODEL_HH1952 ? 4 : 19;
    *NG = model == ESDC_MODEL_HH1952 ? 3 : 12;
    return ESDC_OK;
}

extern "C" {

void esdc_default_options(esdc_options* opt)
{
    if (!opt) return;
    opt->M_max = 8;
    opt->tol_cg = 1e-14;
    opt->cg_maxit = 200;
    opt->precond = 1;
    opt->precision = 0;
    opt->solver = 0;
    opt->fuse_node1 = 1;
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
    ModelDev mp{};
    ModelDevF mpf{};
    int64_t NS = 0, NG = 0;              // they size the workspace below
    {
        int ns = 0, ng = 0;
        const int mrc = esdc_model_setup(model, params, n_params, &mp, &mpf, &ns, &ng);
        if (mrc != ESDC_OK) return mrc;
        NS = ns;
        NG = ng;
    }
    esdc_options o;
    esdc_default_options(&o);
    if (opt) o = *opt;
    if (o.M_max < 1 || o.M_max > ESDC_MMAX || !(o.tol_cg >= 0.0) || o.cg_maxit < 1) return ESDC_ERR_INVALID_ARG;
    if (o.precision != 0 && o.precision != 1) return ESDC_ERR_INVALID_ARG;
    if (o.solver < 0 || o.solver > 3) return ESDC_ERR_INVALID_ARG;
    if (o.fuse_node1 != 0 && o.fuse_node1 != 1) return ESDC_ERR_INVALID_ARG;
    if (o.solver == 2 && o.precision != 0) return ESDC_ERR_UNSUPPORTED;     // the DCT solve is FP64

    esdc_handle* h = new (std::nothrow) esdc_handle();
    if (!h) return ESDC_ERR_NO_MEMORY;
    h->opt = o;
    h->model = model;
    h->NS = NS;
    h->NG = NG;
    h->NA = h->NS - 1 - h->NG;
    h->sigma = sigma; h->chi = chi; h->Cm = Cm;
    h->D = sigma / (chi * Cm);
    h->mesh.nx = mesh->nx; h->mesh.ny = mesh->ny; h->mesh.nz = mesh->nz;
    h->mesh.N = (int)N;
    h->mesh.ld = (N + 31) / 32 * 32;
    h->mesh.ih2 = 1.0 / (mesh->h * mesh->h);
    h->mp = mp;
    h->mpf = mpf;

    auto fail = [&](int code) { free_all(h); delete h; return code; };
    for (int M = 1; M <= ESDC_MMAX; ++M)
        if (esdc_colloc_build(M, &h->col[M - 1])) return fail(ESDC_ERR_CUDA);
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    if (esdc_vtab_upload(h) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(ESDC_ERR_CUDA);
    {
        std::lock_guard<std::mutex> lk(g_const_mu);
        if (upload_constants_local(g_const_done, h->device) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    }

    const int64_t ld = h->mesh.ld, Mx = o.M_max;
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
    if (cudaMalloc((void**)&h->cg.part, sizeof(double) * 8 * h->cg.max_blocks) != cudaSuccess ||
        cudaMalloc((void**)&h->cg.bar, sizeof(unsigned) * 4) != cudaSuccess ||
        cudaMalloc((void**)&h->cg.status, sizeof(int) * 2) != cudaSuccess ||
        cudaMalloc((void**)&h->rmax, sizeof(unsigned long long) * 2 * ESDC_NSMAX) != cudaSuccess ||
        cudaMalloc((void**)&h->flags, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&h->cg_log, sizeof(int) * 64 * ESDC_MMAX) != cudaSuccess)
        return fail(ESDC_ERR_NO_MEMORY);
    h->cg_log_len = 64 * ESDC_MMAX;
    if (o.precision == 1) {                       // FP32 vectors of the inner solves
        float** fv[] = {&h->cg.r32, &h->cg.p32, &h->cg.q32, &h->cg.z32, &h->cg.e32};
        for (float** f : fv) {
            if (cudaMalloc((void**)f, sizeof(float) * ld) != cudaSuccess) return fail(ESDC_ERR_NO_MEMORY);
            cudaMemset(*f, 0, sizeof(float) * ld);
        }
    }
    cudaMemset(h->cg.bar, 0, sizeof(unsigned) * 4);
    cudaMemset(h->cg.status, 0, sizeof(int) * 2);
    cudaMemset(h->flags, 0, sizeof(int));
    cudaMemset(h->cg_log, 0, sizeof(int) * h->cg_log_len);
    // the DCT-II tables: for the DCT solve itself (2) and for the automatic
    // choice on the FP64 path (0), which takes it while sigma is scalar and the
    // transforms are cheap (x and y; the fourth order, set later, adds z)
    const bool dct_auto = o.solver == 0 && o.precision == 0 && esdc_dct_supported(h->mesh) &&
                          esdc_dct_cheap(h->mesh, 2);
    if (o.solver == 2 || dct_auto) {
        if (!esdc_dct_supported(h->mesh)) return fail(ESDC_ERR_UNSUPPORTED);
        const cudaError_t e = esdc_dct_create(h->mesh, o.M_max, &h->dct);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? ESDC_ERR_NO_MEMORY : ESDC_ERR_CUDA);
        h->cg.dct = &h->dct;
    }
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

int esdc_set_conductivity_layers(esdc_handle* h, const double* sxx, const double* syy, const double* sxy,
                                 const double* szz)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!sxx && !syy && !sxy && !szz) {                 // back to the scalar sigma (or the field)
        if (!h->lay) return ESDC_OK;
        cudaFree(h->lay);
        if (h->layf) cudaFree(h->layf);
        h->lay = nullptr;
        h->layf = nullptr;
        h->mesh.lay = nullptr; h->mesh.layf = nullptr;
        h->mesh.lam_bound = 0.0;
        if (!h->sigf) {
            if (h->wdiag) cudaFree(h->wdiag);
            h->wdiag = nullptr;
            h->mesh.wdiag = nullptr;
            h->D = h->sigma / (h->chi * h->Cm);
        }
        return ESDC_OK;
    }
    if (!sxx || !syy || !sxy || !szz) return set_err(h, ESDC_ERR_INVALID_ARG, "all four layer arrays are needed");
    if (h->opt.solver == 2) return set_err(h, ESDC_ERR_UNSUPPORTED, "the DCT solve needs the scalar sigma");
    if (h->mesh.order != 2)
        return set_err(h, ESDC_ERR_UNSUPPORTED, "layered conductivity needs the second-order stencil");
    if (h->sigf) {                                       // layers replace a conductivity field
        cudaFree(h->sigf);
        h->sigf = nullptr;
        h->mesh.sig = nullptr;
    }
    const int nz = h->mesh.nz;
    const double ih2 = h->mesh.ih2;
    std::vector<double> c(4 * (size_t)nz, 0.0);
    for (int k = 0; k < nz; ++k) {
        const double a = sxx[k], b = syy[k], d = sxy[k], e = szz[k];
        if (!(a > 0.0) || !(b > 0.0) || !(e > 0.0) || !std::isfinite(d) || !(a * b - d * d > 0.0) ||
            !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(e))
            return set_err(h, ESDC_ERR_INVALID_ARG, "layer %d: conductivity tensor not positive definite", k);
        c[k] = a * ih2;
        c[nz + k] = b * ih2;
        c[2 * nz + k] = 0.5 * d * ih2;
        c[3 * nz + k] = (k + 1 < nz) ? 0.5 * (e + szz[k + 1]) * ih2 : 0.0;
    }
    // Gershgorin bound of the spectrum of -A: an interior row has diagonal
    // 2 cx + 2 cy + faces and off-diagonal magnitudes 2 cx + 2 cy + 4 |cd| + faces
    double gb = 0.0;
    for (int k = 0; k < nz; ++k) {
        const double faces = (k > 0 ? c[3 * nz + k - 1] : 0.0) + c[3 * nz + k];
        gb = std::max(gb, 4.0 * c[k] + 4.0 * c[nz + k] + 4.0 * std::fabs(c[2 * nz + k]) + 2.0 * faces);
    }
    std::vector<float> cf(c.begin(), c.end());
    if (!h->lay) {
        CUDA_TRY(h, cudaMalloc((void**)&h->lay, sizeof(double) * 4 * nz));
        CUDA_TRY(h, cudaMalloc((void**)&h->layf, sizeof(float) * 4 * nz));
        CUDA_TRY(h, cudaMalloc((void**)&h->wdiag, sizeof(double) * h->mesh.ld));
    }
    CUDA_TRY(h, cudaMemcpy(h->lay, c.data(), sizeof(double) * 4 * nz, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->layf, cf.data(), sizeof(float) * 4 * nz, cudaMemcpyHostToDevice));
    h->mesh.lay = h->lay;
    h->mesh.lam_bound = gb;
    h->mesh.layf = h->layf;
    h->mesh.wdiag = h->wdiag;
    k_wdiag<<<grid_for(h, 256), 256>>>(h->mesh, h->wdiag);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaDeviceSynchronize());
    h->D = 1.0 / (h->chi * h->Cm);                      // sigma now lives in the coefficients
    return ESDC_OK;
}

int esdc_set_stencil_order(esdc_handle* h, int order)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (order != 2 && order != 4) return set_err(h, ESDC_ERR_INVALID_ARG, "order must be 2 or 4");
    if (order == h->mesh.order) return ESDC_OK;
    if (order == 2) {
        h->mesh.order = 2;
        if (h->wdiag && !h->lay && !h->sigf) { cudaFree(h->wdiag); h->wdiag = nullptr; h->mesh.wdiag = nullptr; }
        if (h->cg.dct) CUDA_TRY(h, esdc_dct_set_order(h->mesh, &h->dct));
        return ESDC_OK;
    }
    if (h->lay || h->sigf) return set_err(h, ESDC_ERR_UNSUPPORTED, "the fourth-order stencil needs the scalar sigma");
    if (h->opt.precision != 0) return set_err(h, ESDC_ERR_UNSUPPORTED, "the fourth-order stencil runs on the FP64 path");
    if (!h->wdiag) CUDA_TRY(h, cudaMalloc((void**)&h->wdiag, sizeof(double) * h->mesh.ld));
    h->mesh.order = 4;
    h->mesh.wdiag = h->wdiag;
    k_wdiag<<<grid_for(h, 256), 256>>>(h->mesh, h->wdiag);
    CUDA_TRY(h, cudaGetLastError());
    if (h->cg.dct) CUDA_TRY(h, esdc_dct_set_order(h->mesh, &h->dct));
    CUDA_TRY(h, cudaDeviceSynchronize());
    return ESDC_OK;
}

int esdc_get_solver(const esdc_handle* h, int* solver)
{
    if (!h || !solver) return ESDC_ERR_INVALID_ARG;
    const int o = h->opt.solver;
    if (o != 0) *solver = o;
    else *solver = (h->cg.dct && h->dct.cheap && !h->mesh.lay && !h->mesh.sig) ? 2 : 3;
    return ESDC_OK;
}

int esdc_set_conductivity_field(esdc_handle* h, const double* sigma)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (!sigma) {                                        // back to the scalar sigma
        if (h->sigf) cudaFree(h->sigf);
        if (h->wdiag && !h->lay) { cudaFree(h->wdiag); h->wdiag = nullptr; h->mesh.wdiag = nullptr; }
        h->sigf = nullptr;
        h->mesh.sig = nullptr;
        if (!h->lay) {
            h->D = h->sigma / (h->chi * h->Cm);
            h->mesh.lam_bound = 0.0;
        }
        return ESDC_OK;
    }
    if (h->opt.precision != 0)
        return set_err(h, ESDC_ERR_UNSUPPORTED, "a conductivity field runs on the FP64 path only");
    if (h->opt.solver == 2) return set_err(h, ESDC_ERR_UNSUPPORTED, "the DCT solve needs the scalar sigma");
    if (h->mesh.order != 2)
        return set_err(h, ESDC_ERR_UNSUPPORTED, "a conductivity field needs the second-order stencil");
    const int64_t N = h->mesh.N;
    for (int64_t p = 0; p < N; ++p)
        if (!(sigma[p] > 0.0) || !std::isfinite(sigma[p]))
            return set_err(h, ESDC_ERR_INVALID_ARG, "sigma[%lld] must be positive and finite", (long long)p);
    if (h->lay) {                                        // a field replaces the layers
        const int rc = esdc_set_conductivity_layers(h, nullptr, nullptr, nullptr, nullptr);
        if (rc != ESDC_OK) return rc;
    }
    if (!h->sigf) CUDA_TRY(h, cudaMalloc((void**)&h->sigf, sizeof(double) * h->mesh.ld));
    if (!h->wdiag) CUDA_TRY(h, cudaMalloc((void**)&h->wdiag, sizeof(double) * h->mesh.ld));
    CUDA_TRY(h, cudaMemcpy(h->sigf, sigma, sizeof(double) * N, cudaMemcpyHostToDevice));
    h->mesh.sig = h->sigf;
    h->mesh.wdiag = h->wdiag;
    // Gershgorin bound of the spectrum of -A: the off-diagonals (face means over
    // h^2) are positive and sum to the diagonal, so the bound is twice the
    // largest diagonal, max_p sum_faces (sigma_p + sigma_q)/h^2
    {
        const int nx = h->mesh.nx, ny = h->mesh.ny, nz = h->mesh.nz;
        const int64_t sxy = (int64_t)nx * ny;
        double gb = 0.0;
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    const int64_t p = ix + nx * (int64_t)iy + sxy * iz;
                    double s = 0.0;
                    if (ix > 0) s += sigma[p] + sigma[p - 1];
                    if (ix < nx - 1) s += sigma[p] + sigma[p + 1];
                    if (iy > 0) s += sigma[p] + sigma[p - nx];
                    if (iy < ny - 1) s += sigma[p] + sigma[p + nx];
                    if (iz > 0) s += sigma[p] + sigma[p - sxy];
                    if (iz < nz - 1) s += sigma[p] + sigma[p + sxy];
                    gb = std::max(gb, s);
                }
        h->mesh.lam_bound = gb * h->mesh.ih2;
    }
    k_wdiag<<<grid_for(h, 256), 256>>>(h->mesh, h->wdiag);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaDeviceSynchronize());
    h->D = 1.0 / (h->chi * h->Cm);                      // sigma now lives in the field
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
    StepArgs a{};                        // value-initialised: every pointer null, every count 0
    a.m = h->mesh; a.st = h->stim; a.mp = h->mp; a.mpf = h->mpf;
    a.dt = dt; a.t_n = t; a.D = h->D; a.inv_Cm = 1.0 / h->Cm;
    a.yn = y; a.Y = h->Y; a.FI = h->FI; a.S = h->S; a.PHI = h->PHI; a.LAMN = h->LAMN; a.rhs = h->rhs;
    a.R = h->R; a.rmax = h->rmax; a.flags = h->flags; a.Vprev = h->Vprev;
    cudaError_t e;
    if (h->opt.precision == 1)
        e = esdc_dispatch_mixed(h, a, y, M, K, s);
    else
        e = h->model == ESDC_MODEL_HH1952 ? dispatch_M<esdc::HH1952, false>(h, a, y, M, K, s)
                                          : dispatch_M<esdc::SYN19, false>(h, a, y, M, K, s);
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
    if (h->opt.precision == 1)
        CUDA_TRY(h, esdc_cg_mixed_launch(h->mesh, h->cg, g, b, x, h->opt.tol_cg, h->opt.cg_maxit,
                                         h->opt.precond, h->opt.solver, nullptr, h->flags, s));
    else
        CUDA_TRY(h, esdc_cg_launch(h->mesh, h->cg, g, b, x, h->opt.tol_cg, h->opt.cg_maxit, h->opt.precond,
                                   h->opt.solver, nullptr, h->flags, s));
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

int esdc_debug_barrier(esdc_handle* h, int skip_block, unsigned limit_us)
{
    if (!h) return ESDC_ERR_INVALID_ARG;
    if (limit_us > 1000000u) return set_err(h, ESDC_ERR_INVALID_ARG, "limit_us above 1 s");
    // grid_barrier reads bar[2] (1 + the block that skips its first arrival) and bar[3] (the wait limit)
    const unsigned w[2] = {skip_block >= 0 ? (unsigned)skip_block + 1u : 0u, limit_us};
    CUDA_TRY(h, cudaDeviceSynchronize());
    CUDA_TRY(h, cudaMemcpy(h->cg.bar + 2, w, sizeof w, cudaMemcpyHostToDevice));
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

int esdc_table_errors(int model, const double* params, int n_params, int M, double dt, double* err)
{
    if (!err || !params || M < 1 || M > ESDC_MMAX || !(dt > 0.0) || !std::isfinite(dt)) return ESDC_ERR_INVALID_ARG;
    const int need = model == ESDC_MODEL_HH1952 ? 7 : model == ESDC_MODEL_SYN19 ? 88 : -1;
    if (need < 0 || n_params != need) return ESDC_ERR_INVALID_ARG;
    for (int k = 0; k < n_params; ++k)
        if (!std::isfinite(params[k])) return ESDC_ERR_INVALID_ARG;
    std::vector<double> rows;
    if (esdc_vtab_build(model, params, rows, &err[0], &err[1]) == -1) return ESDC_ERR_INVALID_ARG;
    ColloData C;
    if (esdc_colloc_build(M, &C) != 0) return ESDC_ERR_INVALID_ARG;
    if (esdc_ztab_build(M, dt, C, rows, &err[2]) == -1) return ESDC_ERR_INVALID_ARG;
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

int esdc_fma_probe(int fp32, int64_t n, double* ms, double* flops, void* stream)
{
    if (!ms || !flops || n < 1 || (fp32 != 0 && fp32 != 1)) return ESDC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ESDC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256, per_sm = 4, blocks = sms * per_sm;
    double* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(double)) != cudaSuccess) return ESDC_ERR_NO_MEMORY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = ESDC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ESDC_ERR_CUDA;
    if (rc == ESDC_OK) {
        cudaEventRecord(e0, s);
        if (fp32) k_fma_probe<float><<<blocks, threads, 0, s>>>(sink, n, 0.999999f, 1e-6f);
        else k_fma_probe<double><<<blocks, threads, 0, s>>>(sink, n, 0.999999, 1e-6);
        cudaEventRecord(e1, s);
        float t = 0.0f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            rc = ESDC_ERR_CUDA;
        *ms = t;
        *flops = 2.0 * ESDC_FMA_CHAINS * (double)n * (double)blocks * threads;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
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
