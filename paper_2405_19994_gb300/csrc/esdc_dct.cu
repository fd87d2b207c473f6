// Direct solve of the implicit diffusion rows by the DCT-II (Sec. 5: the
// paper's linear solver), for the scalar conductivity with the second- or the
// fourth-order stencil and mirrored ghost cells.
//
// With mirrored ghosts the cosine modes v_k(i) = cos(pi k (i + 1/2)/n) extend
// symmetrically across both ends of an axis, so they are eigenvectors of the
// one-dimensional difference operator of either order:
//   second order (-1, 2, -1)/h^2:            mu_k = -(4/h^2) sin^2(pi k/(2n))
//   fourth order (1, -16, 30, -16, 1)/(12h^2): mu_k = (32 cos t - 2 cos 2t - 30)/(12 h^2), t = pi k/n
// and the Laplacian of the box is their sum over the axes.  With C the
// orthonormal DCT-II matrix of each axis (C[k][i] = s_k cos(pi k (i + 1/2)/n),
// s_0 = sqrt(1/n), s_k = sqrt(2/n)), the solution of (I - g L) x = b is
//   x = (Cx^T Cy^T Cz^T) diag(1/(1 - g (mu_x + mu_y + mu_z))) (Cz Cy Cx) b.
// Each axis transform is a plain dense matrix product over all lines of the
// box (cuBLAS DGEMM); the spectral division is this file's own kernel.  The
// solve is exact up to rounding: no iteration, no stop test.
#include <cmath>
#include <cstdio>
#include <vector>

#include <cublas_v2.h>

#include "esdc_internal.h"

namespace {

// x_hat /= 1 - g (ex[kx] + ey[ky] + ez[kz]); also records the solve in the
// status words (one "iteration") and flags a non-finite result.
__global__ void __launch_bounds__(256) k_dct_scale(DctDev d, int nx, int ny, int nz, double g, double* xh,
                                                   int* status, int* iter_log, int* flags)
{
    const long long N = (long long)nx * ny * nz;
    bool bad = false;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(p % nx);
        const long long r = p / nx;
        const int ky = (int)(r % ny);
        const int kz = (int)(r / ny);
        const double v = xh[p] / (1.0 - g * ((d.ex[kx] + d.ey[ky]) + d.ez[kz]));
        xh[p] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(flags, ESDC_FLAG_NONFINITE);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status[0] = 1;
        if (iter_log) *iter_log = 1;
    }
}

// Orthonormal DCT-II matrix of n points in column-major order: element (k, i)
// at [k + i n] is s_k cos(pi k (i + 1/2)/n).
std::vector<double> dct_matrix(int n)
{
    std::vector<double> c((size_t)n * n);
    const double s0 = std::sqrt(1.0 / n), s1 = std::sqrt(2.0 / n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k)
            c[(size_t)k + (size_t)i * n] = (k == 0 ? s0 : s1) * std::cos(M_PI * k * (i + 0.5) / n);
    return c;
}

std::vector<double> axis_eigs(int n, double ih2, int order)
{
    std::vector<double> e(n, 0.0);
    if (n == 1) return e;
    for (int k = 0; k < n; ++k) {
        if (order == 2) {
            const double s = std::sin(M_PI * k / (2.0 * n));
            e[k] = -4.0 * ih2 * s * s;
        } else {
            const double t = M_PI * k / n;
            e[k] = (32.0 * std::cos(t) - 2.0 * std::cos(2.0 * t) - 30.0) * ih2 / 12.0;
        }
    }
    return e;
}

cudaError_t upload(double** dst, const std::vector<double>& v)
{
    cudaError_t e = cudaMalloc((void**)dst, sizeof(double) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
}

cudaError_t blas_err(cublasStatus_t s)
{
    return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess
         : s == CUBLAS_STATUS_ALLOC_FAILED ? cudaErrorMemoryAllocation : cudaErrorUnknown;
}

}  // namespace

cudaError_t esdc_dct_create(const MeshDev& m, DctDev* d)
{
    *d = DctDev{};
    cublasHandle_t hb = nullptr;
    if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    d->blas = hb;
    // plain FP64 products: no emulation of FP64 by lower-precision tensor-core passes
    if (cublasSetMathMode(hb, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const int n[3] = {m.nx, m.ny, m.nz};
    double** c[3] = {&d->cx, &d->cy, &d->cz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] == 1) continue;
        cudaError_t e = upload(c[a], dct_matrix(n[a]));
        if (e != cudaSuccess) return e;
    }
    return esdc_dct_set_order(m, d);
}

cudaError_t esdc_dct_set_order(const MeshDev& m, DctDev* d)
{
    const int n[3] = {m.nx, m.ny, m.nz};
    double** e[3] = {&d->ex, &d->ey, &d->ez};
    for (int a = 0; a < 3; ++a) {
        const std::vector<double> v = axis_eigs(n[a], m.ih2, m.order);
        cudaError_t err = cudaSuccess;
        if (!*e[a]) err = cudaMalloc((void**)e[a], sizeof(double) * v.size());
        if (err == cudaSuccess) err = cudaMemcpy(*e[a], v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

void esdc_dct_destroy(DctDev* d)
{
    if (d->blas) cublasDestroy((cublasHandle_t)d->blas);
    double* ptrs[] = {d->cx, d->cy, d->cz, d->ex, d->ey, d->ez};
    for (double* p : ptrs)
        if (p) cudaFree(p);
    *d = DctDev{};
}

cudaError_t esdc_dct_launch(const MeshDev& m, const CgWork& w, double g, const double* b, double* x,
                            int* iter_log, int* flags, cudaStream_t s)
{
    const DctDev& d = *w.dct;
    cublasHandle_t hb = (cublasHandle_t)d.blas;
    cudaError_t e = blas_err(cublasSetStream(hb, s));
    if (e != cudaSuccess) return e;
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const long long sxy = (long long)nx * ny;
    const double one = 1.0, zero = 0.0;
    // The data moves b -> t1 -> t2 -> t1 ...; axes of one cell are the identity and are skipped.
    const double* src = b;
    double* bufs[2] = {w.r, w.p};
    int nb = 0;
    auto next = [&]() { return bufs[nb]; };
    auto done = [&](double* out) { src = out; nb ^= 1; };
    // forward: x, then y (per z-plane), then z
    if (nx > 1) {
        double* out = next();
        if ((e = blas_err(cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, nx, ny * nz, nx, &one, d.cx, nx, src, nx,
                                      &zero, out, nx))) != cudaSuccess)
            return e;
        done(out);
    }
    if (ny > 1) {
        double* out = next();
        if ((e = blas_err(cublasDgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_T, nx, ny, ny, &one, src, nx, sxy,
                                                    d.cy, ny, 0, &zero, out, nx, sxy, nz))) != cudaSuccess)
            return e;
        done(out);
    }
    if (nz > 1) {
        double* out = next();
        if ((e = blas_err(cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, (int)sxy, nz, nz, &one, src, (int)sxy, d.cz, nz,
                                      &zero, out, (int)sxy))) != cudaSuccess)
            return e;
        done(out);
    }
    // spectral division (in place; a box of one cell still needs b copied to a work vector)
    if (src == b) {
        double* out = next();
        if ((e = cudaMemcpyAsync(out, b, sizeof(double) * m.N, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        done(out);
    }
    double* xh = const_cast<double*>(src);
    {
        const long long N = m.N;
        long long nblk = (N + 255) / 256;
        if (nblk > 4096) nblk = 4096;
        k_dct_scale<<<(int)nblk, 256, 0, s>>>(d, nx, ny, nz, g, xh, w.status, iter_log, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // inverse: z, then y, then x; the last stage writes x
    int stages = (nx > 1) + (ny > 1) + (nz > 1);
    auto target = [&]() { return --stages == 0 ? x : next(); };
    if (nz > 1) {
        double* out = target();
        if ((e = blas_err(cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, (int)sxy, nz, nz, &one, src, (int)sxy, d.cz, nz,
                                      &zero, out, (int)sxy))) != cudaSuccess)
            return e;
        done(out);
    }
    if (ny > 1) {
        double* out = target();
        if ((e = blas_err(cublasDgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, nx, ny, ny, &one, src, nx, sxy,
                                                    d.cy, ny, 0, &zero, out, nx, sxy, nz))) != cudaSuccess)
            return e;
        done(out);
    }
    if (nx > 1) {
        double* out = target();
        if ((e = blas_err(cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, nx, ny * nz, nx, &one, d.cx, nx, src, nx,
                                      &zero, out, nx))) != cudaSuccess)
            return e;
        done(out);
    }
    if (src != x) return cudaMemcpyAsync(x, src, sizeof(double) * m.N, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}
