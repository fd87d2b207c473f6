// Direct solve of the implicit diffusion rows by the DCT-II (Sec. 5: the
// paper's linear solver), for the scalar conductivity with the second- or the
// fourth-order stencil and mirrored ghost cells.
//
// With mirrored ghosts the cosine modes v_k(i) = cos(pi k (2i + 1)/(2n)) extend
// symmetrically across both ends of an axis, so they are eigenvectors of the
// one-dimensional difference operator of either order:
//   second order (-1, 2, -1)/h^2:            mu_k = -(4/h^2) sin^2(pi k/(2n))
//   fourth order (1, -16, 30, -16, 1)/(12h^2): mu_k = (32 cos t - 2 cos 2t - 30)/(12 h^2), t = pi k/n
// and the Laplacian of the box is their sum over the axes.  With U the
// unnormalised DCT-II of an axis (U[k][i] = cos(pi k (2i + 1)/(2n))), the
// orthonormal transform is diag(s) U with s_0^2 = 1/n, s_k^2 = 2/n, and
//   (I - g L)^{-1} = prod_axes (U^T diag(s^2)) diag(1/(1 - g sum_axes mu)) prod_axes U.
//
// How this file evaluates it, with FP64 operations as the scarce resource (a
// GB300 SM issues two FP64 lane operations per clock):
//  * x and y (and z for the fourth-order stencil): one kernel per axis and
//    direction.  A block loads a tile of lines into shared memory and
//    transforms each pair of real lines with one complex FFT (line a in the
//    real part, line b in the imaginary part), after Makhoul's reordering
//    (J. Makhoul, IEEE Trans. ASSP 28 (1980), "A fast cosine transform in one
//    and two dimensions"): v[m] = x[2m], v[n-1-m] = x[2m+1] gives
//    X[k] = Re(e^{-i pi k/(2n)} V[k]), V = DFT(v).  The FFT is a Stockham
//    decimation-in-time (Cooley-Tukey) in shared memory with radix-4 stages
//    (24 FP64 operations per four points) and one radix-2 stage when log2 n
//    is odd (see fft_pow2).  The inverse packs V[k] = e^{i pi k/(2n)}
//    (Y[k] - i Y[n-k]) and runs the same FFT on the conjugate.  Axes whose
//    length is not a power of two use a plain dense product with a cosine
//    table instead.
//  * z (second-order stencil): after the x and y transforms the operator is,
//    per mode (kx, ky), the tridiagonal a I - g L_z with a = 1 - g(mu_x + mu_y).
//    It is solved directly (Thomas' elimination) with its factors tabulated
//    once per value of g: r'_k = r_k A_k - r'_{k-1} C_k, x_k = r'_k - C_k x_{k+1},
//    three FP64 operations per node.  A 2D or 1D mesh has nz = 1, where this
//    reduces to the division by a.  When the y-z slab of one x-mode fits a
//    block (ny a power of two >= 16, nz >= 2), k_dct_yzy does the y forward
//    transform, these z solves and the y inverse transform of that x-mode in
//    shared memory: three kernels per solve (x forward, yzy, x inverse).
//  * Scaling: the inverse of this pair packing computes U^T diag(1, 1/2, ...,
//    1/2), so with the forward transform unnormalised, every transformed axis
//    contributes the same factor 1/n to the spectral weight.
// The solve is exact up to rounding: no iteration, no stop test.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "esdc_internal.h"

namespace {

constexpr int kDctMaxN = 4096;          // longest axis of the FFT path
constexpr int kDctSmemLimit = 200 * 1024;
constexpr int kDctDenseCheap = 32;      // dense axes' total length up to which the automatic choice takes the DCT
#ifndef ESDC_DCT_MAXPAIRS
#define ESDC_DCT_MAXPAIRS 2             // line pairs per block of an FFT pass beyond one warp's worth
#endif
#ifndef ESDC_DCT_ZTHREADS
#define ESDC_DCT_ZTHREADS 64            // threads per block of the z solve
#endif

struct AxisArgs {
    const double* src;
    double* dst;
    int n, logn;            // logn < 0: dense product
    int lines;              // number of lines (all index combinations of the other axes)
    int inner;              // element stride of the axis (1 for x)
    int lpt, loglpt;        // lines per tile (a power of two, at least 2)
    int G;                  // threads per line pair (FFT path)
    const double2* tw;      // [n] e^{-2 pi i k/n}
    const double2* csh;     // [n/2 + 1] (cos, sin)(pi k/(2n)) / 2 (forward)
    const double2* cs;      // [n/2 + 1] (cos, sin)(pi k/(2n))     (inverse)
    const double* dmat;     // dense path: [n][n], row = output index
};

// First element of line L: lines are all combinations (o, t) of the slower
// index o and the faster index t < inner; element i sits at base + i * inner.
__device__ __forceinline__ int line_base(const AxisArgs& a, int L)
{
    if (a.inner == 1) return L * a.n;
    const int o = L / a.inner, t = L - o * a.inner;
    return o * a.n * a.inner + t;
}

// The tile's line bases (-1 past the last line), one division per line.
__device__ __forceinline__ void tile_bases(const AxisArgs& a, int L0, int* base)
{
    if (threadIdx.x < a.lpt) {
        const int L = L0 + threadIdx.x;
        base[threadIdx.x] = L < a.lines ? line_base(a, L) : -1;
    }
}

// Tile element e -> (line in tile, element): along the line for x (contiguous
// lines), across lines for the strided axes (consecutive lines are adjacent
// in memory), so that consecutive threads touch consecutive addresses.
// Shifts and masks on the FFT path (n and lpt powers of two).
__device__ __forceinline__ void tile_pos(const AxisArgs& a, int e, int& l, int& i)
{
    if (a.inner == 1) {
        if (a.logn >= 0) { l = e >> a.logn; i = e & (a.n - 1); }
        else { l = e / a.n; i = e - l * a.n; }
    } else {
        i = e >> a.loglpt;
        l = e & (a.lpt - 1);
    }
}

// Barrier among the G threads of a line pair: the warp's when the pair lies
// within one warp, else the block's (all pairs of a block run the same stages).
__device__ __forceinline__ void pair_sync(int G)
{
    if (G > 32) __syncthreads();
    else __syncwarp();
}

// Stockham FFT (decimation in time) of n = 2^logn points held by the G
// threads g = 0..G-1 of a line pair; x -> y ping-pong, returns the buffer that
// holds the result.  Radix-4 stages while they fit, then one radix-2 stage if
// logn is odd.  A radix-4 stage combines sub-transforms of length Ns:
//   v_r = x[j + r n/4], w_r = e^{-2 pi i r k/(4 Ns)}, k = j mod Ns,
//   t0 = v0 + w2 v2, t1 = 2 v0 - t0, t2 = w1 v1 + w3 v3, t3 = 2 w1 v1 - t2,
//   y[4(j - k) + k + q Ns] = t0 + t2, t1 - i t3, t0 - t2, t1 + i t3  (q = 0..3),
// 24 FP64 operations per four points (the twiddle products fused into the
// sums); the first stage (w = 1) takes 16 additions.  The radix-2 stage is
//   y[2(j - k) + k] = a + w b, y[2(j - k) + k + Ns] = 2a - (a + w b).
// tw: e^{-2 pi i m/n}, m = 0..n-1, in shared memory.  Threads with
// active = false run the same loops without butterflies, so that every thread
// meets the same barriers.
__device__ __forceinline__ double2* fft_pow2(double2* x, double2* y, int n, int logn, int g, int G, bool active,
                                             const double2* tw)
{
    const int q4 = n >> 2;
    int Ns = 1;
    for (int s = 0; s + 2 <= logn; s += 2) {
        const int stride = n >> (s + 2);                 // n / (4 Ns)
        for (int j = active ? g : q4; j < q4; j += G) {
            const int k = j & (Ns - 1);
            const double2 v0 = x[j], v1 = x[j + q4], v2 = x[j + 2 * q4], v3 = x[j + 3 * q4];
            double t0r, t0i, t1r, t1i, t2r, t2i, t3r, t3i;
            if (s == 0) {
                t0r = v0.x + v2.x; t0i = v0.y + v2.y;
                t1r = v0.x - v2.x; t1i = v0.y - v2.y;
                t2r = v1.x + v3.x; t2i = v1.y + v3.y;
                t3r = v1.x - v3.x; t3i = v1.y - v3.y;
            } else {
                const double2 w1 = tw[k * stride], w2 = tw[2 * k * stride], w3 = tw[3 * k * stride];
                const double b1r = fma(w1.x, v1.x, -w1.y * v1.y), b1i = fma(w1.x, v1.y, w1.y * v1.x);
                t0r = fma(w2.x, v2.x, fma(-w2.y, v2.y, v0.x));
                t0i = fma(w2.x, v2.y, fma(w2.y, v2.x, v0.y));
                t1r = fma(2.0, v0.x, -t0r);
                t1i = fma(2.0, v0.y, -t0i);
                t2r = fma(w3.x, v3.x, fma(-w3.y, v3.y, b1r));
                t2i = fma(w3.x, v3.y, fma(w3.y, v3.x, b1i));
                t3r = fma(2.0, b1r, -t2r);
                t3i = fma(2.0, b1i, -t2i);
            }
            const int idx = ((j - k) << 2) + k;
            y[idx] = make_double2(t0r + t2r, t0i + t2i);
            y[idx + Ns] = make_double2(t1r + t3i, t1i - t3r);
            y[idx + 2 * Ns] = make_double2(t0r - t2r, t0i - t2i);
            y[idx + 3 * Ns] = make_double2(t1r - t3i, t1i + t3r);
        }
        pair_sync(G);
        double2* t = x; x = y; y = t;
        Ns <<= 2;
    }
    if (logn & 1) {                                      // the last stage: radix 2, Ns = n/2
        const int h = n >> 1;
        for (int j = active ? g : h; j < h; j += G) {
            const int k = j & (Ns - 1);
            const double2 a = x[j], b = x[j + h];
            const int idx = ((j - k) << 1) + k;
            double cr, ci, dr, di;
            if (Ns == 1) {
                cr = a.x + b.x; ci = a.y + b.y;
                dr = a.x - b.x; di = a.y - b.y;
            } else {
                const double2 w = tw[k];                 // e^{-2 pi i k/(2 Ns)} = e^{-2 pi i k/n}
                cr = fma(w.x, b.x, fma(-w.y, b.y, a.x));
                ci = fma(w.x, b.y, fma(w.y, b.x, a.y));
                dr = fma(2.0, a.x, -cr);
                di = fma(2.0, a.y, -ci);
            }
            y[idx] = make_double2(cr, ci);
            y[idx + Ns] = make_double2(dr, di);
        }
        pair_sync(G);
        double2* t = x; x = y; y = t;
    }
    return x;
}

// Position of x[i] in Makhoul's reordering v[m] = x[2m], v[n-1-m] = x[2m+1].
__device__ __forceinline__ int makhoul_pos(int i, int n) { return (i & 1) ? n - 1 - (i >> 1) : (i >> 1); }

// One tile of lines along one axis, FFT path.  FWD: X = U x (unnormalised
// DCT-II).  !FWD: y = U^T diag(1, 1/2, ..., 1/2) Y.  Shared memory: two
// complex buffers of P = lpt/2 pair rows with a pitch of n + 1 (bank offset
// between pair rows).
template <bool FWD>
__global__ void __launch_bounds__(256) k_dct_fft(AxisArgs a)
{
    extern __shared__ double2 smem_all[];
    const int n = a.n, pitch = n + 1, P = a.lpt >> 1;
    double2* stw = smem_all;                            // the twiddles e^{-2 pi i m/n}, m < n
    double2* sm = smem_all + n;                         // then the two tile buffers
    const size_t bstride = (size_t)P * pitch;           // buffer c starts at sm + c * bstride
    __shared__ int base[32];
    tile_bases(a, blockIdx.x * a.lpt, base);
    __syncthreads();
    // the twiddles (first used by the FFT stages) load together with the tile
    for (int m = threadIdx.x; m < n; m += blockDim.x) stw[m] = __ldg(a.tw + m);
    const int tile_elems = a.lpt * n;

    // load: line l of the tile into the real (l even) or imaginary (l odd)
    // part of pair row l/2 of buffer 0, at its reordered position (forward)
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        int l, i;
        tile_pos(a, e, l, i);
        const int b = base[l];
        const double v = b >= 0 ? a.src[b + i * a.inner] : 0.0;
        const int m = FWD ? makhoul_pos(i, n) : i;
        double* row = reinterpret_cast<double*>(sm + (size_t)(l >> 1) * pitch);
        row[2 * m + (l & 1)] = v;
    }
    __syncthreads();

    const int p0 = threadIdx.x / a.G, g = threadIdx.x - p0 * a.G;
    const bool active = p0 < P;
    const int p = active ? p0 : 0;
    const int h = n >> 1;
    int cur = 0;                                          // buffer holding the data
    if (!FWD) {
        // Z[k] = conj(Va[k] + i Vb[k]), Va[k] = e^{i th_k}(A[k] - i A[n-k]) (A[n] = 0),
        // th_k = pi k/(2n), and Z[n-k] from Va[n-k] = conj(Va[k]): buffer 0 -> 1
        const double2* x = sm + (size_t)p * pitch;
        double2* y = sm + bstride + (size_t)p * pitch;
        for (int k = active ? g : h + 1; k <= h; k += a.G) {
            if (k == 0) { y[0] = make_double2(x[0].x, -x[0].y); continue; }
            const double2 Ak = x[k], Am = x[n - k];     // (.x: line a, .y: line b)
            const double2 t = __ldg(a.cs + k);
            const double ar = fma(t.x, Ak.x, t.y * Am.x), ai = fma(t.y, Ak.x, -t.x * Am.x);
            const double br = fma(t.x, Ak.y, t.y * Am.y), bi = fma(t.y, Ak.y, -t.x * Am.y);
            y[k] = make_double2(ar - bi, -(ai + br));
            if (k < h) y[n - k] = make_double2(ar + bi, ai - br);
        }
        pair_sync(a.G);
        cur = 1;
    }
    double2* z = fft_pow2(sm + cur * bstride + (size_t)p * pitch, sm + (cur ^ 1) * bstride + (size_t)p * pitch, n,
                          a.logn, g, a.G, active, stw);
    cur = (cur + (a.logn >> 1) + (a.logn & 1)) & 1;     // the FFT ends in this buffer (one swap per stage)
    // the other buffer takes the real output rows: row l at pitch n + 1 doubles
    double* out = reinterpret_cast<double*>(sm + (cur ^ 1) * bstride);
    if (active) {
        double* ra = out + (size_t)(2 * p) * pitch;
        double* rb = ra + pitch;
        if (FWD) {
            // X[k] = Re(e^{-i th_k} V[k]); P = Z[k] + conj(Z[n-k]) = 2 Va[k],
            // Q = Z[k] - conj(Z[n-k]) = 2i Vb[k]; csh holds (cos, sin)/2
            for (int k = g; k <= h; k += a.G) {
                if (k == 0) { ra[0] = z[0].x; rb[0] = z[0].y; continue; }
                const double2 Zk = z[k], Zm = z[n - k];
                const double Pr = Zk.x + Zm.x, Pi = Zk.y - Zm.y;
                const double Qr = Zk.x - Zm.x, Qi = Zk.y + Zm.y;
                const double2 t = __ldg(a.csh + k);
                ra[k] = fma(t.x, Pr, t.y * Pi);
                rb[k] = fma(t.x, Qi, -t.y * Qr);
                if (k < h) {
                    ra[n - k] = fma(t.y, Pr, -t.x * Pi);
                    rb[n - k] = fma(t.y, Qi, t.x * Qr);
                }
            }
        } else {
            // y = conj(FFT(conj Z)), undone from the reordering
            for (int i = g; i < n; i += a.G) {
                const double2 v = z[makhoul_pos(i, n)];
                ra[i] = v.x;
                rb[i] = -v.y;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        int l, i;
        tile_pos(a, e, l, i);
        const int b = base[l];
        if (b >= 0) a.dst[b + i * a.inner] = out[l * pitch + i];
    }
}

// One tile of lines, dense path (any n): out[l][k] = sum_i in[l][i] dmat[k][i].
__global__ void k_dct_dense(AxisArgs a)
{
    extern __shared__ double2 sm[];
    const int n = a.n, pitch = n + 1;
    double* in = reinterpret_cast<double*>(sm);
    double* out = in + (size_t)a.lpt * pitch;
    __shared__ int base[32];
    tile_bases(a, blockIdx.x * a.lpt, base);
    __syncthreads();
    const int tile_elems = a.lpt * n;
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        int l, i;
        tile_pos(a, e, l, i);
        const int b = base[l];
        in[l * pitch + i] = b >= 0 ? a.src[b + i * a.inner] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        const int l = e / n, k = e - l * n;
        const double* row = in + l * pitch;
        const double* w = a.dmat + (size_t)k * n;
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = fma(row[i], __ldg(w + i), s);
        out[l * pitch + k] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        int l, i;
        tile_pos(a, e, l, i);
        const int b = base[l];
        if (b >= 0) a.dst[b + i * a.inner] = out[l * pitch + i];
    }
}

// Factor tables of the z-direction tridiagonal systems for one g (second
// order): per mode m = (kx, ky), a = 1 - g (mu_x + mu_y), off-diagonal e = -g/h^2,
// diagonal d_k = a + (g/h^2) (number of z-neighbours of layer k);
// inv_k = 1/(d_k - e C_{k-1}), A_k = w inv_k, C_k = e inv_k, with w the
// spectral weight of the transformed axes.
// Layout: [z][ky][kx] (the z kernel), or [kx][z][ky] (yzy: the fused kernel's
// blocks read their kx contiguously).
__global__ void k_dct_ztab(DctDev d, int nx, int ny, int nz, double ih2, double g, double w,
                           double* A, double* C, bool yzy)
{
    const int sxy = nx * ny;
    const double e = -g * ih2;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < sxy; m += gridDim.x * blockDim.x) {
        const int ky = m / nx, kx = m - ky * nx;
        const double a = 1.0 - g * (d.ex[kx] + d.ey[ky]);
        double cprev = 0.0;
        for (int k = 0; k < nz; ++k) {
            const int nb = (k > 0) + (k < nz - 1);
            const double inv = 1.0 / ((a + g * ih2 * nb) - e * cprev);
            const size_t q = yzy ? ((size_t)kx * nz + k) * ny + ky : (size_t)k * sxy + m;
            A[q] = w * inv;
            cprev = e * inv;
            C[q] = cprev;
        }
    }
}

// The z-direction solves (second order) on the transformed data, with the
// spectral weight folded into A; records the solve in the status words and
// flags a non-finite result.  One thread per mode; the loads of ZCH layers
// are issued together before the recurrence uses them (one L2 round trip per
// chunk instead of one per layer).
constexpr int ZCH = 8;
__global__ void __launch_bounds__(ESDC_DCT_ZTHREADS) k_dct_z(const double* __restrict__ src, double* __restrict__ dst,
                                              const double* __restrict__ A, const double* __restrict__ C, int nx,
                                              int ny, int nz, int* status, int* iter_log, int* flags)
{
    const int sxy = nx * ny;
    bool bad = false;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < sxy; m += gridDim.x * blockDim.x) {
        double rp = 0.0;
        for (int c0 = 0; c0 < nz; c0 += ZCH) {
            double sv[ZCH], av[ZCH], cv[ZCH];
#pragma unroll
            for (int j = 0; j < ZCH; ++j) {
                const int k = c0 + j;
                if (k < nz) {
                    const int q = k * sxy + m;
                    sv[j] = src[q];
                    av[j] = A[q];
                    cv[j] = C[q];
                }
            }
#pragma unroll
            for (int j = 0; j < ZCH; ++j) {
                const int k = c0 + j;
                if (k < nz) {
                    rp = fma(sv[j], av[j], -rp * cv[j]);
                    dst[k * sxy + m] = rp;
                }
            }
        }
        double xn = rp;
        bad |= !isfinite(xn);
        for (int c1 = nz - 1; c1 > 0; c1 -= ZCH) {          // layers c1-1 down to c1-ZCH
            double rv[ZCH], cv[ZCH];
#pragma unroll
            for (int j = 0; j < ZCH; ++j) {
                const int k = c1 - 1 - j;
                if (k >= 0) {
                    const int q = k * sxy + m;
                    rv[j] = dst[q];
                    cv[j] = C[q];
                }
            }
#pragma unroll
            for (int j = 0; j < ZCH; ++j) {
                const int k = c1 - 1 - j;
                if (k >= 0) {
                    xn = fma(-cv[j], xn, rv[j]);
                    dst[k * sxy + m] = xn;
                    bad |= !isfinite(xn);
                }
            }
        }
    }
    if (bad) atomicOr(flags, ESDC_FLAG_NONFINITE);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status[0] = 1;
        if (iter_log) *iter_log = 1;
    }
}

// The y forward transform, the z solves and the y inverse transform of the
// second-order solve in one kernel: block kx holds the y-z slab of x-mode kx
// (nz lines of n = ny values, paired into (nz + 1)/2 complex lines) in shared
// memory, transforms it along y (as k_dct_fft), solves the tridiagonal z
// system of every y-mode ky in place (as k_dct_z, factors in the [kx][z][ky]
// layout, loaded into shared memory with the data), transforms back and
// stores it.  One pass over the data instead of three, and the z recurrences
// read shared memory.
struct YzyArgs {
    const double* src;
    double* dst;
    int nx, n, logn, nz, pairs, G;
    const double2* tw;                  // y axis: [n] e^{-2 pi i k/n}
    const double2* csh;                 // [n/2 + 1] (cos, sin)(pi k/(2n)) / 2
    const double2* cs;                  // [n/2 + 1] (cos, sin)(pi k/(2n))
    const double* A;                    // [nx][nz][n]
    const double* C;
    int* status;
    int* iter_log;
    int* flags;
};

__global__ void __launch_bounds__(1024) k_dct_yzy(YzyArgs a)
{
    extern __shared__ double2 smem_all[];
    const int n = a.n, pitch = n + 1, P = a.pairs, nz = a.nz, nx = a.nx, h = n >> 1;
    const int kx = blockIdx.x;
    double2* stw = smem_all;
    double2* sm = smem_all + n;
    const size_t bstride = (size_t)P * pitch;
    double* zA = reinterpret_cast<double*>(sm + 2 * bstride);   // this kx's z factors, [z][ky]
    double* zC = zA + (size_t)nz * n;
    for (int m = threadIdx.x; m < n; m += blockDim.x) stw[m] = __ldg(a.tw + m);
    // the factors load with the data (contiguous per kx), used after the forward transform
    for (int e = threadIdx.x; e < nz * n; e += blockDim.x) {
        zA[e] = __ldg(a.A + (size_t)kx * nz * n + e);
        zC[e] = __ldg(a.C + (size_t)kx * nz * n + e);
    }
    // line z (its n values along y) into the real (z even) or imaginary part of
    // pair row z/2 of buffer 0, at its reordered position; a missing last line is 0
    for (int e = threadIdx.x; e < 2 * P * n; e += blockDim.x) {
        const int z = e >> a.logn, y = e & (n - 1);
        const double v = z < nz ? a.src[((size_t)z * n + y) * nx + kx] : 0.0;
        double* row = reinterpret_cast<double*>(sm + (size_t)(z >> 1) * pitch);
        row[2 * makhoul_pos(y, n) + (z & 1)] = v;
    }
    __syncthreads();
    const int p0 = threadIdx.x / a.G, g = threadIdx.x - p0 * a.G;
    const bool active = p0 < P;
    const int p = active ? p0 : 0;
    const int stages = (a.logn >> 1) + (a.logn & 1);
    // forward along y: buffer 0 -> buffer c1; real rows of X into buffer c1 ^ 1
    const double2* zf = fft_pow2(sm + (size_t)p * pitch, sm + bstride + (size_t)p * pitch, n, a.logn, g, a.G, active,
                                 stw);
    const int c1 = stages & 1;
    double* rows = reinterpret_cast<double*>(sm + (size_t)(c1 ^ 1) * bstride);   // row z at pitch n + 1 doubles
    if (active) {
        double* ra = rows + (size_t)(2 * p) * pitch;
        double* rb = ra + pitch;
        for (int k = g; k <= h; k += a.G) {
            if (k == 0) { ra[0] = zf[0].x; rb[0] = zf[0].y; continue; }
            const double2 Zk = zf[k], Zm = zf[n - k];
            const double Pr = Zk.x + Zm.x, Pi = Zk.y - Zm.y;
            const double Qr = Zk.x - Zm.x, Qi = Zk.y + Zm.y;
            const double2 t = __ldg(a.csh + k);
            ra[k] = fma(t.x, Pr, t.y * Pi);
            rb[k] = fma(t.x, Qi, -t.y * Qr);
            if (k < h) {
                ra[n - k] = fma(t.y, Pr, -t.x * Pi);
                rb[n - k] = fma(t.y, Qi, t.x * Qr);
            }
        }
    }
    __syncthreads();
    // z: the tridiagonal system of y-mode ky, in place in the real rows
    bool bad = false;
    for (int ky = threadIdx.x; ky < n; ky += blockDim.x) {
        double rp = 0.0;
        for (int z = 0; z < nz; ++z) {
            rp = fma(rows[(size_t)z * pitch + ky], zA[(size_t)z * n + ky], -rp * zC[(size_t)z * n + ky]);
            rows[(size_t)z * pitch + ky] = rp;
        }
        double xn = rp;
        bad |= !isfinite(xn);
        for (int z = nz - 2; z >= 0; --z) {
            xn = fma(-zC[(size_t)z * n + ky], xn, rows[(size_t)z * pitch + ky]);
            rows[(size_t)z * pitch + ky] = xn;
            bad |= !isfinite(xn);
        }
    }
    if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = 1;
        if (a.iter_log) *a.iter_log = 1;
    }
    __syncthreads();
    // inverse along y: the real rows (buffer c1 ^ 1) packed into buffer c1 as in
    // k_dct_fft, then the FFT; a pair writes only its own two rows' storage
    double2* xi = sm + (size_t)c1 * bstride + (size_t)p * pitch;
    if (active) {
        const double* ra = rows + (size_t)(2 * p) * pitch;
        const double* rb = ra + pitch;
        for (int k = g; k <= h; k += a.G) {
            if (k == 0) { xi[0] = make_double2(ra[0], -rb[0]); continue; }
            const double Akx = ra[k], Aky = rb[k], Amx = ra[n - k], Amy = rb[n - k];
            const double2 t = __ldg(a.cs + k);
            const double ar = fma(t.x, Akx, t.y * Amx), ai = fma(t.y, Akx, -t.x * Amx);
            const double br = fma(t.x, Aky, t.y * Amy), bi = fma(t.y, Aky, -t.x * Amy);
            xi[k] = make_double2(ar - bi, -(ai + br));
            if (k < h) xi[n - k] = make_double2(ar + bi, ai - br);
        }
    }
    pair_sync(a.G);
    const double2* zi = fft_pow2(xi, sm + (size_t)(c1 ^ 1) * bstride + (size_t)p * pitch, n, a.logn, g, a.G, active,
                                 stw);
    const int c2 = (c1 + stages) & 1;
    double* out = reinterpret_cast<double*>(sm + (size_t)(c2 ^ 1) * bstride);
    if (active) {
        double* ra = out + (size_t)(2 * p) * pitch;
        double* rb = ra + pitch;
        for (int i = g; i < n; i += a.G) {
            const double2 v = zi[makhoul_pos(i, n)];
            ra[i] = v.x;
            rb[i] = -v.y;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nz * n; e += blockDim.x) {
        const int z = e >> a.logn, y = e & (n - 1);
        a.dst[((size_t)z * n + y) * nx + kx] = out[(size_t)z * pitch + y];
    }
}

// Spectral division of the fourth-order solve (all axes transformed):
// x_hat *= w / (1 - g (ex[kx] + ey[ky] + ez[kz])).
__global__ void __launch_bounds__(256) k_dct_scale(DctDev d, int nx, int ny, int nz, double g, double w, double* xh,
                                                   int* status, int* iter_log, int* flags)
{
    const int N = nx * ny * nz;
    bool bad = false;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int r = p / nx, kx = p - r * nx;
        const int kz = r / ny, ky = r - kz * ny;
        const double v = w * xh[p] / (1.0 - g * ((d.ex[kx] + d.ey[ky]) + d.ez[kz]));
        xh[p] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(flags, ESDC_FLAG_NONFINITE);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status[0] = 1;
        if (iter_log) *iter_log = 1;
    }
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

int log2_exact(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return ((1 << l) == n && n >= 2 && n <= kDctMaxN) ? l : -1;
}

template <class T>
cudaError_t upload(const T** dst, const std::vector<T>& v)
{
    T* p = nullptr;
    cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    *dst = p;
    return cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Twiddle and post-processing tables of an axis (FFT path) or its two dense
// matrices (forward U, inverse U^T diag(1, 1/2, ..., 1/2) scaled by 2: see
// dense_inverse below).
cudaError_t axis_tables(DctAxisDev& ax, int n)
{
    ax = DctAxisDev{};
    ax.n = n;
    ax.logn = log2_exact(n);
    if (n == 1) return cudaSuccess;
    if (ax.logn >= 0) {
        std::vector<double2> tw(n), csh(n / 2 + 1), cs(n / 2 + 1);
        for (int k = 0; k < n; ++k)
            tw[k] = make_double2(std::cos(2.0 * M_PI * k / n), -std::sin(2.0 * M_PI * k / n));
        for (int k = 0; k <= n / 2; ++k) {
            const double c = std::cos(M_PI * k / (2.0 * n)), s = std::sin(M_PI * k / (2.0 * n));
            cs[k] = make_double2(c, s);
            csh[k] = make_double2(0.5 * c, 0.5 * s);
        }
        cudaError_t e;
        if ((e = upload(&ax.tw, tw)) != cudaSuccess) return e;
        if ((e = upload(&ax.csh, csh)) != cudaSuccess) return e;
        return upload(&ax.cs, cs);
    }
    // Dense: forward F[k][i] = cos(pi k (2i+1)/(2n)); inverse B[i][k] = c_k cos(pi k (2i+1)/(2n))
    // with c_0 = 1, c_k = 2 for k >= 1, so that B F = n I and the spectral weight
    // of the axis is 1/n, as on the FFT path.
    std::vector<double> F((size_t)n * n), B((size_t)n * n);
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) {
            const double c = std::cos(M_PI * k * (2.0 * i + 1.0) / (2.0 * n));
            F[(size_t)k * n + i] = c;
            B[(size_t)i * n + k] = (k == 0 ? 1.0 : 2.0) * c;
        }
    cudaError_t e;
    if ((e = upload(&ax.fwd, F)) != cudaSuccess) return e;
    return upload(&ax.inv, B);
}

void axis_free(DctAxisDev& ax)
{
    const void* ptrs[] = {ax.tw, ax.csh, ax.cs, ax.fwd, ax.inv};
    for (const void* p : ptrs)
        if (p) cudaFree(const_cast<void*>(p));
    ax = DctAxisDev{};
}

int g_sms = 0;

// Launch shape of one axis pass.  FFT path: n/4 threads per line pair (one
// radix-4 butterfly per thread and stage; at most 256), pairs per block enough
// to fill a warp, else ESDC_DCT_MAXPAIRS; a 128-point line pair is one warp,
// so its stages meet at warp barriers.  Small blocks spread the tiles evenly
// over the SMs (measured on the 128x128x32 slab: 2 pairs of 128-point lines
// per block solve 3.8% faster than 8).  Dense path: 128 threads per
// block of up to 32 lines.  Both keep the tile's shared memory below
// kDctSmemLimit.
void axis_shape(const DctAxisDev& ax, int lines, AxisArgs& a, int& threads, size_t& smem, int& tiles)
{
    const int n = ax.n;
    int lpt;
    if (ax.logn >= 0) {
        int G = n / 4;
        if (G < 1) G = 1;
        if (G > 256) G = 256;
        int P = 32 / G > ESDC_DCT_MAXPAIRS ? 32 / G : ESDC_DCT_MAXPAIRS;
        if (P > 256 / G) P = 256 / G;
        if (P > 16) P = 16;                                      // lpt <= 32: the tile's line bases
        if (P < 1) P = 1;
        lpt = 2 * P;
        while (lpt > 2 && (size_t)(lpt * (n + 1) + n) * 16 > (size_t)kDctSmemLimit) lpt >>= 1;
        a.G = G;
        threads = (lpt / 2) * G;
        threads = (threads + 31) / 32 * 32;
        smem = (size_t)(lpt * (n + 1) + n) * sizeof(double2);   // twiddles + 2 buffers x lpt/2 pairs x (n+1)
    } else {
        lpt = 32;
        while (lpt > 2 && (size_t)lpt * (n + 1) * 16 > (size_t)kDctSmemLimit) lpt >>= 1;
        a.G = 1;
        threads = 128;
        smem = (size_t)2 * lpt * (n + 1) * sizeof(double);
    }
    a.n = n;
    a.logn = ax.logn;
    a.lpt = lpt;
    a.loglpt = 0;
    while ((1 << a.loglpt) < lpt) ++a.loglpt;
    a.lines = lines;
    tiles = (lines + lpt - 1) / lpt;
}

cudaError_t axis_pass(const DctAxisDev& ax, bool fwd, const double* src, double* dst, int lines, int inner,
                      cudaStream_t s)
{
    AxisArgs a{};
    int threads;
    size_t smem;
    int tiles;
    axis_shape(ax, lines, a, threads, smem, tiles);
    a.src = src;
    a.dst = dst;
    a.inner = inner;
    a.tw = ax.tw;
    a.csh = ax.csh;
    a.cs = ax.cs;
    a.dmat = fwd ? ax.fwd : ax.inv;
    if (ax.logn >= 0) {
        if (fwd) k_dct_fft<true><<<(unsigned)tiles, threads, smem, s>>>(a);
        else k_dct_fft<false><<<(unsigned)tiles, threads, smem, s>>>(a);
    } else {
        k_dct_dense<<<(unsigned)tiles, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t prepare_kernels()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int lim = kDctSmemLimit + 4096;
    if ((e = cudaFuncSetAttribute(k_dct_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_dct_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_dct_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_dct_yzy, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    done = true;
    return cudaSuccess;
}

}  // namespace

bool esdc_dct_supported(const MeshDev& m)
{
    // every axis length is accepted (FFT for powers of two up to kDctMaxN,
    // dense products otherwise); the dense tile of the longest axis must fit
    const int n[3] = {m.nx, m.ny, m.nz};
    for (int a = 0; a < 3; ++a)
        if (n[a] > 1 && log2_exact(n[a]) < 0 && (size_t)2 * 2 * (n[a] + 1) * 8 > (size_t)kDctSmemLimit) return false;
    return true;
}

bool esdc_dct_cheap(const MeshDev& m, int order)
{
    const int n[3] = {m.nx, m.ny, order == 4 ? m.nz : 1};
    int dense = 0;
    for (int a = 0; a < 3; ++a)
        if (n[a] > 1 && log2_exact(n[a]) < 0) dense += n[a];
    return dense <= kDctDenseCheap;
}

cudaError_t esdc_dct_create(const MeshDev& m, int nslot, DctDev* d)
{
    *d = DctDev{};
    cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    const int n[3] = {m.nx, m.ny, m.nz};
    DctAxisDev* ax[3] = {&d->ax, &d->ay, &d->az};
    for (int a = 0; a < 3; ++a)
        if ((e = axis_tables(*ax[a], n[a])) != cudaSuccess) return e;
    if (nslot < 1) nslot = 1;
    if (nslot > ESDC_DCT_SLOTS) nslot = ESDC_DCT_SLOTS;
    d->nslot = nslot;
    const size_t bytes = sizeof(double) * 2 * (size_t)m.N * nslot;
    if ((e = cudaMalloc((void**)&d->ztab, bytes)) != cudaSuccess) return e;
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
    for (int k = 0; k < ESDC_DCT_SLOTS; ++k) d->used[k] = false;   // the z tables follow the eigenvalues
    d->cheap = esdc_dct_cheap(m, m.order);
    // the fused y-z kernel: second order, y of power-of-two length >= 16, and a
    // y-z slab that fits a block (threads and shared memory)
    d->yzy = false;
    if (m.order == 2 && m.nz >= 2 && m.ny >= 16 && log2_exact(m.ny) >= 0) {
        const int n = m.ny, G = n / 4 < 256 ? n / 4 : 256, P = (m.nz + 1) / 2;
        const int threads = (P * G + 31) / 32 * 32;
        const size_t smem = (size_t)(n + 2 * (size_t)P * (n + 1)) * sizeof(double2) +
                            2 * (size_t)m.nz * n * sizeof(double);          // + the z factors
        if (threads <= 1024 && smem <= (size_t)kDctSmemLimit) {
            d->yzy = true;
            d->yzy_threads = threads;
            d->yzy_smem = smem;
        }
    }
    return cudaSuccess;
}

void esdc_dct_destroy(DctDev* d)
{
    axis_free(d->ax);
    axis_free(d->ay);
    axis_free(d->az);
    double* ptrs[] = {d->ex, d->ey, d->ez, d->ztab};
    for (double* p : ptrs)
        if (p) cudaFree(p);
    *d = DctDev{};
}

cudaError_t esdc_dct_launch(const MeshDev& m, const CgWork& w, double g, const double* b, double* x,
                            int* iter_log, int* flags, cudaStream_t s)
{
    DctDev& d = *w.dct;
    const int nx = m.nx, ny = m.ny, nz = m.nz;
    const int N = m.N, sxy = nx * ny;
    cudaError_t e;
    double* bufs[2] = {w.r, w.p};
    int nb = 0;
    const double* src = b;
    auto next = [&]() { double* o = bufs[nb]; nb ^= 1; return o; };
    double wgt = 1.0;
    // forward: x, then y (then z for the fourth order)
    if (nx > 1) {
        double* o = next();
        if ((e = axis_pass(d.ax, true, src, o, N / nx, 1, s)) != cudaSuccess) return e;
        src = o;
        wgt /= nx;
    }
    const bool yzy = m.order == 2 && d.yzy;        // y forward, z, y inverse in k_dct_yzy
    if (ny > 1) {
        if (!yzy) {
            double* o = next();
            if ((e = axis_pass(d.ay, true, src, o, N / ny, nx, s)) != cudaSuccess) return e;
            src = o;
        }
        wgt /= ny;
    }
    if (m.order == 2) {
        // tables of this g (cached per value of g)
        int slot = -1;
        for (int k = 0; k < d.nslot; ++k)
            if (d.used[k] && d.gkey[k] == g) { slot = k; break; }
        double* A;
        double* C;
        if (slot < 0) {
            slot = d.next_slot;
            d.next_slot = (d.next_slot + 1) % d.nslot;
            A = d.ztab + (size_t)2 * N * slot;
            C = A + N;
            const int nblk = (sxy + 127) / 128;
            k_dct_ztab<<<(unsigned)(nblk < 4096 ? nblk : 4096), 128, 0, s>>>(d, nx, ny, nz, m.ih2, g, wgt, A, C, yzy);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            d.used[slot] = true;
            d.gkey[slot] = g;
        }
        A = d.ztab + (size_t)2 * N * slot;
        C = A + N;
        if (yzy) {
            double* o = nx > 1 ? next() : x;
            YzyArgs ya{};
            ya.src = src;
            ya.dst = o;
            ya.nx = nx;
            ya.n = ny;
            ya.logn = d.ay.logn;
            ya.nz = nz;
            ya.pairs = (nz + 1) / 2;
            ya.G = ny / 4 < 256 ? ny / 4 : 256;
            ya.tw = d.ay.tw;
            ya.csh = d.ay.csh;
            ya.cs = d.ay.cs;
            ya.A = A;
            ya.C = C;
            ya.status = w.status;
            ya.iter_log = iter_log;
            ya.flags = flags;
            k_dct_yzy<<<(unsigned)nx, (unsigned)d.yzy_threads, d.yzy_smem, s>>>(ya);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            src = o;
        } else {
            double* o = next();
            const int nblk = (sxy + ESDC_DCT_ZTHREADS - 1) / ESDC_DCT_ZTHREADS;
            k_dct_z<<<(unsigned)(nblk < 65535 ? nblk : 65535), ESDC_DCT_ZTHREADS, 0, s>>>(src, o, A, C, nx, ny, nz,
                                                                                       w.status, iter_log, flags);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            src = o;
        }
    } else {
        if (nz > 1) {
            double* o = next();
            if ((e = axis_pass(d.az, true, src, o, sxy, sxy, s)) != cudaSuccess) return e;
            src = o;
            wgt /= nz;
        }
        if (src == b) {                              // a box of one cell: b into a work vector first
            double* o = next();
            if ((e = cudaMemcpyAsync(o, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
            src = o;
        }
        double* xh = const_cast<double*>(src);
        int nblk = (N + 255) / 256;
        if (nblk > 4096) nblk = 4096;
        k_dct_scale<<<nblk, 256, 0, s>>>(d, nx, ny, nz, g, wgt, xh, w.status, iter_log, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (nz > 1) {
            double* o = (nx > 1 || ny > 1) ? next() : x;
            if ((e = axis_pass(d.az, false, src, o, sxy, sxy, s)) != cudaSuccess) return e;
            src = o;
        }
    }
    // inverse: y, then x; the last stage writes x
    if (ny > 1 && !yzy) {
        double* o = nx > 1 ? next() : x;
        if ((e = axis_pass(d.ay, false, src, o, N / ny, nx, s)) != cudaSuccess) return e;
        src = o;
    }
    if (nx > 1) {
        if ((e = axis_pass(d.ax, false, src, x, N / nx, 1, s)) != cudaSuccess) return e;
        src = x;
    }
    if (src != x) return cudaMemcpyAsync(x, src, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}
