// Matrix-free iterative solves of the implicit diffusion rows of the HSDC
// preconditioner (eq. def_P: the f_I(y_{n,i}) term is taken implicitly, so each
// node solves (I - g L) V_i = rhs with g = dt d_i sigma/(chi C_m)), one node per
// thread: Jacobi-preconditioned conjugate gradients (k_cg), the Chebyshev
// semi-iteration on a known spectrum interval (k_cheb), and the precision
// form's refinement (k_cg_mixed); esdc_cg_launch also dispatches to the quad
// form (esdc_cg4.cu) and the DCT-II solve (esdc_dct.cu).  The paper solves these
// systems with DCT-II (Sec. 5).
//
// One cooperative launch runs the whole solve: the blocks stay resident and
// meet at a grid barrier (bounded spin; on timeout a flag is raised and every
// block returns).  Dot products are reduced deterministically: each block
// writes one partial per quantity, and after the barrier every block sums the
// partials in block order, so all blocks take identical control decisions.
// Each phase writes its own partial slots (set-up 0-2, [A] 3, [B] 4-5), so a
// slot is rewritten only after every block has passed a later barrier and so
// finished reading it.
#include <cooperative_groups.h>

#include "esdc_internal.h"
#include "esdc_cg_common.cuh"
#include "esdc_fmath.cuh"

namespace {

// (I - g L) v at node p (L: mirrored-ghost 3/5/7-point Laplacian) and the
// number of in-domain neighbours.  The vectors are rewritten by other blocks
// between phases, so neighbour values are read with __ldcg (L2, coherent).
// Layered anisotropic operator (A v)_p (coefficients include sigma and 1/h^2).
__device__ __forceinline__ double layered_A(const MeshDev& m, const double* v, int p, NodeIdx n, double vp)
{
    const int sxy = m.nx * m.ny;
    const double cxx = __ldg(m.lay + n.iz), cyy = __ldg(m.lay + m.nz + n.iz), cd = __ldg(m.lay + 2 * m.nz + n.iz);
    double s = 0.0;
    if (n.ix > 0)        s = fma(cxx, __ldcg(v + p - 1) - vp, s);
    if (n.ix < m.nx - 1) s = fma(cxx, __ldcg(v + p + 1) - vp, s);
    if (n.iy > 0)        s = fma(cyy, __ldcg(v + p - m.nx) - vp, s);
    if (n.iy < m.ny - 1) s = fma(cyy, __ldcg(v + p + m.nx) - vp, s);
    if (n.iz > 0)        s = fma(__ldg(m.lay + 3 * m.nz + n.iz - 1), __ldcg(v + p - sxy) - vp, s);
    if (n.iz < m.nz - 1) s = fma(__ldg(m.lay + 3 * m.nz + n.iz), __ldcg(v + p + sxy) - vp, s);
    const bool xm = n.ix > 0, xp = n.ix < m.nx - 1, ym = n.iy > 0, yp = n.iy < m.ny - 1;
    double c = 0.0;
    if (xp && yp) c += __ldcg(v + p + 1 + m.nx) - vp;
    if (xm && ym) c += __ldcg(v + p - 1 - m.nx) - vp;
    if (xp && ym) c -= __ldcg(v + p + 1 - m.nx) - vp;
    if (xm && yp) c -= __ldcg(v + p - 1 + m.nx) - vp;
    return fma(cd, c, s);
}

__device__ __forceinline__ float layered_A_f(const MeshDev& m, const float* v, int p, NodeIdx n, float vp)
{
    const int sxy = m.nx * m.ny;
    const float cxx = __ldg(m.layf + n.iz), cyy = __ldg(m.layf + m.nz + n.iz), cd = __ldg(m.layf + 2 * m.nz + n.iz);
    float s = 0.0f;
    if (n.ix > 0)        s = fmaf(cxx, __ldcg(v + p - 1) - vp, s);
    if (n.ix < m.nx - 1) s = fmaf(cxx, __ldcg(v + p + 1) - vp, s);
    if (n.iy > 0)        s = fmaf(cyy, __ldcg(v + p - m.nx) - vp, s);
    if (n.iy < m.ny - 1) s = fmaf(cyy, __ldcg(v + p + m.nx) - vp, s);
    if (n.iz > 0)        s = fmaf(__ldg(m.layf + 3 * m.nz + n.iz - 1), __ldcg(v + p - sxy) - vp, s);
    if (n.iz < m.nz - 1) s = fmaf(__ldg(m.layf + 3 * m.nz + n.iz), __ldcg(v + p + sxy) - vp, s);
    const bool xm = n.ix > 0, xp = n.ix < m.nx - 1, ym = n.iy > 0, yp = n.iy < m.ny - 1;
    float c = 0.0f;
    if (xp && yp) c += __ldcg(v + p + 1 + m.nx) - vp;
    if (xm && ym) c += __ldcg(v + p - 1 - m.nx) - vp;
    if (xp && ym) c -= __ldcg(v + p + 1 - m.nx) - vp;
    if (xm && yp) c -= __ldcg(v + p - 1 + m.nx) - vp;
    return fmaf(cd, c, s);
}

// Heterogeneous operator (A v)_p, face conductivity (sigma_p + sigma_q)/2.
__device__ __forceinline__ double field_A(const MeshDev& m, const double* v, int p, NodeIdx n, double vp)
{
    const int sxy = m.nx * m.ny;
    const double sp = __ldg(m.sig + p);
    double s = 0.0;
    if (n.ix > 0)        s = fma(sp + __ldg(m.sig + p - 1), __ldcg(v + p - 1) - vp, s);
    if (n.ix < m.nx - 1) s = fma(sp + __ldg(m.sig + p + 1), __ldcg(v + p + 1) - vp, s);
    if (n.iy > 0)        s = fma(sp + __ldg(m.sig + p - m.nx), __ldcg(v + p - m.nx) - vp, s);
    if (n.iy < m.ny - 1) s = fma(sp + __ldg(m.sig + p + m.nx), __ldcg(v + p + m.nx) - vp, s);
    if (n.iz > 0)        s = fma(sp + __ldg(m.sig + p - sxy), __ldcg(v + p - sxy) - vp, s);
    if (n.iz < m.nz - 1) s = fma(sp + __ldg(m.sig + p + sxy), __ldcg(v + p + sxy) - vp, s);
    return 0.5 * m.ih2 * s;
}

// Jacobi factor 1/diag(I - g A) at node p with c in-domain face neighbours.
__device__ __forceinline__ double jacobi(const MeshDev& m, const double* dinv, int p, int c, double g)
{
    if (m.lay || m.sig || m.order == 4) return esdc::esdc_rcp(fma(g, __ldg(m.wdiag + p), 1.0));
    return dinv[c];
}

__device__ __forceinline__ double apply_op(const MeshDev& m, const double* v, int p,
                                           NodeIdx n, double gih2, int* nnb)
{
    const double vp = __ldcg(v + p);
    if (m.lay) {                       // layered conductivity: gih2 carries g only
        *nnb = 0;
        return fma(-gih2, layered_A(m, v, p, n, vp), vp);
    }
    if (m.sig) {                       // conductivity field: likewise
        *nnb = 0;
        return fma(-gih2, field_A(m, v, p, n, vp), vp);
    }
    if (m.order == 4) {                // fourth-order stencil: v_p - g/(12 h^2) S4 v (L2-coherent loads)
        *nnb = 0;
        auto ax = [&](int i, int nn, int st) -> double {
            if (nn == 1) return 0.0;
            const double a4 = __ldcg(v + p + (esdc_mirror(i - 2, nn) - i) * st);
            const double b4 = __ldcg(v + p + (esdc_mirror(i - 1, nn) - i) * st);
            const double c4 = __ldcg(v + p + (esdc_mirror(i + 1, nn) - i) * st);
            const double d4 = __ldcg(v + p + (esdc_mirror(i + 2, nn) - i) * st);
            return fma(16.0, b4 + c4, -(a4 + d4)) - 30.0 * vp;
        };
        const double s4 = ax(n.ix, m.nx, 1) + ax(n.iy, m.ny, m.nx) + ax(n.iz, m.nz, m.nx * m.ny);
        return fma(-gih2 * (1.0 / 12.0), s4, vp);
    }
    const int sxy = m.nx * m.ny;
    double s = 0.0;
    int c = 0;
    if (n.ix > 0)        { s += __ldcg(v + p - 1); ++c; }
    if (n.ix < m.nx - 1) { s += __ldcg(v + p + 1); ++c; }
    if (n.iy > 0)        { s += __ldcg(v + p - m.nx); ++c; }
    if (n.iy < m.ny - 1) { s += __ldcg(v + p + m.nx); ++c; }
    if (n.iz > 0)        { s += __ldcg(v + p - sxy); ++c; }
    if (n.iz < m.nz - 1) { s += __ldcg(v + p + sxy); ++c; }
    *nnb = c;
    // v_p - g/h^2 * (sum_q v_q - c v_p)
    return fma(gih2, fma((double)c, vp, -s), vp);
}

// Jacobi-PCG with two grid barriers per iteration.  The search direction
// p = z + beta p and its image q = A p are both updated by recurrences,
// q = A z + beta q, so the stencil acts on z, which is complete at the barrier
// that also completes the reduction for beta:
//   [A] p = z + beta p; q = A z + beta q; partial p.q        | barrier -> alpha
//   [B] x += alpha p; r -= alpha q; z = D^{-1} r; r.z, r.r   | barrier -> beta, stop test
// Each thread handles ESDC_CG_UNROLL nodes per pass of its grid-stride loop and
// issues all their loads before the arithmetic, so their L2 latencies overlap.
#ifndef ESDC_CG_UNROLL
#define ESDC_CG_UNROLL 2        // best of 1/2/4/8 on GB300 (with 512-thread blocks)
#endif
// FP32 (I - g L) v for the inner solves of the precision form.
__device__ __forceinline__ float apply_op_f(const MeshDev& m, const float* v, int p, NodeIdx n, float gih2, int* nnb)
{
    const float vp = __ldcg(v + p);
    if (m.lay) {
        *nnb = 0;
        return fmaf(-gih2, layered_A_f(m, v, p, n, vp), vp);
    }
    const int sxy = m.nx * m.ny;
    float s = 0.0f;
    int c = 0;
    if (n.ix > 0)        { s += __ldcg(v + p - 1); ++c; }
    if (n.ix < m.nx - 1) { s += __ldcg(v + p + 1); ++c; }
    if (n.iy > 0)        { s += __ldcg(v + p - m.nx); ++c; }
    if (n.iy < m.ny - 1) { s += __ldcg(v + p + m.nx); ++c; }
    if (n.iz > 0)        { s += __ldcg(v + p - sxy); ++c; }
    if (n.iz < m.nz - 1) { s += __ldcg(v + p + sxy); ++c; }
    *nnb = c;
    return fmaf(gih2, fmaf((float)c, vp, -s), vp);
}

__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cg(CgArgs a)
{
    constexpr int U = ESDC_CG_UNROLL;
    const MeshDev& m = a.m;
    const int N = m.N;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* part = a.part;
    const double gih2 = (m.lay || m.sig) ? a.g : a.g * m.ih2;     // layered coefficients carry 1/h^2
    __shared__ double bs[3];
    unsigned target = 0;

    // r = b - A x, z = D^{-1} r, p = q = 0; partials r.z, r.r, b.b
    {
        double v[3] = {0.0, 0.0, 0.0};
        for (int p = tid; p < N; p += stride) {
            NodeIdx n = node_idx(m, p);
            int c;
            double ax = apply_op(m, a.x, p, n, gih2, &c);
            double bp = a.b[p];
            double rp = bp - ax;
            double zp = a.precond ? jacobi(m, a.dinv, p, c, a.g) * rp : rp;
            a.r[p] = rp;
            a.z[p] = zp;
            a.p[p] = 0.0;
            a.q[p] = 0.0;
            v[0] += rp * zp;
            v[1] += rp * rp;
            v[2] += bp * bp;
        }
        block_sum<3>(v, bs);
        if (threadIdx.x == 0) for (int k = 0; k < 3; ++k) part[k * gridDim.x + blockIdx.x] = bs[k];
    }
    if (!grid_barrier(a.bar, target, a.flags)) return;
    double tot[3];
    grid_total<3>(part, 0, tot);
    double rz = tot[0], rr = tot[1];
    const double stop = a.tol2 * tot[2];
    double beta = 0.0;
    int it = 0;
    bool done = rr <= stop;
    bool bad = !isfinite(rr) || !isfinite(stop);
    while (!done && !bad && it < a.maxit) {
        // [A] p = z + beta p, q = A z + beta q, partial p.q (slot 3)
        {
            double v[1] = {0.0};
            for (int p0 = tid; p0 < N; p0 += U * stride) {
                double az[U], zp[U], po[U], qo[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * stride;
                    if (p < N) {
                        NodeIdx n = node_idx(m, p);
                        int c;
                        az[u] = apply_op(m, a.z, p, n, gih2, &c);
                        zp[u] = __ldcg(a.z + p);
                        po[u] = a.p[p];
                        qo[u] = a.q[p];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * stride;
                    if (p < N) {
                        const double pp = fma(beta, po[u], zp[u]);
                        const double qp = fma(beta, qo[u], az[u]);
                        a.p[p] = pp;
                        a.q[p] = qp;
                        v[0] = fma(pp, qp, v[0]);
                    }
                }
            }
            block_sum<1>(v, bs);
            if (threadIdx.x == 0) part[3 * gridDim.x + blockIdx.x] = bs[0];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double pq[1], alpha;
        grid_total_q<1, 1>(part, 3, pq, rz, alpha);
        // [B] x += alpha p, r -= alpha q, z = D^{-1} r, partials r.z, r.r (slots 4, 5)
        {
            double v[2] = {0.0, 0.0};
            for (int p0 = tid; p0 < N; p0 += U * stride) {
                double qv[U], rv[U], xv[U], pv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * stride;
                    if (p < N) { qv[u] = a.q[p]; rv[u] = a.r[p]; xv[u] = a.x[p]; pv[u] = a.p[p]; }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * stride;
                    if (p < N) {
                        const double rp = fma(-alpha, qv[u], rv[u]);
                        a.x[p] = fma(alpha, pv[u], xv[u]);
                        a.r[p] = rp;
                        double zq = rp;
                        if (a.precond) {
                            NodeIdx n = node_idx(m, p);
                            int c = (n.ix > 0) + (n.ix < m.nx - 1) + (n.iy > 0) + (n.iy < m.ny - 1) +
                                    (n.iz > 0) + (n.iz < m.nz - 1);
                            zq = jacobi(m, a.dinv, p, c, a.g) * rp;
                        }
                        a.z[p] = zq;
                        v[0] = fma(rp, zq, v[0]);
                        v[1] = fma(rp, rp, v[1]);
                    }
                }
            }
            block_sum<2>(v, bs);
            if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[(4 + k) * gridDim.x + blockIdx.x] = bs[k];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double t2[2];
        grid_total_q<2, 2>(part, 4, t2, rz, beta);
        rz = t2[0];
        rr = t2[1];
        ++it;
        if (!isfinite(rr)) { bad = true; break; }
        if (rr <= stop) { done = true; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = it;
        if (a.iter_log) *a.iter_log = it;
        if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
        else if (!done) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
    }
}


// Chebyshev semi-iteration, one node per thread: the meshes the quad form does
// not take (a conductivity field, the fourth-order stencil, nx not a multiple
// of 4, unaligned vectors).  The recurrence, the bound-derived iteration count
// and the stop checks are those of the quad form (x += d, r -= B d,
// d = ca d + cb r); the interval comes from esdc_cheb_interval.  One grid
// barrier per iteration; the residual is reduced only at the checks.
__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cheb(CgArgs a, ChebArgs c)
{
    const MeshDev& m = a.m;
    const int N = m.N;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* part = a.part;
    const double gih2 = (m.lay || m.sig) ? a.g : a.g * m.ih2;     // layered / field coefficients carry 1/h^2
    __shared__ double bs[3];
    unsigned target = 0;
    double* dc = a.p;            // d_k
    double* dn = a.q;            // d_{k+1}
    const double inv_theta = c.inv_theta;

    // r = b - B x, d_0 = r / theta; partials r.r, b.b
    {
        double v[2] = {0.0, 0.0};
        for (int p = tid; p < N; p += stride) {
            int nnb;
            const double bx = apply_op(m, a.x, p, node_idx(m, p), gih2, &nnb);
            const double bp = a.b[p];
            const double rp = bp - bx;
            a.r[p] = rp;
            dc[p] = rp * inv_theta;
            v[0] = fma(rp, rp, v[0]);
            v[1] = fma(bp, bp, v[1]);
        }
        block_sum<2>(v, bs);
        if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[k * gridDim.x + blockIdx.x] = bs[k];
    }
    if (!grid_barrier(a.bar, target, a.flags)) return;
    double tot[2];
    grid_total<2>(part, 0, tot);
    const double stop = a.tol2 * tot[1];
    bool done = tot[0] <= stop;
    bool bad = !isfinite(tot[0]) || !isfinite(stop);
    // iterations the bound asks for (one thread per block evaluates it)
    __shared__ int s_kneed;
    if (threadIdx.x == 0) {
        int kn = 1;
        if (!done && !bad && c.q > 0.0) {
            const double kd = stop > 0.0 ? ceil(log(0.5 * sqrt(stop / tot[0])) / c.log_q) : (double)a.maxit;
            kn = kd < (double)a.maxit ? (int)kd : a.maxit;
        }
        s_kneed = kn < 1 ? 1 : kn;
    }
    __syncthreads();
    int it = 0;
    int chunk_end = s_kneed < a.maxit ? s_kneed : a.maxit;
    while (!done && !bad && it < a.maxit) {
        const bool check = it + 1 >= chunk_end;
        const int ki = it < ESDC_CHEB_TAB ? it : ESDC_CHEB_TAB - 1;
        const double ca = c.ca[ki], cb = c.cb[ki];
        double v[1] = {0.0};
        for (int p = tid; p < N; p += stride) {
            int nnb;
            const double bd = apply_op(m, dc, p, node_idx(m, p), gih2, &nnb);
            const double dp = __ldcg(dc + p);
            const double rn = __ldcg(a.r + p) - bd;
            a.x[p] = __ldcg(a.x + p) + dp;
            a.r[p] = rn;
            dn[p] = fma(ca, dp, cb * rn);
            if (check) v[0] = fma(rn, rn, v[0]);
        }
        double* sw = dc; dc = dn; dn = sw;
        ++it;
        if (check) {
            block_sum<1>(v, bs);
            if (threadIdx.x == 0) part[(2 + (it & 1)) * gridDim.x + blockIdx.x] = bs[0];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        if (check) {
            double rr[1];
            grid_total<1>(part, 2 + (it & 1), rr);
            if (!isfinite(rr[0])) { bad = true; break; }
            if (rr[0] <= stop) { done = true; break; }
            chunk_end = it + 2 < a.maxit ? it + 2 : a.maxit;     // rounding left it short: two more, then check
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = it;
        if (a.iter_log) *a.iter_log = it;
        if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
        else if (!done) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
    }
}

// Precision form of the solve: iterative refinement with FP64 residuals and
// FP32 inner Jacobi-PCG (the matrix-vector products of the inner solve are FP32):
//   r = b - A x (FP64); until ||r|| <= tol ||b||:
//     solve A e = r in FP32 to ||r - A e|| <= eta ||r|| (at most maxin iterations);
//     x += e (FP64); r = b - A x (FP64).
// Same barrier, reduction order and slot discipline as k_cg; partial slots:
// 0-1 initial r.r, b.b | 2-3 inner start | 4 p.q | 5-6 r.z, r.r | 7 outer r.r.
struct CgMixArgs {
    float *r, *p, *q, *z, *e;   // FP32 inner vectors [ld]
    float dinv[7];
    float eta2;
    int maxin, maxout;
};

__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cg_mixed(CgArgs a, CgMixArgs f)
{
    const MeshDev& m = a.m;
    const int N = m.N;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* part = a.part;
    const double gih2 = (m.lay || m.sig) ? a.g : a.g * m.ih2;     // layered coefficients carry 1/h^2
    const float gih2f = (float)gih2;
    __shared__ double bs[3];
    unsigned target = 0;

    // r = b - A x (FP64); partials r.r, b.b
    {
        double v[2] = {0.0, 0.0};
        for (int p = tid; p < N; p += stride) {
            NodeIdx n = node_idx(m, p);
            int c;
            const double bp = a.b[p];
            const double rp = bp - apply_op(m, a.x, p, n, gih2, &c);
            a.r[p] = rp;
            v[0] = fma(rp, rp, v[0]);
            v[1] = fma(bp, bp, v[1]);
        }
        block_sum<2>(v, bs);
        if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[k * gridDim.x + blockIdx.x] = bs[k];
    }
    if (!grid_barrier(a.bar, target, a.flags)) return;
    double t0[2];
    grid_total<2>(part, 0, t0);
    double rr = t0[0];
    const double stop = a.tol2 * t0[1];
    bool done = rr <= stop;
    bool bad = !isfinite(rr) || !isfinite(stop);
    int outer = 0, inner_total = 0;
    while (!done && !bad && outer < f.maxout) {
        // inner start: r32 = r, e = 0, z = D^{-1} r32, p = q = 0; partials r.z, r.r
        {
            double v[2] = {0.0, 0.0};
            for (int p = tid; p < N; p += stride) {
                const float rp = (float)a.r[p];
                float zp = rp;
                if (a.precond) {
                    NodeIdx n = node_idx(m, p);
                    int c = (n.ix > 0) + (n.ix < m.nx - 1) + (n.iy > 0) + (n.iy < m.ny - 1) +
                            (n.iz > 0) + (n.iz < m.nz - 1);
                    zp = (m.lay ? (float)jacobi(m, a.dinv, p, c, a.g) : f.dinv[c]) * rp;
                }
                f.r[p] = rp; f.z[p] = zp; f.p[p] = 0.0f; f.q[p] = 0.0f; f.e[p] = 0.0f;
                v[0] += (double)(rp * zp);
                v[1] += (double)(rp * rp);
            }
            block_sum<2>(v, bs);
            if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[(2 + k) * gridDim.x + blockIdx.x] = bs[k];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double ti[2];
        grid_total<2>(part, 2, ti);
        double rz = ti[0], rri = ti[1];
        const double stop_in = f.eta2 * rri;
        double beta = 0.0;
        int inner = 0;
        while (rri > stop_in && inner < f.maxin) {
            // [A] p = z + beta p, q = A z + beta q (FP32); partial p.q
            {
                constexpr int U = ESDC_CG_UNROLL;
                float acc = 0.0f;
                const float bf = (float)beta;
                for (int p0 = tid; p0 < N; p0 += U * stride) {
                    float az[U], zp[U], po[U], qo[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + u * stride;
                        if (p < N) {
                            NodeIdx n = node_idx(m, p);
                            int c;
                            az[u] = apply_op_f(m, f.z, p, n, gih2f, &c);
                            zp[u] = __ldcg(f.z + p);
                            po[u] = f.p[p];
                            qo[u] = f.q[p];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + u * stride;
                        if (p < N) {
                            const float pp = fmaf(bf, po[u], zp[u]);
                            const float qp = fmaf(bf, qo[u], az[u]);
                            f.p[p] = pp;
                            f.q[p] = qp;
                            acc = fmaf(pp, qp, acc);
                        }
                    }
                }
                double v[1] = {(double)acc};
                block_sum<1>(v, bs);
                if (threadIdx.x == 0) part[4 * gridDim.x + blockIdx.x] = bs[0];
            }
            if (!grid_barrier(a.bar, target, a.flags)) return;
            double pq[1], alpha64;
            grid_total_q<1, 1>(part, 4, pq, rz, alpha64);
            const float alpha = (float)alpha64;
            // [B] e += alpha p, r -= alpha q, z = D^{-1} r; partials r.z, r.r
            {
                constexpr int U = ESDC_CG_UNROLL;
                float acc0 = 0.0f, acc1 = 0.0f;
                for (int p0 = tid; p0 < N; p0 += U * stride) {
                    float qv[U], rv[U], ev[U], pv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + u * stride;
                        if (p < N) { qv[u] = f.q[p]; rv[u] = f.r[p]; ev[u] = f.e[p]; pv[u] = f.p[p]; }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + u * stride;
                        if (p < N) {
                            const float rp = fmaf(-alpha, qv[u], rv[u]);
                            f.e[p] = fmaf(alpha, pv[u], ev[u]);
                            f.r[p] = rp;
                            float zp = rp;
                            if (a.precond) {
                                NodeIdx n = node_idx(m, p);
                                int c = (n.ix > 0) + (n.ix < m.nx - 1) + (n.iy > 0) + (n.iy < m.ny - 1) +
                                        (n.iz > 0) + (n.iz < m.nz - 1);
                                zp = (m.lay ? 1.0f / fmaf((float)a.g, (float)__ldg(m.wdiag + p), 1.0f) : f.dinv[c]) * rp;
                            }
                            f.z[p] = zp;
                            acc0 = fmaf(rp, zp, acc0);
                            acc1 = fmaf(rp, rp, acc1);
                        }
                    }
                }
                double v[2] = {(double)acc0, (double)acc1};
                block_sum<2>(v, bs);
                if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[(5 + k) * gridDim.x + blockIdx.x] = bs[k];
            }
            if (!grid_barrier(a.bar, target, a.flags)) return;
            double t2[2];
            grid_total_q<2, 2>(part, 5, t2, rz, beta);
            rz = t2[0];
            rri = t2[1];
            ++inner;
            if (!isfinite(rri)) { bad = true; break; }
        }
        inner_total += inner;
        if (bad) break;
        // x += e (FP64)
        for (int p = tid; p < N; p += stride) a.x[p] += (double)f.e[p];
        if (!grid_barrier(a.bar, target, a.flags)) return;
        // r = b - A x (FP64); partial r.r
        {
            double v[1] = {0.0};
            for (int p = tid; p < N; p += stride) {
                NodeIdx n = node_idx(m, p);
                int c;
                const double rp = a.b[p] - apply_op(m, a.x, p, n, gih2, &c);
                a.r[p] = rp;
                v[0] = fma(rp, rp, v[0]);
            }
            block_sum<1>(v, bs);
            if (threadIdx.x == 0) part[7 * gridDim.x + blockIdx.x] = bs[0];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double t3[1];
        grid_total<1>(part, 7, t3);
        rr = t3[0];
        ++outer;
        if (!isfinite(rr)) { bad = true; break; }
        done = rr <= stop;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = inner_total;
        a.status[1] = outer;
        if (a.iter_log) *a.iter_log = inner_total;
        if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
        else if (!done) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
    }
}

}  // namespace

int esdc_cg_blocks(const MeshDev& mesh, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg, threads, 0) != cudaSuccess) return 0;
    long long want = ((long long)mesh.N + threads - 1) / threads;     // a node per thread: every SM busy sooner
    long long cap = (long long)sms * (per_sm < 1 ? per_sm : 1);   // one block per SM
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t esdc_cg_launch(const MeshDev& mesh, const CgWork& w, double g, const double* b,
                           double* x, double tol, int maxit, int precond, int solver, int* iter_log,
                           int* flags, cudaStream_t s)
{
    // the DCT-II solve: requested (2), or automatic (0) on the scalar sigma
    // where the handle holds its tables
    if (solver == 2 || (solver == 0 && w.dct && w.dct->cheap && !mesh.lay && !mesh.sig)) {
        if (!w.dct) return cudaErrorInvalidValue;
        return esdc_dct_launch(mesh, w, g, b, x, iter_log, flags, s);
    }
    if (solver == 3) solver = 0;                 // the iterative choice of the automatic mode
    if (esdc_cg4_eligible(mesh, b, x)) {
        CgArgsHost hq{mesh, w, g, b, x, tol, maxit, precond, iter_log, flags};
        if (solver == 0 && g > 0.0 && esdc_cheb_eligible(mesh, b, x)) return esdc_cheb_launch(hq, s);
        return esdc_cg4_launch(hq, false, s);
    }
    ChebArgs cheb;
    const bool use_cheb = solver == 0 && g > 0.0 && esdc_cheb_interval(mesh, g, cheb);
    CgArgs a;
    a.m = mesh;
    a.g = g;
    for (int c = 0; c < 7; ++c) a.dinv[c] = 1.0 / (1.0 + g * mesh.ih2 * c);
    a.b = b;
    a.x = x;
    a.r = w.r; a.p = w.p; a.q = w.q; a.z = w.z;
    a.part = w.part;
    a.bar = w.bar;
    a.status = w.status;
    a.iter_log = iter_log;
    a.flags = flags;
    a.tol2 = tol * tol;
    a.maxit = maxit;
    a.precond = precond;
    int nb = w.max_blocks;
    // The arrival counter starts from zero in every solve.
    cudaError_t e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (use_cheb) {
        void* args[] = {&a, &cheb};
        return cudaLaunchCooperativeKernel((const void*)k_cheb, dim3(nb), dim3(w.threads), args, 0, s);
    }
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_cg, dim3(nb), dim3(w.threads), args, 0, s);
}

cudaError_t esdc_cg_mixed_launch(const MeshDev& mesh, const CgWork& w, double g, const double* b, double* x,
                                 double tol, int maxit, int precond, int solver, int* iter_log, int* flags,
                                 cudaStream_t s)
{
    if (solver == 3) solver = 0;
    if (esdc_cg4_eligible(mesh, b, x)) {
        CgArgsHost hq{mesh, w, g, b, x, tol, maxit, precond, iter_log, flags};
        if (solver == 0 && g > 0.0 && esdc_cheb_eligible(mesh, b, x)) return esdc_cheb_mixed_launch(hq, s);
        return esdc_cg4_launch(hq, true, s);
    }
    CgArgs a;
    a.m = mesh;
    a.g = g;
    for (int c = 0; c < 7; ++c) a.dinv[c] = 1.0 / (1.0 + g * mesh.ih2 * c);
    a.b = b;
    a.x = x;
    a.r = w.r; a.p = w.p; a.q = w.q; a.z = w.z;
    a.part = w.part;
    a.bar = w.bar;
    a.status = w.status;
    a.iter_log = iter_log;
    a.flags = flags;
    a.tol2 = tol * tol;
    a.maxit = maxit;
    a.precond = precond;
    CgMixArgs f;
    f.r = w.r32; f.p = w.p32; f.q = w.q32; f.z = w.z32; f.e = w.e32;
    for (int c = 0; c < 7; ++c) f.dinv[c] = (float)a.dinv[c];
    f.eta2 = 1e-10f;            // inner solves reduce the residual by 1e-5
    f.maxin = maxit < 60 ? maxit : 60;
    f.maxout = 8;
    int nb = w.max_blocks;
    void* args[] = {&a, &f};
    cudaError_t e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)k_cg_mixed, dim3(nb), dim3(w.threads), args, 0, s);
}
