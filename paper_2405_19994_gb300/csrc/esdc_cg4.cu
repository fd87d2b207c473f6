// Quad form of the persistent solves of the implicit diffusion rows
// (eq. def_P: (I - g A) V_i = rhs at every collocation node): the Jacobi-PCG
// (k_cg4), the Chebyshev semi-iteration (k_cheb4, the default), and the
// precision form's refinement with CG or Chebyshev inner solves (k_cg4_mixed,
// k_cheb4_mixed).
//
// Each thread owns runs of four x-consecutive nodes ("quads"), so every vector
// access is a 16-byte (FP32) or 2 x 16-byte (FP64) load or store and a thread
// keeps ten or more independent loads in flight.  The diagonal of I - g A and
// its inverse (the Jacobi preconditioner) depend only on the layer and on
// which faces of the node lie on the boundary, so both come from small tables
// in shared memory, built by every block at the start of the solve; for the
// layered operator the coefficients are scaled by g once, in the same tables.
// Per node and iteration the plain FP64 solve then costs 15 (scalar sigma) or
// 19 (layered) FP64 operations, the minimum for the two recurrences, the
// stencil and three dot products: the FP64 pipe, not HBM, bounds it on GB300.
//
// The precision form (iterative refinement) keeps the outer residual
// b - A x in FP64 and runs the inner Jacobi-PCG in FP32.  Its residual pass
// also starts the next inner solve (FP32 residual, preconditioned residual and
// their dot products), and the first inner iteration needs no zeroed vectors,
// so an outer step costs two FP64 passes over the mesh.
//
// Requirements (checked by esdc_cg4_eligible): nx a multiple of 4, b and x
// 16-byte aligned, and for the layered operator nz <= ESDC_CG4_MAX_LAYERS.
#include <cmath>

#include "esdc_internal.h"
#include "esdc_cg_common.cuh"

namespace {

template <typename T> struct Q4 { T v[4]; };

__device__ __forceinline__ Q4<double> ld4(const double* a)
{
    const double2 u = __ldcg(reinterpret_cast<const double2*>(a));
    const double2 w = __ldcg(reinterpret_cast<const double2*>(a) + 1);
    return {{u.x, u.y, w.x, w.y}};
}

__device__ __forceinline__ Q4<float> ld4(const float* a)
{
    const float4 u = __ldcg(reinterpret_cast<const float4*>(a));
    return {{u.x, u.y, u.z, u.w}};
}

__device__ __forceinline__ void st4(double* a, const Q4<double>& q)
{
    __stcg(reinterpret_cast<double2*>(a), make_double2(q.v[0], q.v[1]));
    __stcg(reinterpret_cast<double2*>(a) + 1, make_double2(q.v[2], q.v[3]));
}

__device__ __forceinline__ void st4(float* a, const Q4<float>& q)
{
    __stcg(reinterpret_cast<float4*>(a), make_float4(q.v[0], q.v[1], q.v[2], q.v[3]));
}

// Geometry of the quad starting at node p = 4 qi.
struct Geo {
    int p, iz;
    bool xl, xr, yn, ys, zb, zt;     // neighbour planes present: x0-1, x0+4, y-1, y+1, z-1, z+1
};

__device__ __forceinline__ Geo geo(const MeshDev& m, int qi)
{
    Geo G;
    G.p = 4 * qi;
    const int r = G.p / m.nx;
    const int x0 = G.p - r * m.nx;
    G.iz = r / m.ny;
    const int iy = r - G.iz * m.ny;
    G.xl = x0 > 0;
    G.xr = x0 + 4 < m.nx;
    G.yn = iy > 0;
    G.ys = iy < m.ny - 1;
    G.zb = G.iz > 0;
    G.zt = G.iz < m.nz - 1;
    return G;
}

// Tables in shared memory.  Scalar sigma: D[c] = 1 + c g/h^2 and I[c] = 1/D[c]
// for c in-domain neighbours (c = 0..6).  Layered: per layer k the
// g-scaled coefficients cx, cy, cd (in-plane diagonals) and cz (face k|k+1),
// and per (k, x class, y class) D = 1 + g w and I = 1/D, where w = -diag(A)
// and the class of an axis is 0 inside, 1 on the low face, 2 on the high face,
// 3 on both (a single cell across).
template <typename T>
struct Tab {
    T *D, *I, *cx, *cy, *cd, *cz;
    T g;             // g/h^2 (scalar sigma); unused when layered
};

__host__ __device__ inline int tab_entries(const MeshDev& m)
{
    return m.lay ? 36 * m.nz : 16;
}

template <typename T>
__device__ Tab<T> carve(T* base, const MeshDev& m)
{
    Tab<T> t;
    if (!m.lay) {
        t.D = base; t.I = base + 8;
        t.cx = t.cy = t.cd = t.cz = nullptr;
    } else {
        const int nz = m.nz;
        t.cx = base; t.cy = base + nz; t.cd = base + 2 * nz; t.cz = base + 3 * nz;
        t.D = base + 4 * nz; t.I = base + 20 * nz;
    }
    return t;
}

// Representative index along an axis of n cells for class cls, or -1 if the
// class does not occur.
__device__ __forceinline__ int rep_index(int cls, int n)
{
    switch (cls) {
        case 0: return n >= 3 ? 1 : -1;
        case 1: return n >= 2 ? 0 : -1;
        case 2: return n >= 2 ? n - 1 : -1;
        default: return n == 1 ? 0 : -1;
    }
}

// Fills the tables (all threads of the block take part; ends with a block barrier).
template <typename T>
__device__ void build_tab(const MeshDev& m, double g, bool precond, Tab<T>& t)
{
    if (!m.lay) {
        const double gih2 = g * m.ih2;
        t.g = (T)gih2;
        if (threadIdx.x < 8) {
            const double d = 1.0 + gih2 * (double)threadIdx.x;
            t.D[threadIdx.x] = (T)d;
            t.I[threadIdx.x] = precond ? (T)(1.0 / d) : (T)1;
        }
    } else {
        t.g = (T)g;
        const int nz = m.nz;
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            t.cx[k] = (T)(g * m.lay[k]);
            t.cy[k] = (T)(g * m.lay[nz + k]);
            t.cd[k] = (T)(g * m.lay[2 * nz + k]);
            t.cz[k] = k < nz - 1 ? (T)(g * m.lay[3 * nz + k]) : (T)0;
        }
        for (int e = threadIdx.x; e < 16 * nz; e += blockDim.x) {
            const int k = e >> 4, xc = (e >> 2) & 3, yc = e & 3;
            const int ix = rep_index(xc, m.nx), iy = rep_index(yc, m.ny);
            double d = 1.0;
            if (ix >= 0 && iy >= 0) d = 1.0 + g * m.wdiag[((size_t)k * m.ny + iy) * m.nx + ix];
            t.D[e] = (T)d;
            t.I[e] = precond ? (T)(1.0 / d) : (T)1;
        }
    }
    __syncthreads();
}

// Table rows of the three diagonal classes of a quad: node 0 (may sit on the
// low x face), nodes 1-2 (inside), node 3 (may sit on the high x face).
struct DiagIdx { int l, m, r; };

template <bool LAY>
__device__ __forceinline__ DiagIdx diag_idx(const Geo& G)
{
    DiagIdx d;
    if (!LAY) {
        const int cyz = G.yn + G.ys + G.zb + G.zt;
        d.l = cyz + 1 + G.xl;
        d.m = cyz + 2;
        d.r = cyz + 1 + G.xr;
    } else {
        const int row = G.iz * 16 + (G.yn ? 0 : 1) + (G.ys ? 0 : 2);
        d.m = row;
        d.l = row + (G.xl ? 0 : 4);
        d.r = row + (G.xr ? 0 : 8);
    }
    return d;
}

// out = (I - g A) v on the quad; c = v on the quad.
template <typename T, bool LAY>
__device__ __forceinline__ void apply4(const MeshDev& m, const Tab<T>& t, const T* v, const Geo& G,
                                       const DiagIdx& di, Q4<T>& c, Q4<T>& out)
{
    const int nx = m.nx, sxy = m.nx * m.ny, p = G.p;
    c = ld4(v + p);
    const T vl = G.xl ? __ldcg(v + p - 1) : T(0);
    const T vr = G.xr ? __ldcg(v + p + 4) : T(0);
    Q4<T> vn = {{T(0), T(0), T(0), T(0)}}, vs = vn, vb = vn, vt = vn;
    if (G.yn) vn = ld4(v + p - nx);
    if (G.ys) vs = ld4(v + p + nx);
    if (G.zb) vb = ld4(v + p - sxy);
    if (G.zt) vt = ld4(v + p + sxy);
    const T dl = t.D[di.l], dm = t.D[di.m], dr = t.D[di.r];
    if (!LAY) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T xm = j > 0 ? c.v[j - 1] : vl;
            const T xp = j < 3 ? c.v[j + 1] : vr;
            const T s = ((xm + xp) + (vn.v[j] + vs.v[j])) + (vb.v[j] + vt.v[j]);
            const T d = j == 0 ? dl : (j == 3 ? dr : dm);
            out.v[j] = fma(d, c.v[j], -(t.g * s));
        }
    } else {
        // in-plane diagonal neighbours outside the quad's x range
        const T nl = (G.xl && G.yn) ? __ldcg(v + p - nx - 1) : T(0);   // (x0-1, y-1)
        const T nr = (G.xr && G.yn) ? __ldcg(v + p - nx + 4) : T(0);   // (x0+4, y-1)
        const T sl = (G.xl && G.ys) ? __ldcg(v + p + nx - 1) : T(0);   // (x0-1, y+1)
        const T sr = (G.xr && G.ys) ? __ldcg(v + p + nx + 4) : T(0);   // (x0+4, y+1)
        const T cx = t.cx[G.iz], cy = t.cy[G.iz], cd = t.cd[G.iz];
        const T czb = G.zb ? t.cz[G.iz - 1] : T(0), czt = t.cz[G.iz];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T xm = j > 0 ? c.v[j - 1] : vl;
            const T xp = j < 3 ? c.v[j + 1] : vr;
            const T pp = j < 3 ? vs.v[j + 1] : sr;     // (x+1, y+1)
            const T mm = j > 0 ? vn.v[j - 1] : nl;     // (x-1, y-1)
            const T pm = j < 3 ? vn.v[j + 1] : nr;     // (x+1, y-1)
            const T mp = j > 0 ? vs.v[j - 1] : sl;     // (x-1, y+1)
            T s = cx * (xm + xp);
            s = fma(cy, vn.v[j] + vs.v[j], s);
            s = fma(czb, vb.v[j], s);
            s = fma(czt, vt.v[j], s);
            s = fma(cd, (pp + mm) - (pm + mp), s);
            const T d = j == 0 ? dl : (j == 3 ? dr : dm);
            out.v[j] = fma(d, c.v[j], -s);
        }
    }
}

template <typename T>
__device__ __forceinline__ T pick(const Tab<T>& t, const DiagIdx& di, int j)
{
    return j == 0 ? t.I[di.l] : (j == 3 ? t.I[di.r] : t.I[di.m]);
}

// ---------------------------------------------------------------- FP64 Jacobi-PCG
// Same iteration, barriers, reduction order and slot discipline as the scalar
// kernel: [A] p = z + beta p, q = A z + beta q, p.q | [B] x += alpha p,
// r -= alpha q, z = D^{-1} r, r.z, r.r.  The first [A] takes p = z, q = A z.
template <bool LAY>
__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cg4(CgArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const MeshDev& m = a.m;
    Tab<double> t = carve<double>(reinterpret_cast<double*>(dsm), m);
    build_tab(m, a.g, a.precond != 0, t);
    const int nq = m.N >> 2;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* part = a.part;
    __shared__ double bs[3];
    unsigned target = 0;

    // r = b - A x, z = D^{-1} r; partials r.z, r.r, b.b
    {
        double v[3] = {0.0, 0.0, 0.0};
        for (int qi = tid; qi < nq; qi += stride) {
            const Geo G = geo(m, qi);
            const DiagIdx di = diag_idx<LAY>(G);
            Q4<double> xc, ax;
            apply4<double, LAY>(m, t, a.x, G, di, xc, ax);
            const Q4<double> b = ld4(a.b + G.p);
            Q4<double> r, z;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                r.v[j] = b.v[j] - ax.v[j];
                z.v[j] = pick(t, di, j) * r.v[j];
                v[0] = fma(r.v[j], z.v[j], v[0]);
                v[1] = fma(r.v[j], r.v[j], v[1]);
                v[2] = fma(b.v[j], b.v[j], v[2]);
            }
            st4(a.r + G.p, r);
            st4(a.z + G.p, z);
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
        const bool first = it == 0;
        {
            double v[1] = {0.0};
            for (int qi = tid; qi < nq; qi += stride) {
                const Geo G = geo(m, qi);
                const DiagIdx di = diag_idx<LAY>(G);
                Q4<double> zc, az;
                apply4<double, LAY>(m, t, a.z, G, di, zc, az);
                Q4<double> pn = zc, qn = az;
                if (!first) {
                    const Q4<double> po = ld4(a.p + G.p), qo = ld4(a.q + G.p);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        pn.v[j] = fma(beta, po.v[j], zc.v[j]);
                        qn.v[j] = fma(beta, qo.v[j], az.v[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) v[0] = fma(pn.v[j], qn.v[j], v[0]);
                st4(a.p + G.p, pn);
                st4(a.q + G.p, qn);
            }
            block_sum<1>(v, bs);
            if (threadIdx.x == 0) part[3 * gridDim.x + blockIdx.x] = bs[0];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double pq[1], alpha;
        grid_total_q<1, 1>(part, 3, pq, rz, alpha);
        {
            double v[2] = {0.0, 0.0};
            for (int qi = tid; qi < nq; qi += stride) {
                const Geo G = geo(m, qi);
                const DiagIdx di = diag_idx<LAY>(G);
                const Q4<double> qv = ld4(a.q + G.p), rv = ld4(a.r + G.p), xv = ld4(a.x + G.p),
                                 pv = ld4(a.p + G.p);
                Q4<double> rn, xn, zn;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    rn.v[j] = fma(-alpha, qv.v[j], rv.v[j]);
                    xn.v[j] = fma(alpha, pv.v[j], xv.v[j]);
                    zn.v[j] = pick(t, di, j) * rn.v[j];
                    v[0] = fma(rn.v[j], zn.v[j], v[0]);
                    v[1] = fma(rn.v[j], rn.v[j], v[1]);
                }
                st4(a.r + G.p, rn);
                st4(a.x + G.p, xn);
                st4(a.z + G.p, zn);
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

// ---------------------------------------------------------------- Chebyshev semi-iteration
// For the scalar-sigma second-order stencil the spectrum of B = I - g L is
// known exactly: the cosine modes are its eigenvectors, so it lies in
// [lmin, lmax] = [1, 1 + (g/h^2) sum_axes 4 sin^2(pi (n-1)/(2n))].  For the
// layered operator lmin = 1 still holds (constants are the null space of A)
// and lmax = 1 + g lam_bound with the host's Gershgorin bound.  The
// Chebyshev semi-iteration on that interval needs no dot products:
//   x_{k+1} = x_k + d_k,  r_{k+1} = r_k - B d_k,
//   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) r_{k+1},
//   rho_0 = delta/theta, rho_{k+1} = 1/(2 theta/delta - rho_k),
// theta, delta the centre and half-width of the interval (the coefficients are
// precomputed on the host).  ||r_k|| <= 2 q^k ||r_0|| with
// q = (sqrt(kappa) - 1)/(sqrt(kappa) + 1), kappa = lmax/lmin, so the number of
// iterations to ||r|| <= tol ||b|| follows from ||r_0||; the residual is then
// checked, and a short extension runs if rounding left it above the tolerance.
// One grid barrier per iteration (CG needs two and three dot products), and
// 11 FP64 operations per node: the stencil, r, x and d.
#define ESDC_CHEB_THREADS 1024   // one block per SM; the quads of a mesh are too few to fill more warps

// 1024 threads for the scalar stencil (64 registers suffice); the layered
// stencil's extra neighbours and coefficients need more registers: 512.
template <bool LAY> constexpr int cheb_threads() { return LAY ? 512 : ESDC_CHEB_THREADS; }

template <bool LAY>
__global__ void __launch_bounds__(cheb_threads<LAY>(), 1) k_cheb4(CgArgs a, ChebArgs c)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const MeshDev& m = a.m;
    Tab<double> t = carve<double>(reinterpret_cast<double*>(dsm), m);
    build_tab(m, a.g, false, t);
    const int nq = m.N >> 2;
    // a contiguous, balanced range of quads per block (one block per SM)
    const int q0 = (int)((long long)blockIdx.x * nq / gridDim.x);
    const int q1 = (int)((long long)(blockIdx.x + 1) * nq / gridDim.x);
    double* part = a.part;
    __shared__ double bs[3];
    unsigned target = 0;
    double* dc = a.p;            // d_k
    double* dn = a.q;            // d_{k+1}
    const double inv_theta = c.inv_theta;

    // r = b - B x, d_0 = r / theta; partials r.r, b.b
    {
        double v[2] = {0.0, 0.0};
        for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
            const Geo G = geo(m, qi);
            const DiagIdx di = diag_idx<LAY>(G);
            Q4<double> xc, bx;
            apply4<double, LAY>(m, t, a.x, G, di, xc, bx);
            const Q4<double> b = ld4(a.b + G.p);
            Q4<double> r, d;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                r.v[j] = b.v[j] - bx.v[j];
                d.v[j] = r.v[j] * inv_theta;
                v[0] = fma(r.v[j], r.v[j], v[0]);
                v[1] = fma(b.v[j], b.v[j], v[1]);
            }
            st4(a.r + G.p, r);
            st4(dc + G.p, d);
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
    // iterations the bound asks for: 2 q^k ||r_0|| <= tol ||b||.  One thread per block
    // evaluates it (a few dozen FP64 operations) and shares it; every block gets the same value.
    __shared__ int s_kneed;
    if (threadIdx.x == 0) {
        int kn = 1;
        if (!done && !bad && c.q > 0.0) {
            const double kd = stop > 0.0 ? ceil(log(0.5 * sqrt(stop / tot[0])) / c.log_q) : (double)a.maxit;
            kn = kd < (double)a.maxit ? (int)kd : a.maxit;     // tol 0: run to the cap
        }
        s_kneed = kn < 1 ? 1 : kn;
    }
    __syncthreads();
    const int k_need = s_kneed;
    int it = 0;
    int chunk_end = k_need < a.maxit ? k_need : a.maxit;
    while (!done && !bad && it < a.maxit) {
        const bool check = it + 1 >= chunk_end;
        const int ki = it < ESDC_CHEB_TAB ? it : ESDC_CHEB_TAB - 1;
        const double ca = c.ca[ki], cb = c.cb[ki];
        double v[1] = {0.0};
        for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
            const Geo G = geo(m, qi);
            const DiagIdx di = diag_idx<LAY>(G);
            Q4<double> d, bd;
            apply4<double, LAY>(m, t, dc, G, di, d, bd);
            const Q4<double> r = ld4(a.r + G.p), x = ld4(a.x + G.p);
            Q4<double> rn, xn, dnew;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                rn.v[j] = r.v[j] - bd.v[j];
                xn.v[j] = x.v[j] + d.v[j];
                dnew.v[j] = fma(ca, d.v[j], cb * rn.v[j]);
                if (check) v[0] = fma(rn.v[j], rn.v[j], v[0]);
            }
            st4(a.r + G.p, rn);
            st4(a.x + G.p, xn);
            st4(dn + G.p, dnew);
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

// ---------------------------------------------------------------- iterative refinement
struct Cg4MixArgs {
    float *r, *p, *q, *z, *e;   // FP32 inner vectors
    double eta2;                // inner stop: r.r <= eta2 (r.r at the inner start)
    int maxin, maxout;
};

template <bool LAY>
__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cg4_mixed(CgArgs a, Cg4MixArgs f)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const MeshDev& m = a.m;
    const int ne = tab_entries(m);
    Tab<double> t = carve<double>(reinterpret_cast<double*>(dsm), m);
    Tab<float> tf = carve<float>(reinterpret_cast<float*>(dsm + sizeof(double) * ne), m);
    build_tab(m, a.g, a.precond != 0, t);
    build_tab(m, a.g, a.precond != 0, tf);
    const int nq = m.N >> 2;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* part = a.part;
    __shared__ double bs[3];
    unsigned target = 0;

    // b.b (slot 7), once
    {
        double v[1] = {0.0};
        for (int qi = tid; qi < nq; qi += stride) {
            const Q4<double> b = ld4(a.b + 4 * qi);
#pragma unroll
            for (int j = 0; j < 4; ++j) v[0] = fma(b.v[j], b.v[j], v[0]);
        }
        block_sum<1>(v, bs);
        if (threadIdx.x == 0) part[7 * gridDim.x + blockIdx.x] = bs[0];
    }
    double stop = 0.0;
    bool first_outer = true, done = false, bad = false;
    int outer = 0, inner_total = 0;
    for (;;) {
        // [R] r = b - A x (FP64), r.r; start of the inner solve: r32 = r,
        // z32 = D^{-1} r32, r32.z32, r32.r32 (slots 0-2)
        {
            double v[3] = {0.0, 0.0, 0.0};
            float rz32 = 0.0f, rr32 = 0.0f;
            for (int qi = tid; qi < nq; qi += stride) {
                const Geo G = geo(m, qi);
                const DiagIdx di = diag_idx<LAY>(G);
                Q4<double> xc, ax;
                apply4<double, LAY>(m, t, a.x, G, di, xc, ax);
                const Q4<double> b = ld4(a.b + G.p);
                Q4<float> r32, z32;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double r = b.v[j] - ax.v[j];
                    v[0] = fma(r, r, v[0]);
                    r32.v[j] = (float)r;
                    z32.v[j] = pick(tf, di, j) * r32.v[j];
                    rz32 = fmaf(r32.v[j], z32.v[j], rz32);
                    rr32 = fmaf(r32.v[j], r32.v[j], rr32);
                }
                st4(f.r + G.p, r32);
                st4(f.z + G.p, z32);
            }
            v[1] = rz32;
            v[2] = rr32;
            block_sum<3>(v, bs);
            if (threadIdx.x == 0) for (int k = 0; k < 3; ++k) part[k * gridDim.x + blockIdx.x] = bs[k];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double tr[3];
        grid_total<3>(part, 0, tr);
        if (first_outer) {
            double bb[1];
            grid_total<1>(part, 7, bb);
            stop = a.tol2 * bb[0];
            first_outer = false;
            if (!isfinite(stop)) { bad = true; break; }
        }
        if (!isfinite(tr[0])) { bad = true; break; }
        if (tr[0] <= stop) { done = true; break; }
        if (outer >= f.maxout) break;
        double rz = tr[1], rri = tr[2];
        if (!(rri > 0.0)) break;               // residual below FP32 range: cannot refine further
        const double stop_in = f.eta2 * rri;
        double beta = 0.0;
        int inner = 0;
        while (rri > stop_in && inner < f.maxin) {
            const bool first = inner == 0;
            // [A] p = z + beta p, q = A z + beta q (FP32); p.q (slot 3)
            {
                float acc = 0.0f;
                const float bf = (float)beta;
                for (int qi = tid; qi < nq; qi += stride) {
                    const Geo G = geo(m, qi);
                    const DiagIdx di = diag_idx<LAY>(G);
                    Q4<float> zc, az;
                    apply4<float, LAY>(m, tf, f.z, G, di, zc, az);
                    Q4<float> pn = zc, qn = az;
                    if (!first) {
                        const Q4<float> po = ld4(f.p + G.p), qo = ld4(f.q + G.p);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            pn.v[j] = fmaf(bf, po.v[j], zc.v[j]);
                            qn.v[j] = fmaf(bf, qo.v[j], az.v[j]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc = fmaf(pn.v[j], qn.v[j], acc);
                    st4(f.p + G.p, pn);
                    st4(f.q + G.p, qn);
                }
                double v[1] = {(double)acc};
                block_sum<1>(v, bs);
                if (threadIdx.x == 0) part[3 * gridDim.x + blockIdx.x] = bs[0];
            }
            if (!grid_barrier(a.bar, target, a.flags)) return;
            double pq[1], alpha64;
            grid_total_q<1, 1>(part, 3, pq, rz, alpha64);
            const float alpha = (float)alpha64;
            // [B] e += alpha p (e = alpha p at first), r -= alpha q, z = D^{-1} r; r.z, r.r (slots 4-5)
            {
                float acc0 = 0.0f, acc1 = 0.0f;
                for (int qi = tid; qi < nq; qi += stride) {
                    const Geo G = geo(m, qi);
                    const DiagIdx di = diag_idx<LAY>(G);
                    const Q4<float> qv = ld4(f.q + G.p), rv = ld4(f.r + G.p), pv = ld4(f.p + G.p);
                    Q4<float> ev = {{0.0f, 0.0f, 0.0f, 0.0f}};
                    if (!first) ev = ld4(f.e + G.p);
                    Q4<float> rn, en, zn;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        rn.v[j] = fmaf(-alpha, qv.v[j], rv.v[j]);
                        en.v[j] = fmaf(alpha, pv.v[j], ev.v[j]);
                        zn.v[j] = pick(tf, di, j) * rn.v[j];
                        acc0 = fmaf(rn.v[j], zn.v[j], acc0);
                        acc1 = fmaf(rn.v[j], rn.v[j], acc1);
                    }
                    st4(f.r + G.p, rn);
                    st4(f.e + G.p, en);
                    st4(f.z + G.p, zn);
                }
                double v[2] = {(double)acc0, (double)acc1};
                block_sum<2>(v, bs);
                if (threadIdx.x == 0) for (int k = 0; k < 2; ++k) part[(4 + k) * gridDim.x + blockIdx.x] = bs[k];
            }
            if (!grid_barrier(a.bar, target, a.flags)) return;
            double t2[2];
            grid_total_q<2, 2>(part, 4, t2, rz, beta);
            rz = t2[0];
            rri = t2[1];
            ++inner;
            if (!isfinite(rri)) { bad = true; break; }
        }
        inner_total += inner;
        if (bad || inner == 0) break;
        // [X] x += e (FP64)
        for (int qi = tid; qi < nq; qi += stride) {
            const int p = 4 * qi;
            const Q4<float> e = ld4(f.e + p);
            Q4<double> x = ld4(a.x + p);
#pragma unroll
            for (int j = 0; j < 4; ++j) x.v[j] += (double)e.v[j];
            st4(a.x + p, x);
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        ++outer;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = inner_total;
        a.status[1] = outer;
        if (a.iter_log) *a.iter_log = inner_total;
        if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
        else if (!done) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
    }
}

// ---------------------------------------------------------------- refinement, Chebyshev inner solves
// The precision form's refinement (FP64 residual r = b - A x, FP32 inner solve
// of A e = r from e = 0, x += e in FP64) with each inner solve done by kin
// Chebyshev iterations on the operator's interval.  kin comes from the bound
// 2 q^kin <= 1e-5, the same reduction the CG's inner stop asks for, so the
// inner iterations need no reductions: one grid barrier each.  The outer stop
// is the FP64 test ||b - A x|| <= tol ||b|| of every other solve.
template <bool LAY>
__global__ void __launch_bounds__(ESDC_CG_THREADS) k_cheb4_mixed(CgArgs a, Cg4MixArgs f, ChebArgs c, int kin)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const MeshDev& m = a.m;
    const int ne = tab_entries(m);
    Tab<double> t = carve<double>(reinterpret_cast<double*>(dsm), m);
    Tab<float> tf = carve<float>(reinterpret_cast<float*>(dsm + sizeof(double) * ne), m);
    build_tab(m, a.g, false, t);
    build_tab(m, a.g, false, tf);
    const int nq = m.N >> 2;
    const int q0 = (int)((long long)blockIdx.x * nq / gridDim.x);
    const int q1 = (int)((long long)(blockIdx.x + 1) * nq / gridDim.x);
    double* part = a.part;
    __shared__ double bs[3];
    unsigned target = 0;
    const float inv_theta = (float)c.inv_theta;

    // b.b (slot 7), once
    {
        double v[1] = {0.0};
        for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
            const Q4<double> b = ld4(a.b + 4 * qi);
#pragma unroll
            for (int j = 0; j < 4; ++j) v[0] = fma(b.v[j], b.v[j], v[0]);
        }
        block_sum<1>(v, bs);
        if (threadIdx.x == 0) part[7 * gridDim.x + blockIdx.x] = bs[0];
    }
    double stop = 0.0;
    bool first_outer = true, done = false, bad = false;
    int outer = 0, inner_total = 0;
    for (;;) {
        // [R] r = b - A x (FP64), r.r (slot 0); the inner start r32 = r, d32 = r32/theta
        {
            double v[1] = {0.0};
            for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
                const Geo G = geo(m, qi);
                const DiagIdx di = diag_idx<LAY>(G);
                Q4<double> xc, ax;
                apply4<double, LAY>(m, t, a.x, G, di, xc, ax);
                const Q4<double> b = ld4(a.b + G.p);
                Q4<float> r32, d32;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double r = b.v[j] - ax.v[j];
                    v[0] = fma(r, r, v[0]);
                    r32.v[j] = (float)r;
                    d32.v[j] = r32.v[j] * inv_theta;
                }
                st4(f.r + G.p, r32);
                st4(f.p + G.p, d32);
            }
            block_sum<1>(v, bs);
            if (threadIdx.x == 0) part[blockIdx.x] = bs[0];
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        double tr[1];
        grid_total<1>(part, 0, tr);
        if (first_outer) {
            double bb[1];
            grid_total<1>(part, 7, bb);
            stop = a.tol2 * bb[0];
            first_outer = false;
            if (!isfinite(stop)) { bad = true; break; }
        }
        if (!isfinite(tr[0])) { bad = true; break; }
        if (tr[0] <= stop) { done = true; break; }
        if (outer >= f.maxout) break;
        // inner: kin iterations e += d, r -= B d, d = ca d + cb r (FP32), from e = 0
        float* dc = f.p;
        float* dn = f.q;
        for (int it = 0; it < kin; ++it) {
            const int ki = it < ESDC_CHEB_TAB ? it : ESDC_CHEB_TAB - 1;
            const float ca = (float)c.ca[ki], cb = (float)c.cb[ki];
            const bool last = it + 1 == kin;
            for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
                const Geo G = geo(m, qi);
                const DiagIdx di = diag_idx<LAY>(G);
                Q4<float> d, bd;
                apply4<float, LAY>(m, tf, dc, G, di, d, bd);
                Q4<float> ev = {{0.0f, 0.0f, 0.0f, 0.0f}};
                if (it > 0) ev = ld4(f.e + G.p);
                const Q4<float> rv = ld4(f.r + G.p);
                Q4<float> en, rn, dnew;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    en.v[j] = ev.v[j] + d.v[j];
                    rn.v[j] = rv.v[j] - bd.v[j];
                    dnew.v[j] = fmaf(ca, d.v[j], cb * rn.v[j]);
                }
                st4(f.e + G.p, en);
                if (!last) {
                    st4(f.r + G.p, rn);
                    st4(dn + G.p, dnew);
                }
            }
            float* sw = dc; dc = dn; dn = sw;
            if (!grid_barrier(a.bar, target, a.flags)) return;
        }
        inner_total += kin;
        // [X] x += e (FP64)
        for (int qi = q0 + (int)threadIdx.x; qi < q1; qi += blockDim.x) {
            const int p = 4 * qi;
            const Q4<float> e = ld4(f.e + p);
            Q4<double> x = ld4(a.x + p);
#pragma unroll
            for (int j = 0; j < 4; ++j) x.v[j] += (double)e.v[j];
            st4(a.x + p, x);
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        ++outer;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = inner_total;
        a.status[1] = outer;
        if (a.iter_log) *a.iter_log = inner_total;
        if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
        else if (!done) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
    }
}

// Dynamic shared memory of a launch, and the one-time opt-in above 48 KB.
template <typename K>
cudaError_t prepare(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int quad_blocks(const MeshDev& m, const CgWork& w)
{
    const long long nq = m.N / 4;
    long long want = (nq + w.threads - 1) / w.threads;
    if (want < 1) want = 1;
    return (int)(want < w.max_blocks ? want : w.max_blocks);
}

}  // namespace

bool esdc_cg4_eligible(const MeshDev& m, const void* b, const void* x)
{
    if (m.nx % 4 != 0 || m.N < 4 || m.sig || m.order != 2) return false;   // field and fourth order: scalar path
    if ((reinterpret_cast<uintptr_t>(b) & 15u) || (reinterpret_cast<uintptr_t>(x) & 15u)) return false;
    if (m.lay && (m.nz > ESDC_CG4_MAX_LAYERS || !m.wdiag)) return false;
    return true;
}

bool esdc_cheb_interval(const MeshDev& m, double g, ChebArgs& c)
{
    double w = 0.0;
    const int n[3] = {m.nx, m.ny, m.nz};
    if (m.lay || m.sig) {
        w = m.lam_bound;
    } else if (m.order == 4) {
        for (int k = 0; k < 3; ++k)
            if (n[k] > 1) {
                const double t = M_PI * (n[k] - 1) / n[k];
                w += 30.0 + 2.0 * std::cos(2.0 * t) - 32.0 * std::cos(t);
            }
        w *= m.ih2 / 12.0;
    } else {
        for (int k = 0; k < 3; ++k)
            if (n[k] > 1) {
                const double sn = std::sin(M_PI * (n[k] - 1) / (2.0 * n[k]));
                w += 4.0 * sn * sn;
            }
        w *= m.ih2;
    }
    const double lmin = 1.0, lmax = 1.0 + g * w;
    if (!(lmax > lmin) || !std::isfinite(lmax)) return false;
    const double theta = 0.5 * (lmax + lmin);
    c.inv_theta = 1.0 / theta;
    const double delta = 0.5 * (lmax - lmin), s1 = theta / delta;
    const double kap = lmax / lmin;
    c.q = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    c.log_q = c.q > 0.0 ? std::log(c.q) : -1.0;
    double rho = 1.0 / s1;
    for (int k = 0; k < ESDC_CHEB_TAB; ++k) {
        const double rn = 1.0 / (2.0 * s1 - rho);
        c.ca[k] = rn * rho;
        c.cb[k] = 2.0 * rn / delta;
        rho = rn;
    }
    return true;
}

bool esdc_cheb_eligible(const MeshDev& m, const void* b, const void* x)
{
    if (m.sig || m.order != 2 || !esdc_cg4_eligible(m, b, x)) return false;
    if (m.lay) return m.lam_bound > 0.0;                       // the Gershgorin interval
    return m.nx > 1 || m.ny > 1 || m.nz > 1;                   // an interval of positive width
}

cudaError_t esdc_cheb_launch(const CgArgsHost& h, cudaStream_t s)
{
    CgArgs a;
    a.m = h.mesh;
    a.g = h.g;
    for (int c = 0; c < 7; ++c) a.dinv[c] = 0.0;
    a.b = h.b;
    a.x = h.x;
    a.r = h.w.r; a.p = h.w.p; a.q = h.w.q; a.z = h.w.z;
    a.part = h.w.part;
    a.bar = h.w.bar;
    a.status = h.w.status;
    a.iter_log = h.iter_log;
    a.flags = h.flags;
    a.tol2 = h.tol * h.tol;
    a.maxit = h.maxit;
    a.precond = 0;
    ChebArgs c;
    if (!esdc_cheb_interval(h.mesh, h.g, c)) return esdc_cg4_launch(h, false, s);    // no interval
    const int ne = tab_entries(h.mesh);
    const size_t bytes = sizeof(double) * ne;
    const bool lay = h.mesh.lay != nullptr;
    cudaError_t e = lay ? prepare(k_cheb4<true>, bytes) : prepare(k_cheb4<false>, bytes);
    if (e != cudaSuccess) return e;
    // One block per SM, balanced ranges of quads (blocks of at least 128 quads on small meshes).
    int threads = lay ? cheb_threads<true>() : cheb_threads<false>(), per_sm = 0;
    if ((e = lay ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb4<true>, threads, bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb4<false>, threads, bytes)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) threads = h.w.threads;              // fewer registers than expected: the CG block size
    const long long nq = h.mesh.N / 4;
    long long nb = (nq + 127) / 128;
    if (nb > h.w.max_blocks) nb = h.w.max_blocks;
    if (nb < 1) nb = 1;
    if ((e = cudaMemsetAsync(h.w.bar, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    void* args[] = {&a, &c};
    const void* k = lay ? (const void*)k_cheb4<true> : (const void*)k_cheb4<false>;
    return cudaLaunchCooperativeKernel(k, dim3((unsigned)nb), dim3(threads), args, bytes, s);
}

cudaError_t esdc_cheb_mixed_launch(const CgArgsHost& h, cudaStream_t s)
{
    if (!h.w.r32) return cudaErrorInvalidValue;
    ChebArgs c;
    if (!esdc_cheb_interval(h.mesh, h.g, c)) return esdc_cg4_launch(h, true, s);     // no interval
    CgArgs a;
    a.m = h.mesh;
    a.g = h.g;
    for (int k = 0; k < 7; ++k) a.dinv[k] = 0.0;
    a.b = h.b;
    a.x = h.x;
    a.r = h.w.r; a.p = h.w.p; a.q = h.w.q; a.z = h.w.z;
    a.part = h.w.part;
    a.bar = h.w.bar;
    a.status = h.w.status;
    a.iter_log = h.iter_log;
    a.flags = h.flags;
    a.tol2 = h.tol * h.tol;
    a.maxit = h.maxit;
    a.precond = 0;
    Cg4MixArgs f;
    f.r = h.w.r32; f.p = h.w.p32; f.q = h.w.q32; f.z = h.w.z32; f.e = h.w.e32;
    f.eta2 = 1e-10;
    f.maxin = h.maxit < 60 ? h.maxit : 60;
    f.maxout = 8;
    // inner iterations: 2 q^k <= 1e-5 (q > 0 whenever the interval has width)
    int kin = f.maxin;
    if (c.q > 0.0) {
        const double kd = std::ceil(std::log(0.5e-5) / c.log_q);
        if (kd < kin) kin = kd < 1.0 ? 1 : (int)kd;
    }
    const int ne = tab_entries(h.mesh);
    const size_t bytes = (sizeof(double) + sizeof(float)) * ne + 16;
    const bool lay = h.mesh.lay != nullptr;
    cudaError_t e = lay ? prepare(k_cheb4_mixed<true>, bytes) : prepare(k_cheb4_mixed<false>, bytes);
    if (e != cudaSuccess) return e;
    const long long nq = h.mesh.N / 4;
    long long nb = (nq + 127) / 128;
    if (nb > h.w.max_blocks) nb = h.w.max_blocks;
    if (nb < 1) nb = 1;
    if ((e = cudaMemsetAsync(h.w.bar, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    void* args[] = {&a, &f, &c, &kin};
    const void* k = lay ? (const void*)k_cheb4_mixed<true> : (const void*)k_cheb4_mixed<false>;
    return cudaLaunchCooperativeKernel(k, dim3((unsigned)nb), dim3(h.w.threads), args, bytes, s);
}

cudaError_t esdc_cg4_launch(const CgArgsHost& h, bool mixed, cudaStream_t s)
{
    CgArgs a;
    a.m = h.mesh;
    a.g = h.g;
    for (int c = 0; c < 7; ++c) a.dinv[c] = 0.0;
    a.b = h.b;
    a.x = h.x;
    a.r = h.w.r; a.p = h.w.p; a.q = h.w.q; a.z = h.w.z;
    a.part = h.w.part;
    a.bar = h.w.bar;
    a.status = h.w.status;
    a.iter_log = h.iter_log;
    a.flags = h.flags;
    a.tol2 = h.tol * h.tol;
    a.maxit = h.maxit;
    a.precond = h.precond;
    const int ne = tab_entries(h.mesh);
    const int nb = quad_blocks(h.mesh, h.w);
    cudaError_t e = cudaMemsetAsync(h.w.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (!mixed) {
        const size_t bytes = sizeof(double) * ne;
        void* args[] = {&a};
        const void* k = h.mesh.lay ? (const void*)k_cg4<true> : (const void*)k_cg4<false>;
        e = h.mesh.lay ? prepare(k_cg4<true>, bytes) : prepare(k_cg4<false>, bytes);
        if (e != cudaSuccess) return e;
        return cudaLaunchCooperativeKernel(k, dim3(nb), dim3(h.w.threads), args, bytes, s);
    }
    if (!h.w.r32) return cudaErrorInvalidValue;
    Cg4MixArgs f;
    f.r = h.w.r32; f.p = h.w.p32; f.q = h.w.q32; f.z = h.w.z32; f.e = h.w.e32;
    f.eta2 = 1e-10;            // each inner solve reduces its residual by 1e-5
    f.maxin = h.maxit < 60 ? h.maxit : 60;
    f.maxout = 8;
    const size_t bytes = (sizeof(double) + sizeof(float)) * ne + 16;
    void* args[] = {&a, &f};
    const void* k = h.mesh.lay ? (const void*)k_cg4_mixed<true> : (const void*)k_cg4_mixed<false>;
    e = h.mesh.lay ? prepare(k_cg4_mixed<true>, bytes) : prepare(k_cg4_mixed<false>, bytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, dim3(nb), dim3(h.w.threads), args, bytes, s);
}
