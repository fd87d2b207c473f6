// Ragged batches: many tissues (meshes of different sizes and conductivities,
// each with its own stimulus and start time) advanced by one HSDC step with the
// same launches a single tissue needs.
//
// Layout.  The tissues are concatenated in every SoA array; tissue b occupies
// nodes [off_b, off_b + N_b) with off_b a multiple of ESDC_TILE (512), so every
// tile of 512 nodes belongs to exactly one tissue.  Node kernels find a node's
// tissue from its tile and skip the padding at the end of each tissue.
//
// Determinism.  Every dot product of the solves is reduced first over one tile, in
// an order fixed by the tile alone (lane l of a warp adds nodes l, l+32, ...,
// then a fixed shuffle tree), then over the tiles of the tissue in tile order.
// The result of every tissue is therefore independent of which other tissues
// share the batch and of the launch shape (blocks, threads, tiles per warp);
// the residual norms are maxima and order-free.  A batch of many tissues gives
// bit for bit the results of the same tissues stepped one at a time, and the
// launch-shape autotuner may choose any configuration without changing a bit.
//
// Solves.  One cooperative launch solves all tissues' systems (I - dt d_i D_b L_b) x = b
// together: the Chebyshev semi-iteration (k_chebb, the default), each tissue on
// its own exactly known spectrum, or the CG (k_cgb).  The grid meets at the same
// barriers, each tissue has its own coefficients and stop test, and a tissue
// that has converged drops out of the work.
// Each block owns a contiguous range of tiles, hence few tissues; it reduces
// only their totals.  The block holding a tissue's first tile records its
// outcome, and the loop ends after the barrier at which every tissue has
// recorded one.
//
// Graphs.  The launches of a step (set-up, K (M+1) node launches, K M solves,
// residual) are captured once per (state buffer, M, K, dt) in a CUDA graph and
// replayed; the only per-step data, the stimulus windows at the collocation
// times, are copied to the device before each replay.
//
// Persistent step.  With the Chebyshev solves the whole step can instead run
// as one cooperative kernel (k_bstep, esdc_batch_set_persistent): the same
// phases, separated by the bounded grid barrier, with the same arithmetic, so
// the same bits.  The autotuner times both launch modes, with their block
// sizes and node tiles, and keeps the faster.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "esdc_kernels.cuh"
#include "esdc_cg_common.cuh"

namespace {

std::mutex g_bconst_mu;
bool g_bconst_done[64] = {false};

constexpr int kMaxBlockTissues = 128;     // tissues one CG block may touch

// ---------------------------------------------------------------- kernels
template <class Model>
__global__ void k_init_b(int64_t n, int64_t ld, ModelDev mp, double V0, double* y)
{
    constexpr int NS = Model::NS;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double u[NS];
        Model::rest(mp.p, V0, u);
        for (int s = 0; s < NS; ++s) y[s * ld + p] = u[s];
    }
}

// Set-up from the iterate in Y (Q^par iterations after the first).
template <class Model, int M>
__global__ void __launch_bounds__(128) k_setup_iter(StepArgs a)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.m.N; p += gridDim.x * blockDim.x) {
        BatchNode n;
        if (!batch_node(a, p, n)) continue;
        setup_iter_body<Model, M>(a, phase_of(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
        // node 1 of the first sweep (it writes y_1's explicit rows, never the
        // V row the stencils of this launch read)
        if (M >= 2 && a.fuse1)
            node_body<Model, M, false, true>(a, next_node1(a), n.m, n.T->st, n.on, n.T->D, p, n.ix, n.iy, n.iz);
    }
}

// Per-tissue residual maxima.  Warp w walks a contiguous range of 32-node
// groups (a group never spans two tiles); running maxima are flushed to the
// tissue's slots when the tissue changes.
template <class Model, int M>
__device__ __forceinline__ void residual_tissues(const StepArgs& a, const PhaseArgs& ph, unsigned long long* rmax)
{
    constexpr int NS = Model::NS;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long ng = (long long)a.m.N >> 5;
    const long long g0 = gw * ng / nw, g1 = (gw + 1) * ng / nw;
    // maxima kept as the bit patterns of non-negative doubles (integer max, as in residual_state)
    unsigned long long rm[NS], ym[NS];
    int cur = -1;
    bool bad = false;
    auto flush = [&](int b) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            unsigned long long r = rm[s], y = ym[s];
            for (int o = 16; o > 0; o >>= 1) {
                r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
                y = max(y, __shfl_xor_sync(0xffffffffu, y, o));
            }
            if (lane == 0) {
                atomicMax(rmax + (size_t)b * 2 * NS + s, r);
                atomicMax(rmax + (size_t)b * 2 * NS + NS + s, y);
            }
        }
    };
    for (long long gi = g0; gi < g1; ++gi) {
        const int p = (int)(gi * 32 + lane);
        const int b = __ldg(a.tile_tissue + (p >> ESDC_TILE_SHIFT));      // the same for the whole warp
        if (b != cur) {
            if (cur >= 0) flush(cur);
            cur = b;
#pragma unroll
            for (int s = 0; s < NS; ++s) { rm[s] = 0ULL; ym[s] = 0ULL; }
        }
        const TissueDev* T = a.tis + b;
        if (p - T->off < T->N) {
#pragma unroll 1
            for (int s = 0; s < NS; ++s) {
                double r, y;
                bad |= !residual_state<Model, M, true>(a, ph, p, s, r, y);
                rm[s] = max(rm[s], (unsigned long long)__double_as_longlong(r));
                ym[s] = max(ym[s], (unsigned long long)__double_as_longlong(y));
            }
        }
    }
    if (cur >= 0) flush(cur);
    if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
}

template <class Model, int M>
__global__ void __launch_bounds__(128) k_residual_b(StepArgs a, unsigned long long* rmax)
{
    residual_tissues<Model, M>(a, phase_of(a), rmax);
}

// dst_i = beta dst_i + sum_j W_ij src_j for collocation rows i < Md, j < Ms,
// every state and column (the interpolators I_l of Sec. 3.2 between node sets).
struct InterpArgs {
    const double* src;
    double* dst;
    int64_t sld, dld, ncols;
    int Ms, Md, ns;
    double beta;
    double W[ESDC_MMAX][ESDC_MMAX];
};

__global__ void k_interp(InterpArgs a)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.ncols; c += (int64_t)gridDim.x * blockDim.x)
        for (int s = 0; s < a.ns; ++s) {
            double v[ESDC_MMAX];
            for (int j = 0; j < a.Ms; ++j) v[j] = a.src[((int64_t)j * a.ns + s) * a.sld + c];
            for (int i = 0; i < a.Md; ++i) {
                double acc = a.beta != 0.0 ? a.beta * a.dst[((int64_t)i * a.ns + s) * a.dld + c] : 0.0;
                for (int j = 0; j < a.Ms; ++j) acc = fma(a.W[i][j], v[j], acc);
                a.dst[((int64_t)i * a.ns + s) * a.dld + c] = acc;
            }
        }
}

struct BCgArgs {
    const TissueDev* tis;
    const int* tile_tissue;
    int ntis, ntiles;
    double gfac;                 // dt d_i: tissue b solves (I - gfac D_b L_b) x = b
    const double* b;
    double* x;
    double *r, *p, *q, *z;
    double* part;                // [6][ntiles] tile partials: set-up r.z, r.r, b.b | p.q | r.z, r.r
    unsigned* bar;
    int* flags;
    int* done_at;                // [ntis] iteration after which the tissue stopped (INT_MAX: running)
    int* status;                 // [ntis][2] iterations, flag bits of the last solve
    int* iter_log;               // [ntis] iterations (optional)
    double tol2;
    int maxit, precond;
};

// Tile partials: lane l of the warp adds nodes l, l + 32, ... of the tile in
// order; then a fixed shuffle tree.  All lanes return the tile's sum.
__device__ __forceinline__ double warp_tree(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct BlockTissues {
    int lo, n;                   // tissues lo .. lo+n-1 touch this block's tiles
    long long t0, t1;            // this block's tiles
};

// Per-tissue totals of nv tile-partial slots for the block's tissues: warp w
// reduces tissues w, w + nwarps, ...; lane l adds tiles l, l + 32, ... of the
// tissue in order, then the fixed tree.  tot[k * nv + v] in shared memory.
__device__ void tissue_totals(const BCgArgs& a, const BlockTissues& bt, const bool* active, int slot0, int nv,
                              double* tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = w; k < bt.n; k += nw) {
        if (!active[k]) continue;
        const TissueDev* T = a.tis + bt.lo + k;
        const int t0 = T->tile0, nt = T->ntile;
        for (int v = 0; v < nv; ++v) {
            const double* pv = a.part + (size_t)(slot0 + v) * a.ntiles + t0;
            double s = 0.0;
            for (int j = lane; j < nt; j += 32) s += __ldcg(pv + j);
            s = warp_tree(s);
            if (lane == 0) tot[k * nv + v] = s;
        }
    }
    __syncthreads();
}

// Node work of one tile: lane l handles nodes tile*512 + l + 32u, u = 0..15.
struct TileGeo {
    int base, nx, ny, nz, N, off;
};

__global__ void __launch_bounds__(512) k_cgb(BCgArgs a)
{
    constexpr int U = ESDC_TILE / 32;
    __shared__ bool s_active[kMaxBlockTissues];
    __shared__ double s_gih2[kMaxBlockTissues], s_diag[kMaxBlockTissues][8], s_dinv[kMaxBlockTissues][8];
    __shared__ double s_rz[kMaxBlockTissues], s_stop[kMaxBlockTissues];
    __shared__ double s_alpha[kMaxBlockTissues], s_beta[kMaxBlockTissues];
    __shared__ double s_tot[kMaxBlockTissues * 3];
    __shared__ int s_exit;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const long long nwt = (long long)gridDim.x * nwb;
    BlockTissues bt;
    bt.t0 = (long long)blockIdx.x * nwb * a.ntiles / nwt;
    bt.t1 = (long long)(blockIdx.x + 1) * nwb * a.ntiles / nwt;
    const long long wt0 = ((long long)blockIdx.x * nwb + w) * a.ntiles / nwt;
    const long long wt1 = ((long long)blockIdx.x * nwb + w + 1) * a.ntiles / nwt;
    if (bt.t1 > bt.t0) {
        bt.lo = a.tile_tissue[bt.t0];
        bt.n = a.tile_tissue[bt.t1 - 1] - bt.lo + 1;
    } else {
        bt.lo = 0;
        bt.n = 0;
    }
    if (bt.n > kMaxBlockTissues) {
        // The host sizes the grid so that this cannot happen.  Leaving now makes
        // the other blocks give up at their next barrier wait (bounded) and
        // report DEVICE_TIMEOUT; no shared-memory slot is ever out of range.
        if (threadIdx.x == 0) atomicOr(a.flags, ESDC_FLAG_TIMEOUT);
        return;
    }
    for (int k = threadIdx.x; k < bt.n; k += blockDim.x) {
        const TissueDev* T = a.tis + bt.lo + k;
        const double gih2 = a.gfac * T->D * T->ih2;
        s_gih2[k] = gih2;
        for (int c = 0; c < 8; ++c) {
            s_diag[k][c] = 1.0 + gih2 * c;
            s_dinv[k][c] = a.precond ? 1.0 / (1.0 + gih2 * c) : 1.0;
        }
        s_active[k] = true;
        if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) a.done_at[bt.lo + k] = INT_MAX;   // this block records it
    }
    __syncthreads();

    // Stencil at node p of the tile's tissue: returns (I - g L) v and the Jacobi factor.
    auto op = [&](const double* v, int p, const TileGeo& G, int k, double& dinv) -> double {
        const int q = p - G.off;
        const int r = q / G.nx;
        const int ix = q - r * G.nx;
        const int iz = r / G.ny;
        const int iy = r - iz * G.ny;
        const int sxy = G.nx * G.ny;
        const double vp = __ldcg(v + p);
        double s = 0.0;
        int c = 0;
        if (ix > 0)        { s += __ldcg(v + p - 1); ++c; }
        if (ix < G.nx - 1) { s += __ldcg(v + p + 1); ++c; }
        if (iy > 0)        { s += __ldcg(v + p - G.nx); ++c; }
        if (iy < G.ny - 1) { s += __ldcg(v + p + G.nx); ++c; }
        if (iz > 0)        { s += __ldcg(v + p - sxy); ++c; }
        if (iz < G.nz - 1) { s += __ldcg(v + p + sxy); ++c; }
        dinv = s_dinv[k][c];
        return fma(s_diag[k][c], vp, -(s_gih2[k] * s));
    };
    auto tile_geo = [&](long long t, int& k) -> TileGeo {
        const int b = a.tile_tissue[t];
        k = b - bt.lo;
        const TissueDev* T = a.tis + b;
        TileGeo G;
        G.base = (int)(t << ESDC_TILE_SHIFT);
        G.nx = T->nx; G.ny = T->ny; G.nz = T->nz; G.N = T->N; G.off = T->off;
        return G;
    };
    unsigned target = 0;

    // [S] r = b - A x, z = D^{-1} r; tile partials r.z, r.r, b.b (slots 0-2)
    for (long long t = wt0; t < wt1; ++t) {
        int k;
        const TileGeo G = tile_geo(t, k);
        double v0 = 0.0, v1 = 0.0, v2 = 0.0;
#pragma unroll 4
        for (int u = 0; u < U; ++u) {
            const int p = G.base + lane + 32 * u;
            if (p - G.off >= G.N) continue;
            double dinv;
            const double ax = op(a.x, p, G, k, dinv);
            const double bp = __ldcg(a.b + p);
            const double rp = bp - ax;
            const double zp = dinv * rp;
            a.r[p] = rp;
            a.z[p] = zp;
            v0 = fma(rp, zp, v0);
            v1 = fma(rp, rp, v1);
            v2 = fma(bp, bp, v2);
        }
        v0 = warp_tree(v0); v1 = warp_tree(v1); v2 = warp_tree(v2);
        if (lane == 0) {
            a.part[t] = v0;
            a.part[(size_t)a.ntiles + t] = v1;
            a.part[2 * (size_t)a.ntiles + t] = v2;
        }
    }
    if (!grid_barrier(a.bar, target, a.flags)) return;
    tissue_totals(a, bt, s_active, 0, 3, s_tot);
    if (threadIdx.x == 0) {
        for (int k = 0; k < bt.n; ++k) {
            const double rz = s_tot[3 * k], rr = s_tot[3 * k + 1], stop = a.tol2 * s_tot[3 * k + 2];
            s_rz[k] = rz; s_stop[k] = stop;
            const bool bad = !isfinite(rr) || !isfinite(stop);
            const bool conv = rr <= stop;
            if (bad || conv) {
                s_active[k] = false;
                const TissueDev* T = a.tis + bt.lo + k;
                if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) {
                    a.done_at[bt.lo + k] = -1;
                    a.status[2 * (bt.lo + k)] = 0;
                    a.status[2 * (bt.lo + k) + 1] = bad ? ESDC_FLAG_NONFINITE : 0;
                    if (a.iter_log) a.iter_log[bt.lo + k] = 0;
                    if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
                }
            }
        }
    }
    __syncthreads();

    for (int it = 0;; ++it) {
        if (it > a.maxit) {                   // cannot happen: every tissue stops by maxit
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
            break;
        }
        // [A] p = z + beta p, q = A z + beta q (first: p = z, q = A z); tile partials p.q (slot 3)
        for (long long t = wt0; t < wt1; ++t) {
            int k;
            const TileGeo G = tile_geo(t, k);
            if (!s_active[k]) continue;
            const double beta = s_beta[k];
            double v = 0.0;
#pragma unroll 4
            for (int u = 0; u < U; ++u) {
                const int p = G.base + lane + 32 * u;
                if (p - G.off >= G.N) continue;
                double dinv;
                const double az = op(a.z, p, G, k, dinv);
                const double zp = __ldcg(a.z + p);
                double pp = zp, qp = az;
                if (it > 0) {
                    pp = fma(beta, a.p[p], zp);
                    qp = fma(beta, a.q[p], az);
                }
                a.p[p] = pp;
                a.q[p] = qp;
                v = fma(pp, qp, v);
            }
            v = warp_tree(v);
            if (lane == 0) a.part[3 * (size_t)a.ntiles + t] = v;
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        // every tissue has stopped by the previous iteration: leave (the same decision in every block)
        if (threadIdx.x < 32) {
            bool all = true;
            for (int b = threadIdx.x; b < a.ntis; b += 32) all &= __ldcg(a.done_at + b) <= it - 1;
            all = __all_sync(0xffffffffu, all);
            if (threadIdx.x == 0) s_exit = all;
        }
        __syncthreads();
        if (s_exit) break;
        tissue_totals(a, bt, s_active, 3, 1, s_tot);
        for (int k = threadIdx.x; k < bt.n; k += blockDim.x)
            if (s_active[k]) s_alpha[k] = s_rz[k] / s_tot[k];
        __syncthreads();
        // [B] x += alpha p, r -= alpha q, z = D^{-1} r; tile partials r.z, r.r (slots 4-5)
        for (long long t = wt0; t < wt1; ++t) {
            int k;
            const TileGeo G = tile_geo(t, k);
            if (!s_active[k]) continue;
            const double alpha = s_alpha[k];
            double v0 = 0.0, v1 = 0.0;
#pragma unroll 4
            for (int u = 0; u < U; ++u) {
                const int p = G.base + lane + 32 * u;
                const int q = p - G.off;
                if (q >= G.N) continue;
                const double rp = fma(-alpha, a.q[p], a.r[p]);
                a.x[p] = fma(alpha, a.p[p], a.x[p]);
                a.r[p] = rp;
                double zq = rp;
                if (a.precond) {
                    const int rr = q / G.nx;
                    const int ix = q - rr * G.nx;
                    const int iz = rr / G.ny;
                    const int iy = rr - iz * G.ny;
                    const int c = (ix > 0) + (ix < G.nx - 1) + (iy > 0) + (iy < G.ny - 1) + (iz > 0) + (iz < G.nz - 1);
                    zq = s_dinv[k][c] * rp;
                }
                a.z[p] = zq;
                v0 = fma(rp, zq, v0);
                v1 = fma(rp, rp, v1);
            }
            v0 = warp_tree(v0); v1 = warp_tree(v1);
            if (lane == 0) {
                a.part[4 * (size_t)a.ntiles + t] = v0;
                a.part[5 * (size_t)a.ntiles + t] = v1;
            }
        }
        if (!grid_barrier(a.bar, target, a.flags)) return;
        tissue_totals(a, bt, s_active, 4, 2, s_tot);
        if (threadIdx.x == 0) {
            for (int k = 0; k < bt.n; ++k) {
                if (!s_active[k]) continue;
                const double rz = s_tot[2 * k], rr = s_tot[2 * k + 1];
                s_beta[k] = rz / s_rz[k];
                s_rz[k] = rz;

                const bool bad = !isfinite(rr);
                const bool conv = rr <= s_stop[k];
                const bool maxed = it + 1 >= a.maxit;
                if (bad || conv || maxed) {
                    s_active[k] = false;
                    const TissueDev* T = a.tis + bt.lo + k;
                    if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) {
                        const int f = bad ? ESDC_FLAG_NONFINITE : (conv ? 0 : ESDC_FLAG_CG_MAXIT);
                        a.done_at[bt.lo + k] = it;
                        a.status[2 * (bt.lo + k)] = it + 1;
                        a.status[2 * (bt.lo + k) + 1] = f;
                        if (a.iter_log) a.iter_log[bt.lo + k] = it + 1;
                        if (f) atomicOr(a.flags, f);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Chebyshev semi-iteration for all tissues at once (options.solver = 0).  The
// spectrum of tissue b's operator I - g_b L_b is [1, 1 + g_b ih2_b wspec_b]
// (cosine modes), so each tissue runs the three-term recurrence on its own
// interval with no inner products: x += d, r -= B d, d = rho' rho d + (2 rho'/delta) r,
// rho' = 1/(2 theta/delta - rho), d_0 = r_0/theta.  Its iteration count comes
// from the bound 2 q^k ||r_0|| <= tol ||b||, q = (sqrt(kappa) - 1)/(sqrt(kappa) + 1);
// the residual is reduced (tile, then tissue, as in k_cgb) only at that
// iteration and every second one after it, and at the cap.  One grid barrier
// per iteration.  The same bookkeeping as k_cgb: the block holding a tissue's
// first tile records its outcome, and the loop ends after the barrier at which
// every tissue has recorded one.  Results per tissue depend on nothing but the
// tissue, so batching keeps them bit for bit.  cheb_all is the solve as a
// device function: `target` carries the grid barrier's count across the
// phases of a persistent kernel; false means a barrier wait gave up (the
// caller must return).
__device__ bool cheb_all(const BCgArgs& a, unsigned& target)
{
    constexpr int U = ESDC_TILE / 32;
    __shared__ bool s_active[kMaxBlockTissues], s_chk[kMaxBlockTissues];
    __shared__ double s_gih2[kMaxBlockTissues], s_diag[kMaxBlockTissues][8];
    __shared__ double s_s1[kMaxBlockTissues], s_delta[kMaxBlockTissues], s_rho[kMaxBlockTissues];
    __shared__ double s_ca[kMaxBlockTissues], s_cb[kMaxBlockTissues], s_stop[kMaxBlockTissues];
    __shared__ double s_itheta[kMaxBlockTissues];
    __shared__ int s_chunk[kMaxBlockTissues];
    __shared__ double s_tot[kMaxBlockTissues * 2];
    __shared__ int s_exit;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const long long nwt = (long long)gridDim.x * nwb;
    BlockTissues bt;
    bt.t0 = (long long)blockIdx.x * nwb * a.ntiles / nwt;
    bt.t1 = (long long)(blockIdx.x + 1) * nwb * a.ntiles / nwt;
    const long long wt0 = ((long long)blockIdx.x * nwb + w) * a.ntiles / nwt;
    const long long wt1 = ((long long)blockIdx.x * nwb + w + 1) * a.ntiles / nwt;
    if (bt.t1 > bt.t0) {
        bt.lo = a.tile_tissue[bt.t0];
        bt.n = a.tile_tissue[bt.t1 - 1] - bt.lo + 1;
    } else {
        bt.lo = 0;
        bt.n = 0;
    }
    if (bt.n > kMaxBlockTissues) {
        // As in k_cgb: the host sizes the grid so that this cannot happen.
        if (threadIdx.x == 0) atomicOr(a.flags, ESDC_FLAG_TIMEOUT);
        return false;
    }
    for (int k = threadIdx.x; k < bt.n; k += blockDim.x) {
        const TissueDev* T = a.tis + bt.lo + k;
        const double gih2 = a.gfac * T->D * T->ih2;
        s_gih2[k] = gih2;
        for (int c = 0; c < 8; ++c) s_diag[k][c] = 1.0 + gih2 * c;
        const double delta = 0.5 * gih2 * T->wspec, theta = 1.0 + delta;
        s_delta[k] = delta;
        s_itheta[k] = 1.0 / theta;
        s_s1[k] = delta > 0.0 ? theta / delta : 0.0;
        s_rho[k] = delta > 0.0 ? delta / theta : 0.0;        // rho_0
        s_active[k] = true;
        if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) a.done_at[bt.lo + k] = INT_MAX;
    }
    __syncthreads();

    auto op = [&](const double* v, int p, const TileGeo& G, int k) -> double {
        const int q = p - G.off;
        const int r = q / G.nx;
        const int ix = q - r * G.nx;
        const int iz = r / G.ny;
        const int iy = r - iz * G.ny;
        const int sxy = G.nx * G.ny;
        const double vp = __ldcg(v + p);
        double s = 0.0;
        int c = 0;
        if (ix > 0)        { s += __ldcg(v + p - 1); ++c; }
        if (ix < G.nx - 1) { s += __ldcg(v + p + 1); ++c; }
        if (iy > 0)        { s += __ldcg(v + p - G.nx); ++c; }
        if (iy < G.ny - 1) { s += __ldcg(v + p + G.nx); ++c; }
        if (iz > 0)        { s += __ldcg(v + p - sxy); ++c; }
        if (iz < G.nz - 1) { s += __ldcg(v + p + sxy); ++c; }
        return fma(s_diag[k][c], vp, -(s_gih2[k] * s));
    };
    auto tile_geo = [&](long long t, int& k) -> TileGeo {
        const int b = a.tile_tissue[t];
        k = b - bt.lo;
        const TissueDev* T = a.tis + b;
        TileGeo G;
        G.base = (int)(t << ESDC_TILE_SHIFT);
        G.nx = T->nx; G.ny = T->ny; G.nz = T->nz; G.N = T->N; G.off = T->off;
        return G;
    };
    double* dc = a.p;                 // d_k
    double* dn = a.q;                 // d_{k+1}

    // [S] r = b - B x, d_0 = r / theta; tile partials r.r, b.b (slots 0-1)
    for (long long t = wt0; t < wt1; ++t) {
        int k;
        const TileGeo G = tile_geo(t, k);
        const double inv_theta = s_itheta[k];
        double v0 = 0.0, v1 = 0.0;
#pragma unroll 4
        for (int u = 0; u < U; ++u) {
            const int p = G.base + lane + 32 * u;
            if (p - G.off >= G.N) continue;
            const double bx = op(a.x, p, G, k);
            const double bp = __ldcg(a.b + p);
            const double rp = bp - bx;
            a.r[p] = rp;
            dc[p] = rp * inv_theta;
            v0 = fma(rp, rp, v0);
            v1 = fma(bp, bp, v1);
        }
        v0 = warp_tree(v0); v1 = warp_tree(v1);
        if (lane == 0) {
            a.part[t] = v0;
            a.part[(size_t)a.ntiles + t] = v1;
        }
    }
    if (!grid_barrier(a.bar, target, a.flags)) return false;
    tissue_totals(a, bt, s_active, 0, 2, s_tot);
    if (threadIdx.x == 0) {
        for (int k = 0; k < bt.n; ++k) {
            const double rr = s_tot[2 * k], stop = a.tol2 * s_tot[2 * k + 1];
            s_stop[k] = stop;
            const bool bad = !isfinite(rr) || !isfinite(stop);
            const bool conv = rr <= stop;
            if (bad || conv) {
                s_active[k] = false;
                const TissueDev* T = a.tis + bt.lo + k;
                if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) {
                    a.done_at[bt.lo + k] = -1;
                    a.status[2 * (bt.lo + k)] = 0;
                    a.status[2 * (bt.lo + k) + 1] = bad ? ESDC_FLAG_NONFINITE : 0;
                    if (a.iter_log) a.iter_log[bt.lo + k] = 0;
                    if (bad) atomicOr(a.flags, ESDC_FLAG_NONFINITE);
                }
                continue;
            }
            // iterations the bound asks for (tol 0: up to the cap)
            int kn = 1;
            const double kap = 1.0 + 2.0 * s_delta[k];
            const double q = (sqrt(kap) - 1.0) / (sqrt(kap) + 1.0);
            if (q > 0.0) {
                const double kd = stop > 0.0 ? ceil(log(0.5 * sqrt(stop / rr)) / log(q)) : (double)a.maxit;
                kn = kd < (double)a.maxit ? (int)kd : a.maxit;
            }
            s_chunk[k] = kn < 1 ? 1 : kn;
        }
    }
    __syncthreads();

    for (int it = 0;; ++it) {
        if (it > a.maxit) {                   // cannot happen: every tissue stops by maxit
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.flags, ESDC_FLAG_CG_MAXIT);
            break;
        }
        // this iteration's coefficients, and which tissues check their residual after it
        for (int k = threadIdx.x; k < bt.n; k += blockDim.x) {
            if (!s_active[k]) { s_chk[k] = false; continue; }
            const double rho = s_rho[k];
            const double rn = s_delta[k] > 0.0 ? 1.0 / (2.0 * s_s1[k] - rho) : 0.0;
            s_ca[k] = rn * rho;
            s_cb[k] = s_delta[k] > 0.0 ? 2.0 * rn / s_delta[k] : 0.0;
            s_rho[k] = rn;
            s_chk[k] = it + 1 >= s_chunk[k] || it + 1 >= a.maxit;
        }
        __syncthreads();
        // [U] x += d, r -= B d, d' = ca d + cb r; tile partials r.r of the checking tissues (slot 2)
        for (long long t = wt0; t < wt1; ++t) {
            int k;
            const TileGeo G = tile_geo(t, k);
            if (!s_active[k]) continue;
            const double ca = s_ca[k], cb = s_cb[k];
            const bool chk = s_chk[k];
            double v = 0.0;
#pragma unroll 4
            for (int u = 0; u < U; ++u) {
                const int p = G.base + lane + 32 * u;
                if (p - G.off >= G.N) continue;
                const double bd = op(dc, p, G, k);
                const double dp = __ldcg(dc + p);
                const double rp = __ldcg(a.r + p) - bd;
                a.x[p] = __ldcg(a.x + p) + dp;
                a.r[p] = rp;
                dn[p] = fma(ca, dp, cb * rp);
                if (chk) v = fma(rp, rp, v);
            }
            if (chk) {
                v = warp_tree(v);
                if (lane == 0) a.part[2 * (size_t)a.ntiles + t] = v;
            }
        }
        double* sw = dc; dc = dn; dn = sw;
        if (!grid_barrier(a.bar, target, a.flags)) return false;
        // every tissue has stopped by the previous iteration: leave (the same decision in every block)
        if (threadIdx.x < 32) {
            bool all = true;
            for (int b = threadIdx.x; b < a.ntis; b += 32) all &= __ldcg(a.done_at + b) <= it - 1;
            all = __all_sync(0xffffffffu, all);
            if (threadIdx.x == 0) s_exit = all;
        }
        __syncthreads();
        if (s_exit) break;
        tissue_totals(a, bt, s_chk, 2, 1, s_tot);
        if (threadIdx.x == 0) {
            for (int k = 0; k < bt.n; ++k) {
                if (!s_chk[k]) continue;
                const double rr = s_tot[k];
                const bool bad = !isfinite(rr);
                const bool conv = rr <= s_stop[k];
                const bool maxed = it + 1 >= a.maxit;
                if (bad || conv || maxed) {
                    s_active[k] = false;
                    const TissueDev* T = a.tis + bt.lo + k;
                    if (T->tile0 >= bt.t0 && T->tile0 < bt.t1) {
                        const int f = bad ? ESDC_FLAG_NONFINITE : (conv ? 0 : ESDC_FLAG_CG_MAXIT);
                        a.done_at[bt.lo + k] = it;
                        a.status[2 * (bt.lo + k)] = it + 1;
                        a.status[2 * (bt.lo + k) + 1] = f;
                        if (a.iter_log) a.iter_log[bt.lo + k] = it + 1;
                        if (f) atomicOr(a.flags, f);
                    }
                } else {
                    s_chunk[k] = it + 3;          // rounding left it short: two more, then check
                }
            }
        }
        __syncthreads();
    }
    return true;
}

__global__ void __launch_bounds__(512, 1) k_chebb(BCgArgs a)
{
    unsigned target = 0;
    cheb_all(a, target);
}

// ---------------------------------------------------------------- one persistent launch per step
// The whole step of every tissue in one cooperative kernel: the set-up, then
// for each sweep k and node i the node phase (ionic evaluation, quadrature,
// right-hand side) and, for i <= M, the Chebyshev solve of all tissues
// (cheb_all), then the residual.  Phases are separated by the bounded grid
// barrier.  Each phase does exactly the arithmetic of the corresponding kernel
// of the launch sequence (the node bodies are per node; the solve's
// reductions are fixed by the 512-node tiles), so the results are bit for bit
// those of the sequence whatever the grid, block size or node tile.
struct BStepArgs {
    int K;
    int from_iter;
    int fuse1;                      // node 1 of each sweep inside the phase before it (M >= 2)
    int tile;                       // node tile: consecutive nodes a warp takes in a node phase (a multiple of 32)
    double gfac[ESDC_MMAX + 1];     // dt d_i, the solves' shifts
    double rho0[ESDC_MMAX + 1];     // warm-start weights c_i / c_{i-1} of sweep 0 from y^0
    double* G0;
    double* G1;
    double* yout;
    double* Y;
    int64_t row;                    // doubles per collocation row of Y (NS * ld)
    unsigned long long* rmax;
    int* cg_log;
    int cg_log_len;
};

// Nodes of a node phase: warp w takes tiles of s.tile consecutive nodes,
// w, w + #warps, ... (lane l of the warp the nodes l, l + 32, ... of a tile).
template <class F>
__device__ __forceinline__ void node_phase(int n, int tile, F body)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = gw * tile; base < n; base += nw * tile)
        for (int o = lane; o < tile; o += 32) {
            const long long p = base + o;
            if (p < n) body((int)p);
        }
}

template <class Model, int M>
__global__ void __launch_bounds__(512, 1) k_bstep(StepArgs a, BCgArgs c, BStepArgs s)
{
    unsigned target = 0;
    const int n = a.m.N;
    PhaseArgs ph{0, 0.0, s.G0, s.G0, nullptr};
    node_phase(n, s.tile, [&](int p) {
        BatchNode nd;
        if (!batch_node(a, p, nd)) return;
        if (s.from_iter) setup_iter_body<Model, M>(a, ph, nd.m, nd.T->st, nd.on, nd.T->D, p, nd.ix, nd.iy, nd.iz);
        else setup_body<Model, M, false>(a, ph, nd.m, nd.T->st, nd.on, nd.T->D, p, nd.ix, nd.iy, nd.iz);
        if (M >= 2 && s.fuse1)
            node_body<Model, M, false, true>(a, PhaseArgs{1, 0.0, s.G0, s.G0, nullptr}, nd.m, nd.T->st, nd.on,
                                             nd.T->D, p, nd.ix, nd.iy, nd.iz);
    });
    if (!grid_barrier(c.bar, target, c.flags)) return;
    double* Gold = s.G0;
    double* Gnew = s.G1;
    for (int k = 0; k < s.K; ++k) {
        for (int i = 1; i <= M + 1; ++i) {
            ph.i = i;
            ph.Gold = Gold;
            ph.Gnew = Gnew;
            ph.rho = (i >= 2 && i <= M) ? (k == 0 && !s.from_iter ? s.rho0[i] : 1.0) : 0.0;
            const bool fused1 = M >= 2 && s.fuse1;
            const bool next1 = fused1 && i == M + 1 && k + 1 < s.K;      // node 1 of sweep k + 1 as well
            if (!(fused1 && i == 1)) {                                     // node 1 ran in the phase before
                node_phase(n, s.tile, [&](int p) {
                    BatchNode nd;
                    if (!batch_node(a, p, nd)) return;
                    node_body<Model, M, false, true>(a, ph, nd.m, nd.T->st, nd.on, nd.T->D, p, nd.ix, nd.iy, nd.iz);
                    if (next1)
                        node_body<Model, M, false, true>(a, PhaseArgs{1, 0.0, Gnew, Gnew, nullptr}, nd.m, nd.T->st,
                                                         nd.on, nd.T->D, p, nd.ix, nd.iy, nd.iz);
                });
                if (!grid_barrier(c.bar, target, c.flags)) return;
            }
            if (i <= M) {
                BCgArgs ci = c;
                ci.gfac = s.gfac[i];
                ci.x = s.Y + (int64_t)(i - 1) * s.row;
                const int slot = k * M + (i - 1);
                ci.iter_log = (slot + 1) * c.ntis <= s.cg_log_len ? s.cg_log + (size_t)slot * c.ntis : nullptr;
                if (!cheb_all(ci, target)) return;
                if (!grid_barrier(c.bar, target, c.flags)) return;
            }
        }
        double* t = Gold; Gold = Gnew; Gnew = t;
    }
    ph.Gold = Gold;
    ph.yout = s.yout;
    residual_tissues<Model, M>(a, ph, s.rmax);
}

// ---------------------------------------------------------------- host
template <class F>
int occupancy(F kernel, int threads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return 0;
    return per_sm;
}

}  // namespace

struct esdc_batch {
    int device = 0, sms = 152;
    int model = 0, NS = 0, NA = 0, NG = 0;
    int ntis = 0, ntiles = 0;
    int64_t ld = 0;
    double chi = 0, Cm = 0;
    esdc_options opt{};
    ColloData col[ESDC_MMAX];
    ModelDev mp{};
    ModelDevF mpf{};
    double* vtab = nullptr;                // the gate table of the model (see ModelDev)
    ZtabSlots zt;                          // set-up coefficient tables per (M, dt)
    const double* cur_ztab = nullptr;      // the table of the step being launched (asked once per step)
    std::vector<TissueDev> tis_h;
    std::vector<unsigned> on_h;            // [ntis][ESDC_MMAX + 1]
    TissueDev* tis = nullptr;
    int* tile_tissue = nullptr;
    unsigned* tis_on = nullptr;
    double *Y = nullptr, *G0 = nullptr, *G1 = nullptr, *FI = nullptr, *S = nullptr, *PHI = nullptr,
           *LAMN = nullptr, *rhs = nullptr, *Vprev = nullptr;
    double* R = nullptr;                   // residual vectors [M_max][NS][ld] (allocated on first request)
    double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *part = nullptr;
    unsigned* bar = nullptr;
    int *done_at = nullptr, *status = nullptr, *cg_log = nullptr, *flags = nullptr;
    int cg_log_len = 0;
    unsigned long long* rmax = nullptr;    // [ntis][2 NS]
    // launch shapes (esdc_batch_tune)
    int node_waves = 1, cg_threads = 512, cg_blocks = 0;
    int occ_node[ESDC_MMAX + 1] = {0}, occ_setup[ESDC_MMAX + 1] = {0}, occ_res[ESDC_MMAX + 1] = {0},
        occ_iter[ESDC_MMAX + 1] = {0};
    // one persistent launch per step (k_bstep; Chebyshev solves only): on/off,
    // block size, node tile, and the occupancy of k_bstep per M and block size
    int persist = 0, p_threads = 512, p_tile = 128;
    int occ_bstep[ESDC_MMAX + 1][2] = {};
    // graph of one step
    bool use_graph = true, graph_failed = false;
    cudaStream_t cap_stream = nullptr;     // private stream the step is recorded on
    struct Graph {                         // one per set-up kind (from y_n / from the iterate)
        cudaGraphExec_t exec = nullptr;
        const double* yin = nullptr;
        double* yout = nullptr;
        const double* tau = nullptr;
        bool keepR = false;
        int M = 0, K = 0;
        double dt = 0.0;
        unsigned ztgen = 0;                // the set-up tables the recording points to
    } graphs[2];
    bool last_graph = false;
    char graph_err[128] = {0};
    // last step
    int last_M = 0, last_K = 0;
    cudaStream_t last_stream = nullptr;
    char err[256] = {0};
};

namespace {

int set_berr(esdc_batch* b, int code, const char* msg)
{
    std::snprintf(b->err, sizeof b->err, "%s", msg);
    return code;
}

void free_batch(esdc_batch* b)
{
    for (auto& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    esdc_ztab_free(b->zt);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    void* ptrs[] = {b->vtab, b->R, b->tis, b->tile_tissue, b->tis_on, b->Y, b->G0, b->G1, b->FI, b->S, b->PHI, b->LAMN,
                    b->rhs, b->Vprev, b->r, b->p, b->q, b->z, b->part, b->bar, b->done_at, b->status,
                    b->cg_log, b->flags, b->rmax};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

int grid_nodes(const esdc_batch* b, int occ, int waves)
{
    long long cap = (long long)b->sms * (occ < 1 ? 1 : occ) * waves;
    long long need = (b->ld + 127) / 128;
    return (int)std::max(1LL, std::min(cap, need));
}

// Largest number of tissues one CG block touches for a grid of nb blocks.
int max_block_tissues(const esdc_batch* b, int nb, int threads)
{
    const int nwb = threads / 32;
    const long long nwt = (long long)nb * nwb;
    int worst = 0;
    for (int blk = 0; blk < nb; ++blk) {
        const long long t0 = (long long)blk * nwb * b->ntiles / nwt, t1 = (long long)(blk + 1) * nwb * b->ntiles / nwt;
        if (t1 <= t0) continue;
        int lo = 0, hi = 0;
        for (int k = 0; k < b->ntis; ++k) {                // tissues are in tile order
            if (b->tis_h[k].tile0 <= t0) lo = k;
            if (b->tis_h[k].tile0 <= t1 - 1) hi = k;
        }
        worst = std::max(worst, hi - lo + 1);
    }
    return worst;
}

int cg_grid(const esdc_batch* b, int threads, int per_sm_wanted)
{
    const int occ = b->opt.solver == 0 ? occupancy(k_chebb, threads) : occupancy(k_cgb, threads);
    if (occ < 1) return 0;
    int per_sm = std::min(occ, per_sm_wanted);
    long long nb = (long long)b->sms * per_sm;
    const long long need = ((long long)b->ntiles + threads / 32 - 1) / (threads / 32);
    nb = std::max(1LL, std::min(nb, need));
    while (nb > 1 && max_block_tissues(b, (int)nb, threads) > kMaxBlockTissues) --nb;
    return (int)nb;
}

// The step's kernel arguments for M collocation nodes and step dt (the
// launch-sequence and the persistent path build them alike).
StepArgs step_args(esdc_batch* b, const double* yin, const double* tau, bool keepR, double dt, int M)
{
    const ColloData* C = &b->col[M - 1];
    StepArgs a{};
    a.m.nx = 1; a.m.ny = 1; a.m.nz = 1;
    a.m.N = (int)b->ld;
    a.m.ld = b->ld;
    a.m.ih2 = 1.0;
    a.mp = b->mp;
    a.mpf = b->mpf;
    a.Vprev = b->Vprev;
    a.dt = dt;
    a.inv_Cm = 1.0 / b->Cm;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            a.dS0[i][j] = dt * C->S0[i][j];
            for (int q = 0; q < M; ++q) a.dtB[i][j][q] = dt * C->B[i][j][q];
        }
    for (int i = 0; i <= M; ++i) a.dtd[i] = dt * C->d[i];
    a.yn = yin;
    a.Y = b->Y; a.FI = b->FI; a.S = b->S; a.PHI = b->PHI; a.LAMN = b->LAMN; a.rhs = b->rhs;
    a.R = keepR ? b->R : nullptr;
    a.tau = tau;
    a.rmax = nullptr;
    a.flags = b->flags;
    a.tis = b->tis;
    a.tile_tissue = b->tile_tissue;
    a.tis_on = b->tis_on;
    return a;
}

// The batched solve's arguments, for the shift gfac, right-hand side rhs and solution x.
BCgArgs cg_args(esdc_batch* b, double gfac, const double* rhs, double* x, int* log)
{
    BCgArgs a;
    a.tis = b->tis;
    a.tile_tissue = b->tile_tissue;
    a.ntis = b->ntis;
    a.ntiles = b->ntiles;
    a.gfac = gfac;
    a.b = rhs;
    a.x = x;
    a.r = b->r; a.p = b->p; a.q = b->q; a.z = b->z;
    a.part = b->part;
    a.bar = b->bar;
    a.flags = b->flags;
    a.done_at = b->done_at;
    a.status = b->status;
    a.iter_log = log;
    a.tol2 = b->opt.tol_cg * b->opt.tol_cg;
    a.maxit = b->opt.cg_maxit;
    a.precond = b->opt.precond;
    return a;
}

// Grid of the persistent step kernel: one or two blocks per SM (within its
// occupancy), fewer if a block's tile range would touch more than
// kMaxBlockTissues tissues.  0 if the kernel cannot run.
int bstep_grid(const esdc_batch* b, int M)
{
    const int occ = b->occ_bstep[M][b->p_threads == 256 ? 0 : 1];
    if (occ < 1) return 0;
    long long nb = (long long)b->sms * std::min(occ, b->p_threads == 256 ? 2 : 1);
    const long long need = ((long long)b->ntiles + b->p_threads / 32 - 1) / (b->p_threads / 32);
    nb = std::max(1LL, std::min(nb, need));
    while (nb > 1 && max_block_tissues(b, (int)nb, b->p_threads) > kMaxBlockTissues) --nb;
    return (int)nb;
}

cudaError_t launch_cgb(esdc_batch* b, double gfac, const double* rhs, double* x, int* log, cudaStream_t s)
{
    BCgArgs a = cg_args(b, gfac, rhs, x, log);
    void* args[] = {&a};
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const void* k = b->opt.solver == 0 ? (const void*)k_chebb : (const void*)k_cgb;
    return cudaLaunchCooperativeKernel(k, dim3(b->cg_blocks), dim3(b->cg_threads), args, 0, s);
}

// Occupancy of the step kernels (queried before any stream capture).
template <class Model, int M>
void batch_prime(esdc_batch* b)
{
    if (b->occ_node[M]) return;
    b->occ_node[M] = occupancy(k_node<Model, M, false, true>, 128);
    b->occ_setup[M] = occupancy(k_setup<Model, M, false, true>, 128);
    b->occ_res[M] = occupancy(k_residual_b<Model, M>, 128);
    b->occ_iter[M] = occupancy(k_setup_iter<Model, M>, 128);
    b->occ_bstep[M][0] = occupancy(k_bstep<Model, M>, 256);
    b->occ_bstep[M][1] = occupancy(k_bstep<Model, M>, 512);
}

// One step of every tissue: y_{n+1} of tissue b to yout (may alias yin).
// from_iter: start from the iterate left in Y by the previous step with the new
// y_n in yin (a Q^par iteration); otherwise from y^0 = 1 (x) y_n.
template <class Model, int M>
cudaError_t batch_step(esdc_batch* b, const double* yin, double* yout, bool from_iter, const double* tau, bool keepR,
                       double dt, int K, cudaStream_t s)
{
    const int T = 128;
    batch_prime<Model, M>(b);
    const ColloData* C = &b->col[M - 1];
    StepArgs a = step_args(b, yin, tau, keepR, dt, M);
    a.ztab = b->cur_ztab;

    cudaError_t e;
    if ((e = cudaMemsetAsync(b->flags, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->rmax, 0, sizeof(unsigned long long) * 2 * b->NS * b->ntis, s)) != cudaSuccess)
        return e;
    a.Gnew = b->G0;
    a.Gold = b->G0;
    // node 1 of each sweep inside the launch before it (as esdc_sweep does)
    const bool fuse = b->opt.fuse_node1 && M >= 2 && K >= 1;
    a.fuse1 = fuse;
    if (from_iter) k_setup_iter<Model, M><<<grid_nodes(b, b->occ_iter[M], b->node_waves), T, 0, s>>>(a);
    else k_setup<Model, M, false, true><<<grid_nodes(b, b->occ_setup[M], b->node_waves), T, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double* Gold = b->G0;
    double* Gnew = b->G1;
    const int nb_node = grid_nodes(b, b->occ_node[M], b->node_waves);
    for (int k = 0; k < K; ++k) {
        a.Gold = Gold;
        a.Gnew = Gnew;
        for (int i = 1; i <= M + 1; ++i) {
            a.i = i;
            a.k = k;
            a.rho = (i >= 2 && i <= M) ? (k == 0 && !from_iter ? C->c[i] / C->c[i - 1] : 1.0) : 0.0;
            a.fuse1 = fuse && i == M + 1 && k + 1 < K;
            if (!(fuse && i == 1)) {
                k_node<Model, M, false, true><<<nb_node, T, 0, s>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            if (i <= M) {
                double* Vi = b->Y + (int64_t)(i - 1) * b->NS * b->ld;
                const int slot = k * M + (i - 1);
                int* log = (slot + 1) * b->ntis <= b->cg_log_len ? b->cg_log + (size_t)slot * b->ntis : nullptr;
                if ((e = launch_cgb(b, dt * C->d[i], b->rhs, Vi, log, s)) != cudaSuccess) return e;
            }
        }
        std::swap(Gold, Gnew);
    }
    a.Gold = Gold;
    a.yout = yout;
    k_residual_b<Model, M><<<grid_nodes(b, b->occ_res[M], b->node_waves), T, 0, s>>>(a, b->rmax);
    return cudaGetLastError();
}

// The same step as one persistent cooperative launch (k_bstep).
template <class Model, int M>
cudaError_t batch_step_persist(esdc_batch* b, const double* yin, double* yout, bool from_iter, const double* tau,
                               bool keepR, double dt, int K, cudaStream_t s)
{
    batch_prime<Model, M>(b);
    const ColloData* C = &b->col[M - 1];
    const int nb = bstep_grid(b, M);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    StepArgs a = step_args(b, yin, tau, keepR, dt, M);
    a.ztab = b->cur_ztab;
    BCgArgs c = cg_args(b, 0.0, b->rhs, nullptr, nullptr);
    BStepArgs st{};
    st.K = K;
    st.from_iter = from_iter ? 1 : 0;
    st.fuse1 = b->opt.fuse_node1 && M >= 2 && K >= 1;
    st.tile = b->p_tile;
    for (int i = 0; i <= M; ++i) {
        st.gfac[i] = dt * C->d[i];
        st.rho0[i] = i >= 2 ? C->c[i] / C->c[i - 1] : 0.0;
    }
    st.G0 = b->G0;
    st.G1 = b->G1;
    st.yout = yout;
    st.Y = b->Y;
    st.row = (int64_t)b->NS * b->ld;
    st.rmax = b->rmax;
    st.cg_log = b->cg_log;
    st.cg_log_len = b->cg_log_len;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->flags, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->rmax, 0, sizeof(unsigned long long) * 2 * b->NS * b->ntis, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    void* args[] = {&a, &c, &st};
    return cudaLaunchCooperativeKernel((const void*)k_bstep<Model, M>, dim3(nb), dim3(b->p_threads), args, 0, s);
}

template <class Model>
cudaError_t batch_persist_M(esdc_batch* b, const double* yin, double* yout, bool fi, const double* tau, bool keepR,
                            double dt, int M, int K, cudaStream_t s)
{
    switch (M) {
        case 1: return batch_step_persist<Model, 1>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 2: return batch_step_persist<Model, 2>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 3: return batch_step_persist<Model, 3>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 4: return batch_step_persist<Model, 4>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 5: return batch_step_persist<Model, 5>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 6: return batch_step_persist<Model, 6>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 7: return batch_step_persist<Model, 7>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 8: return batch_step_persist<Model, 8>(b, yin, yout, fi, tau, keepR, dt, K, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Model>
cudaError_t batch_step_M(esdc_batch* b, const double* yin, double* yout, bool fi, const double* tau, bool keepR,
                         double dt, int M, int K, cudaStream_t s)
{
    switch (M) {
        case 1: return batch_step<Model, 1>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 2: return batch_step<Model, 2>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 3: return batch_step<Model, 3>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 4: return batch_step<Model, 4>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 5: return batch_step<Model, 5>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 6: return batch_step<Model, 6>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 7: return batch_step<Model, 7>(b, yin, yout, fi, tau, keepR, dt, K, s);
        case 8: return batch_step<Model, 8>(b, yin, yout, fi, tau, keepR, dt, K, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Model>
void batch_prime_M(esdc_batch* b, int M)
{
    switch (M) {
        case 1: batch_prime<Model, 1>(b); break;
        case 2: batch_prime<Model, 2>(b); break;
        case 3: batch_prime<Model, 3>(b); break;
        case 4: batch_prime<Model, 4>(b); break;
        case 5: batch_prime<Model, 5>(b); break;
        case 6: batch_prime<Model, 6>(b); break;
        case 7: batch_prime<Model, 7>(b); break;
        case 8: batch_prime<Model, 8>(b); break;
        default: break;
    }
}

cudaError_t batch_launch(esdc_batch* b, const double* yin, double* yout, bool fi, const double* tau, bool keepR,
                         double dt, int M, int K, cudaStream_t s)
{
    if (b->persist && b->opt.solver == 0)
        return b->model == ESDC_MODEL_HH1952 ? batch_persist_M<esdc::HH1952>(b, yin, yout, fi, tau, keepR, dt, M, K, s)
                                             : batch_persist_M<esdc::SYN19>(b, yin, yout, fi, tau, keepR, dt, M, K, s);
    return b->model == ESDC_MODEL_HH1952 ? batch_step_M<esdc::HH1952>(b, yin, yout, fi, tau, keepR, dt, M, K, s)
                                         : batch_step_M<esdc::SYN19>(b, yin, yout, fi, tau, keepR, dt, M, K, s);
}

void drop_graph(esdc_batch* b)
{
    for (auto& g : b->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = esdc_batch::Graph{};
    }
    b->last_graph = false;
}

// Records one step in a graph for (y, M, K, dt).  The recording runs on the
// batch's own stream (the legacy default stream cannot be recorded); the graph
// is then launched on the caller's stream.  On failure the reason is kept and
// the batch falls back to direct launches for good (graph_failed).
bool capture(esdc_batch* b, const double* yin, double* yout, bool fi, const double* tau, bool keepR, double dt, int M,
             int K)
{
    esdc_batch::Graph& G = b->graphs[fi ? 1 : 0];
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G = esdc_batch::Graph{};
    if (b->model == ESDC_MODEL_HH1952) batch_prime_M<esdc::HH1952>(b, M);
    else batch_prime_M<esdc::SYN19>(b, M);
    auto fail = [&](const char* what, cudaError_t e) {
        std::snprintf(b->graph_err, sizeof b->graph_err, "%s: %s", what, cudaGetErrorString(e));
        cudaGetLastError();
        return false;
    };
    cudaError_t e;
    if (!b->cap_stream && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return fail("stream", e);
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return fail("begin capture", e);
    const cudaError_t el = batch_launch(b, yin, yout, fi, tau, keepR, dt, M, K, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (el != cudaSuccess || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return fail("capture", el != cudaSuccess ? el : e);
    }
    e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        G.exec = nullptr;
        return fail("instantiate", e);
    }
    G.yin = yin; G.yout = yout; G.tau = tau; G.keepR = keepR; G.M = M; G.K = K; G.dt = dt;
    G.ztgen = b->zt.gen;
    return true;
}

// Stimulus windows of every tissue at its collocation times, then the step.
int sweep_impl(esdc_batch* b, const double* yin, double* yout, bool fi, const double* tau, bool keepR, const double* t,
               double dt, int M, int K, cudaStream_t s)
{
    const ColloData& C = b->col[M - 1];
    for (int k = 0; k < b->ntis; ++k) {
        if (!std::isfinite(t[k])) return set_berr(b, ESDC_ERR_INVALID_ARG, "non-finite time");
        const StimDev& st = b->tis_h[k].st;
        for (int i = 0; i <= M; ++i) {
            const double tj = t[k] + C.c[i] * dt;
            unsigned on = 0;
            for (int q = 0; q < st.nbox; ++q)
                if (tj >= st.t_on[q] && tj < st.t_off[q]) on |= 1u << q;
            b->on_h[(size_t)k * (ESDC_MMAX + 1) + i] = on;
        }
    }
    // pageable source: the copy has left on_h when the call returns
    if (cudaMemcpyAsync(b->tis_on, b->on_h.data(), sizeof(unsigned) * b->on_h.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return set_berr(b, ESDC_ERR_CUDA, "stimulus window upload failed");
    b->last_M = M; b->last_K = K; b->last_stream = s;
    b->last_graph = false;
    // the set-up's coefficient table, asked for once per step whatever the launch
    // mode (built at the first step with (M, dt), before any recording; a
    // refilled slot moves zt.gen on, and a recording made before is redone)
    b->cur_ztab = esdc_ztab_device(b->zt, M, dt, b->col[M - 1], s);
    if (b->use_graph && !b->graph_failed) {
        const esdc_batch::Graph& G = b->graphs[fi ? 1 : 0];
        if (!(G.exec && G.yin == yin && G.yout == yout && G.tau == tau && G.keepR == keepR && G.M == M && G.K == K &&
              G.dt == dt && G.ztgen == b->zt.gen)) {
            if (!capture(b, yin, yout, fi, tau, keepR, dt, M, K)) b->graph_failed = true;
        }
        if (b->graphs[fi ? 1 : 0].exec && !b->graph_failed) {
            if (cudaGraphLaunch(b->graphs[fi ? 1 : 0].exec, s) != cudaSuccess)
                return set_berr(b, ESDC_ERR_CUDA, "graph launch failed");
            b->last_graph = true;
            return ESDC_OK;
        }
    }
    if (batch_launch(b, yin, yout, fi, tau, keepR, dt, M, K, s) != cudaSuccess)
        return set_berr(b, ESDC_ERR_CUDA, "step launch failed");
    return ESDC_OK;
}

}  // namespace

extern "C" {

int esdc_batch_create(int n, const esdc_mesh* meshes, const double* sigma, double chi, double Cm, int model,
                      const double* params, int n_params, const esdc_options* opt, esdc_batch** out)
{
    if (!out) return ESDC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !meshes || !sigma || !params) return ESDC_ERR_INVALID_ARG;
    if (!(chi > 0.0) || !(Cm > 0.0) || !std::isfinite(chi) || !std::isfinite(Cm)) return ESDC_ERR_INVALID_ARG;
    long long total = 0;
    for (int k = 0; k < n; ++k) {
        const esdc_mesh& m = meshes[k];
        if (m.dim < 1 || m.dim > 3 || m.nx < 1 || m.ny < 1 || m.nz < 1) return ESDC_ERR_INVALID_ARG;
        if ((m.dim < 3 && m.nz != 1) || (m.dim < 2 && m.ny != 1)) return ESDC_ERR_INVALID_ARG;
        if (!(m.h > 0.0) || !std::isfinite(m.h)) return ESDC_ERR_INVALID_ARG;
        if (!(sigma[k] >= 0.0) || !std::isfinite(sigma[k])) return ESDC_ERR_INVALID_ARG;
        const long long N = (long long)m.nx * m.ny * m.nz;
        total += (N + ESDC_TILE - 1) / ESDC_TILE * ESDC_TILE;
        if (total > 0x7fffffffLL - ESDC_TILE) return ESDC_ERR_TOO_LARGE;
    }
    ModelDev mp{};
    ModelDevF mpf{};
    int NS = 0, NG = 0;
    const int rc = esdc_model_setup(model, params, n_params, &mp, &mpf, &NS, &NG);
    if (rc != ESDC_OK) return rc;
    esdc_options o;
    esdc_default_options(&o);
    if (opt) o = *opt;
    if (o.M_max < 1 || o.M_max > ESDC_MMAX || !(o.tol_cg >= 0.0) || o.cg_maxit < 1) return ESDC_ERR_INVALID_ARG;
    if (o.precision != 0) return ESDC_ERR_UNSUPPORTED;            // batches run the FP64 path
    if (o.solver == 3) o.solver = 0;                               // batches: Chebyshev where exact
    if (o.solver != 0 && o.solver != 1) return ESDC_ERR_INVALID_ARG;

    esdc_batch* b = new (std::nothrow) esdc_batch();
    if (!b) return ESDC_ERR_NO_MEMORY;
    auto fail = [&](int code) { free_batch(b); delete b; return code; };
    b->opt = o;
    b->model = model; b->NS = NS; b->NG = NG; b->NA = NS - 1 - NG;
    b->chi = chi; b->Cm = Cm;
    b->mp = mp; b->mpf = mpf;
    {
        std::vector<double> rows;
        double err[2];
        if (esdc_vtab_build(model, mp.p, rows, &err[0], &err[1]) == 0) {
            if (cudaMalloc((void**)&b->vtab, sizeof(double) * rows.size()) != cudaSuccess ||
                cudaMemcpy(b->vtab, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(ESDC_ERR_NO_MEMORY);
            b->mp.vtab = b->vtab;
        }
    }
    b->ntis = n;
    b->tis_h.resize(n);
    int tile = 0;
    for (int k = 0; k < n; ++k) {
        TissueDev& T = b->tis_h[k];
        std::memset(&T, 0, sizeof T);
        T.nx = meshes[k].nx; T.ny = meshes[k].ny; T.nz = meshes[k].nz;
        T.N = T.nx * T.ny * T.nz;
        T.off = tile * ESDC_TILE;
        T.tile0 = tile;
        T.ntile = (T.N + ESDC_TILE - 1) / ESDC_TILE;
        T.ih2 = 1.0 / (meshes[k].h * meshes[k].h);
        T.D = sigma[k] / (chi * Cm);
        const int ext[3] = {T.nx, T.ny, T.nz};
        for (int d = 0; d < 3; ++d)
            if (ext[d] > 1) {
                const double sn = std::sin(M_PI * (ext[d] - 1) / (2.0 * ext[d]));
                T.wspec += 4.0 * sn * sn;
            }
        tile += T.ntile;
    }
    b->ntiles = tile;
    b->ld = (int64_t)tile * ESDC_TILE;
    b->on_h.assign((size_t)n * (ESDC_MMAX + 1), 0u);
    for (int M = 1; M <= ESDC_MMAX; ++M)
        if (esdc_colloc_build(M, &b->col[M - 1])) return fail(ESDC_ERR_CUDA);
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return fail(ESDC_ERR_CUDA);
    {
        std::lock_guard<std::mutex> lk(g_bconst_mu);
        if (upload_constants_local(g_bconst_done, b->device) != cudaSuccess) return fail(ESDC_ERR_CUDA);
    }
    const int64_t ld = b->ld, Mx = o.M_max;
    struct { double** p; int64_t n; } bufs[] = {
        {&b->Y, Mx * NS * ld}, {&b->G0, Mx * NS * ld}, {&b->G1, Mx * NS * ld}, {&b->FI, Mx * ld},
        {&b->S, Mx * Mx * NG * ld}, {&b->PHI, Mx * NG * ld}, {&b->LAMN, NG * ld}, {&b->rhs, ld},
        {&b->Vprev, ld}, {&b->r, ld}, {&b->p, ld}, {&b->q, ld}, {&b->z, ld}, {&b->part, 6LL * tile}};
    for (auto& bf : bufs) {
        cudaError_t e = cudaMalloc((void**)bf.p, sizeof(double) * bf.n);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? ESDC_ERR_NO_MEMORY : ESDC_ERR_CUDA);
        cudaMemset(*bf.p, 0, sizeof(double) * bf.n);
    }
    b->cg_log_len = 64 * ESDC_MMAX * n;
    if (cudaMalloc((void**)&b->tis, sizeof(TissueDev) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->tile_tissue, sizeof(int) * tile) != cudaSuccess ||
        cudaMalloc((void**)&b->tis_on, sizeof(unsigned) * b->on_h.size()) != cudaSuccess ||
        cudaMalloc((void**)&b->bar, sizeof(unsigned) * 4) != cudaSuccess ||
        cudaMalloc((void**)&b->done_at, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc((void**)&b->status, sizeof(int) * 2 * n) != cudaSuccess ||
        cudaMalloc((void**)&b->cg_log, sizeof(int) * b->cg_log_len) != cudaSuccess ||
        cudaMalloc((void**)&b->flags, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&b->rmax, sizeof(unsigned long long) * 2 * NS * n) != cudaSuccess)
        return fail(ESDC_ERR_NO_MEMORY);
    std::vector<int> tt(tile);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < b->tis_h[k].ntile; ++j) tt[b->tis_h[k].tile0 + j] = k;
    if (cudaMemcpy(b->tis, b->tis_h.data(), sizeof(TissueDev) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tile_tissue, tt.data(), sizeof(int) * tile, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ESDC_ERR_CUDA);
    cudaMemset(b->tis_on, 0, sizeof(unsigned) * b->on_h.size());
    cudaMemset(b->bar, 0, sizeof(unsigned) * 4);
    cudaMemset(b->status, 0, sizeof(int) * 2 * n);
    cudaMemset(b->cg_log, 0, sizeof(int) * b->cg_log_len);
    cudaMemset(b->flags, 0, sizeof(int));
    b->cg_threads = 512;
    b->cg_blocks = cg_grid(b, b->cg_threads, 1);
    if (b->cg_blocks < 1) return fail(ESDC_ERR_CUDA);
    if (max_block_tissues(b, b->cg_blocks, b->cg_threads) > kMaxBlockTissues) return fail(ESDC_ERR_UNSUPPORTED);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(ESDC_ERR_CUDA);
    *out = b;
    return ESDC_OK;
}

void esdc_batch_destroy(esdc_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
}

const char* esdc_batch_last_error(const esdc_batch* b) { return b ? b->err : "null batch"; }

int esdc_batch_set_stimulus(esdc_batch* b, int tissue, int nbox, const int* box, const double* amp,
                            const double* t_on, const double* t_off)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (tissue < 0 || tissue >= b->ntis) return set_berr(b, ESDC_ERR_INVALID_ARG, "tissue out of range");
    if (nbox < 0 || nbox > ESDC_MAXBOX) return set_berr(b, ESDC_ERR_INVALID_ARG, "nbox out of range");
    if (nbox > 0 && (!box || !amp || !t_on || !t_off)) return set_berr(b, ESDC_ERR_INVALID_ARG, "null stimulus array");
    StimDev st{};
    st.nbox = nbox;
    for (int k = 0; k < nbox; ++k) {
        for (int c = 0; c < 6; ++c) st.box[k][c] = box[6 * k + c];
        st.amp[k] = amp[k]; st.t_on[k] = t_on[k]; st.t_off[k] = t_off[k];
        if (!std::isfinite(amp[k]) || std::isnan(t_on[k]) || std::isnan(t_off[k]))
            return set_berr(b, ESDC_ERR_INVALID_ARG, "non-finite stimulus value");
    }
    b->tis_h[tissue].st = st;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(b->tis + tissue, &b->tis_h[tissue], sizeof(TissueDev), cudaMemcpyHostToDevice) != cudaSuccess)
        return set_berr(b, ESDC_ERR_CUDA, "stimulus upload failed");
    return ESDC_OK;
}

int esdc_batch_layout(const esdc_batch* b, int* n_state, int64_t* ld, int64_t* offsets)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (n_state) *n_state = b->NS;
    if (ld) *ld = b->ld;
    if (offsets)
        for (int k = 0; k < b->ntis; ++k) offsets[k] = b->tis_h[k].off;
    return ESDC_OK;
}

int esdc_batch_init_state(esdc_batch* b, double* y, double V0, void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (!y || !std::isfinite(V0)) return set_berr(b, ESDC_ERR_INVALID_ARG, "bad init arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)std::min<int64_t>((b->ld + 127) / 128, (int64_t)b->sms * 16);
    if (b->model == ESDC_MODEL_HH1952) k_init_b<esdc::HH1952><<<nb, 128, 0, s>>>(b->ld, b->ld, b->mp, V0, y);
    else k_init_b<esdc::SYN19><<<nb, 128, 0, s>>>(b->ld, b->ld, b->mp, V0, y);
    if (cudaGetLastError() != cudaSuccess) return set_berr(b, ESDC_ERR_CUDA, "init launch failed");
    return ESDC_OK;
}

int esdc_batch_sweep(esdc_batch* b, double* y, const double* t, double dt, int M, int K, void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (!y || !t) return set_berr(b, ESDC_ERR_INVALID_ARG, "null state or time array");
    if (M < 1 || M > b->opt.M_max || K < 1 || K > 64) return set_berr(b, ESDC_ERR_INVALID_ARG, "M or K out of range");
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_berr(b, ESDC_ERR_INVALID_ARG, "dt must be positive");
    return sweep_impl(b, y, y, false, nullptr, false, t, dt, M, K, (cudaStream_t)stream);
}

int esdc_batch_sweep_ex(esdc_batch* b, const double* y_in, double* y_out, const double* tau, const double* t, double dt,
                        int M, int K, int from_iterate, int want_residual, void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (!y_in || !y_out || !t) return set_berr(b, ESDC_ERR_INVALID_ARG, "null state or time array");
    if (M < 1 || M > b->opt.M_max || K < 0 || K > 64 || (K == 0 && !from_iterate))
        return set_berr(b, ESDC_ERR_INVALID_ARG, "M or K out of range");
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_berr(b, ESDC_ERR_INVALID_ARG, "dt must be positive");
    if (want_residual && !b->R) {
        const size_t n = (size_t)b->opt.M_max * b->NS * b->ld;
        if (cudaMalloc((void**)&b->R, sizeof(double) * n) != cudaSuccess)
            return set_berr(b, ESDC_ERR_NO_MEMORY, "residual buffer");
        cudaMemset(b->R, 0, sizeof(double) * n);
    }
    return sweep_impl(b, y_in, y_out, from_iterate != 0, tau, want_residual != 0, t, dt, M, K, (cudaStream_t)stream);
}

int esdc_batch_sweep_from(esdc_batch* b, const double* y_in, double* y_out, const double* t, double dt, int M, int K,
                          int from_iterate, void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (K < 1) return set_berr(b, ESDC_ERR_INVALID_ARG, "K out of range");
    return esdc_batch_sweep_ex(b, y_in, y_out, nullptr, t, dt, M, K, from_iterate, 0, stream);
}

int esdc_batch_iterate(esdc_batch* b, double** Y, double** R)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (Y) *Y = b->Y;
    if (R) *R = b->R;
    return ESDC_OK;
}

int esdc_batch_qpar(esdc_batch* b, double* y_in, double* y_out, double t0, double dt, int M, int iters, void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (!y_in || !y_out || y_in == y_out || iters < 1) return set_berr(b, ESDC_ERR_INVALID_ARG, "bad Q^par arguments");
    const TissueDev& T0 = b->tis_h[0];
    for (const TissueDev& T : b->tis_h)
        if (T.nx != T0.nx || T.ny != T0.ny || T.nz != T0.nz || T.D != T0.D || T.ih2 != T0.ih2)
            return set_berr(b, ESDC_ERR_INVALID_ARG, "Q^par slices must share mesh and conductivity");
    cudaStream_t s = (cudaStream_t)stream;
    const int P = b->ntis;
    const size_t slice = (size_t)T0.ntile * ESDC_TILE;       // columns per slice
    const size_t pitch = sizeof(double) * b->ld;
    std::vector<double> t(P);
    for (int p = 0; p < P; ++p) t[p] = t0 + p * dt;
    // z^0 = 1 (x) y0 in every slice: y_in[p] = y_in[0]
    for (int p = 1; p < P; ++p)
        if (cudaMemcpy2DAsync(y_in + p * slice, pitch, y_in, pitch, sizeof(double) * slice, b->NS,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return set_berr(b, ESDC_ERR_CUDA, "slice copy failed");
    for (int k = 0; k < iters; ++k) {
        const int rc = esdc_batch_sweep_from(b, y_in, y_out, t.data(), dt, M, 1, k > 0, stream);
        if (rc != ESDC_OK) return rc;
        // y_{p+1,0} <- y_{p,M} for the next iteration (slice 0 keeps y0)
        if (P > 1 && cudaMemcpy2DAsync(y_in + slice, pitch, y_out, pitch, sizeof(double) * slice * (P - 1), b->NS,
                                       cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return set_berr(b, ESDC_ERR_CUDA, "slice shift failed");
    }
    return ESDC_OK;
}

int esdc_batch_residual(esdc_batch* b, double* res_inf, double* y_inf)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->last_stream) != cudaSuccess) return set_berr(b, ESDC_ERR_CUDA, "step failed");
    std::vector<unsigned long long> rm((size_t)2 * b->NS * b->ntis);
    int flags = 0;
    if (cudaMemcpy(rm.data(), b->rmax, sizeof(unsigned long long) * rm.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&flags, b->flags, sizeof flags, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_berr(b, ESDC_ERR_CUDA, "reading the residual failed");
    for (int k = 0; k < b->ntis; ++k) {
        double r = 0.0, y = 0.0;
        for (int s = 0; s < b->NS; ++s) {
            double v;
            unsigned long long u = rm[(size_t)k * 2 * b->NS + s];
            std::memcpy(&v, &u, sizeof v);
            r = std::max(r, v);
            u = rm[(size_t)k * 2 * b->NS + b->NS + s];
            std::memcpy(&v, &u, sizeof v);
            y = std::max(y, v);
        }
        if (res_inf) res_inf[k] = r;
        if (y_inf) y_inf[k] = y;
    }
    if (flags & ESDC_FLAG_TIMEOUT) return set_berr(b, ESDC_ERR_DEVICE_TIMEOUT, "CG grid barrier timed out");
    if (flags & ESDC_FLAG_NONFINITE) return set_berr(b, ESDC_ERR_NONFINITE, "non-finite value in the step");
    if (flags & ESDC_FLAG_CG_MAXIT) return set_berr(b, ESDC_ERR_CG_NOT_CONVERGED, "CG hit cg_maxit");
    return ESDC_OK;
}

int esdc_batch_stats(esdc_batch* b, int* cg_iters, int n_entries)
{
    if (!b || !cg_iters || n_entries < 0) return ESDC_ERR_INVALID_ARG;
    const int n = std::min(n_entries, b->last_K * b->last_M * b->ntis);
    if (cudaStreamSynchronize(b->last_stream) != cudaSuccess ||
        (n > 0 && cudaMemcpy(cg_iters, b->cg_log, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess))
        return set_berr(b, ESDC_ERR_CUDA, "reading the statistics failed");
    return ESDC_OK;
}

int esdc_batch_set_graph(esdc_batch* b, int on)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    drop_graph(b);
    b->use_graph = on != 0;
    b->graph_failed = false;
    return ESDC_OK;
}

int esdc_batch_graph_active(const esdc_batch* b)
{
    return (b && b->last_graph) ? 1 : 0;
}

const char* esdc_batch_graph_error(const esdc_batch* b)
{
    return b ? b->graph_err : "null batch";
}

int esdc_batch_set_persistent(esdc_batch* b, int on, int threads, int tile)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if ((on != 0 && on != 1) || (threads != 256 && threads != 512) || tile < 32 || tile > 2048 || (tile & 31))
        return set_berr(b, ESDC_ERR_INVALID_ARG, "persistent launch: on 0/1, threads 256/512, tile a multiple of 32");
    if (on && b->opt.solver != 0) return set_berr(b, ESDC_ERR_UNSUPPORTED, "the persistent step runs the Chebyshev solves");
    if (cudaDeviceSynchronize() != cudaSuccess) return set_berr(b, ESDC_ERR_CUDA, "synchronise");
    drop_graph(b);
    b->persist = on;
    b->p_threads = threads;
    b->p_tile = tile;
    return ESDC_OK;
}

int esdc_batch_get_persistent(const esdc_batch* b, int* on, int* threads, int* tile)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (on) *on = b->persist;
    if (threads) *threads = b->p_threads;
    if (tile) *tile = b->p_tile;
    return ESDC_OK;
}

int esdc_batch_get_shape(const esdc_batch* b, int* node_waves, int* cg_threads, int* cg_blocks)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (node_waves) *node_waves = b->node_waves;
    if (cg_threads) *cg_threads = b->cg_threads;
    if (cg_blocks) *cg_blocks = b->cg_blocks;
    return ESDC_OK;
}

int esdc_batch_set_shape(esdc_batch* b, int node_waves, int cg_threads, int cg_blocks_per_sm)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (node_waves < 1 || node_waves > 8 || (cg_threads != 256 && cg_threads != 512) || cg_blocks_per_sm < 1 ||
        cg_blocks_per_sm > 4)
        return set_berr(b, ESDC_ERR_INVALID_ARG, "launch shape out of range");
    const int nb = cg_grid(b, cg_threads, cg_blocks_per_sm);
    if (nb < 1) return set_berr(b, ESDC_ERR_CUDA, "CG occupancy query failed");
    if (max_block_tissues(b, nb, cg_threads) > kMaxBlockTissues)
        return set_berr(b, ESDC_ERR_UNSUPPORTED, "too many tissues per CG block for this shape");
    cudaDeviceSynchronize();
    drop_graph(b);
    b->node_waves = node_waves;
    b->cg_threads = cg_threads;
    b->cg_blocks = nb;
    return ESDC_OK;
}

int esdc_batch_tune(esdc_batch* b, double* y_scratch, double V0, double t, double dt, int M, int K, int reps,
                    void* stream)
{
    if (!b) return ESDC_ERR_INVALID_ARG;
    if (!y_scratch || reps < 1 || reps > 100 || !std::isfinite(V0))
        return set_berr(b, ESDC_ERR_INVALID_ARG, "bad tuning arguments");
    cudaStream_t s = (cudaStream_t)stream;
    // Candidates: the launch sequence with its launch shapes (node-kernel waves,
    // solve block size and blocks per SM), and, with the Chebyshev solves, the
    // persistent step kernel with its block size and node tile.  None changes
    // a bit of the results.
    struct Shape { int persist, waves, threads, per_sm, tile; };
    const Shape cand[] = {{0, 1, 512, 1, 0}, {0, 2, 512, 1, 0}, {0, 4, 512, 1, 0}, {0, 1, 256, 1, 0},
                          {0, 1, 256, 2, 0}, {0, 2, 256, 2, 0}, {0, 4, 256, 2, 0},
                          {1, 0, 512, 0, 32}, {1, 0, 512, 0, 128}, {1, 0, 512, 0, 512},
                          {1, 0, 256, 0, 32}, {1, 0, 256, 0, 64}, {1, 0, 256, 0, 128}};
    std::vector<double> tv(b->ntis, t);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return set_berr(b, ESDC_ERR_CUDA, "event creation failed");
    }
    float best = 1e30f;
    Shape pick = {b->persist, b->node_waves, b->cg_threads, 0, b->p_tile};
    int pick_blocks = b->cg_blocks, pick_pthreads = b->p_threads;
    const Shape seq0 = {0, b->node_waves, b->cg_threads, 0, 0};
    int rc = ESDC_OK;
    for (const Shape& c : cand) {
        if (c.persist) {
            if (b->opt.solver != 0) continue;
            if (esdc_batch_set_persistent(b, 1, c.threads, c.tile) != ESDC_OK) continue;
        } else {
            if (esdc_batch_set_persistent(b, 0, b->p_threads, b->p_tile) != ESDC_OK) continue;
            if (esdc_batch_set_shape(b, c.waves, c.threads, c.per_sm) != ESDC_OK) continue;
        }
        rc = esdc_batch_init_state(b, y_scratch, V0, stream);
        if (rc == ESDC_OK) rc = esdc_batch_sweep(b, y_scratch, tv.data(), dt, M, K, stream);   // capture, warm-up
        if (rc == ESDC_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = ESDC_ERR_CUDA;
        for (int r = 0; r < reps && rc == ESDC_OK; ++r) rc = esdc_batch_sweep(b, y_scratch, tv.data(), dt, M, K, stream);
        if (rc == ESDC_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = ESDC_ERR_CUDA;
        if (rc != ESDC_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
            if (!c.persist) pick_blocks = b->cg_blocks;
            else pick_pthreads = c.threads;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ESDC_OK) return rc;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (pick.persist) {
        b->persist = 1;
        b->p_threads = pick_pthreads;
        b->p_tile = pick.tile;
    } else {
        b->persist = 0;
        b->node_waves = pick.waves ? pick.waves : seq0.waves;
        b->cg_threads = pick.threads;
        b->cg_blocks = pick_blocks;
    }
    return ESDC_OK;
}

int esdc_interp(const double* src, int Ms, int64_t src_ld, double* dst, int Md, int64_t dst_ld, int n_state,
                int64_t n_cols, const double* W, double beta, void* stream)
{
    if (!src || !dst || !W || Ms < 1 || Md < 1 || Ms > ESDC_MMAX || Md > ESDC_MMAX || n_state < 1 || n_cols < 0 ||
        src_ld < n_cols || dst_ld < n_cols || !std::isfinite(beta))
        return ESDC_ERR_INVALID_ARG;
    if (n_cols == 0) return ESDC_OK;
    if (src == dst) return ESDC_ERR_INVALID_ARG;              // rows are read before they are written, per column only
    InterpArgs a{};
    a.src = src; a.dst = dst; a.sld = src_ld; a.dld = dst_ld; a.ncols = n_cols;
    a.Ms = Ms; a.Md = Md; a.ns = n_state; a.beta = beta;
    for (int i = 0; i < Md; ++i)
        for (int j = 0; j < Ms; ++j) {
            if (!std::isfinite(W[i * Ms + j])) return ESDC_ERR_INVALID_ARG;
            a.W[i][j] = W[i * Ms + j];
        }
    const long long nb = std::min<long long>((n_cols + 255) / 256, 152LL * 8);
    k_interp<<<(int)nb, 256, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? ESDC_OK : ESDC_ERR_CUDA;
}

int esdc_hsdc(esdc_batch* const* levels, esdc_batch* const* coarse, const int* M, int L, double* y_in,
              double* y_out, double t0, double dt, int iters, void* stream)
{
    if (!levels || !levels[0]) return ESDC_ERR_INVALID_ARG;
    esdc_batch* fine = levels[0];
    if (!coarse || !M || !y_in || !y_out || y_in == y_out || iters < 1 || L < 2 || L > ESDC_MMAX)
        return set_berr(fine, ESDC_ERR_INVALID_ARG, "bad multilevel arguments");
    for (int l = 0; l < L; ++l)
        if (M[l] < 1 || (l > 0 && M[l] >= M[l - 1]) || (l < L - 1 && (!levels[l] || M[l] > levels[l]->opt.M_max)))
            return set_berr(fine, ESDC_ERR_INVALID_ARG, "levels need M_1 > M_2 > ... > M_L and M_l <= M_max");
    const int P = fine->ntis, NSt = fine->NS;
    const TissueDev& T0 = fine->tis_h[0];
    for (const TissueDev& T : fine->tis_h)
        if (T.nx != T0.nx || T.ny != T0.ny || T.nz != T0.nz || T.D != T0.D || T.ih2 != T0.ih2)
            return set_berr(fine, ESDC_ERR_INVALID_ARG, "slices must share mesh and conductivity");
    const int64_t slice = (int64_t)T0.ntile * ESDC_TILE, ldf = fine->ld;
    for (int l = 1; l < L - 1; ++l) {                 // the Q^par levels share the fine level's layout
        const esdc_batch* b = levels[l];
        if (b->ntis != P || b->ld != ldf || b->NS != NSt || b->tis_h[0].N != T0.N || b->tis_h[0].D != T0.D ||
            b->tis_h[0].ih2 != T0.ih2 || b->tis_h[0].ntile != T0.ntile)
            return set_berr(fine, ESDC_ERR_INVALID_ARG, "every Q^par level: the same slices as the finest");
    }
    const int Mc = M[L - 1];
    for (int p = 0; p < P; ++p) {
        const esdc_batch* c = coarse[p];
        if (!c || c->ntis != 1 || c->ld != slice || c->NS != NSt || c->opt.M_max < Mc || c->tis_h[0].N != T0.N ||
            c->tis_h[0].D != T0.D || c->tis_h[0].ih2 != T0.ih2)
            return set_berr(fine, ESDC_ERR_INVALID_ARG, "coarsest level: one single-slice batch per slice, same mesh");
    }
    // Lagrange matrices between the Radau nodes c_1..c_M of consecutive levels
    // (Sec. 3.2: I_l(y, s) = sum_j l_j(s) y_j): restriction S_l [M_{l+1}][M_l],
    // prolongation T_l [M_l][M_{l+1}]
    auto lagrange = [](const double* nodes, int n, const double* pts, int m, double* W) {
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double l = 1.0;
                for (int k = 0; k < n; ++k)
                    if (k != j) l *= (pts[i] - nodes[k]) / (nodes[j] - nodes[k]);
                W[i * n + j] = l;
            }
    };
    std::vector<std::vector<double>> Sm(L - 1), Tm(L - 1);
    for (int l = 0; l < L - 1; ++l) {
        const double* ca = fine->col[M[l] - 1].c + 1;
        const double* cb = fine->col[M[l + 1] - 1].c + 1;
        Sm[l].resize((size_t)M[l + 1] * M[l]);
        Tm[l].resize((size_t)M[l] * M[l + 1]);
        lagrange(ca, M[l], cb, M[l + 1], Sm[l].data());
        lagrange(cb, M[l + 1], ca, M[l], Tm[l].data());
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pitchf = sizeof(double) * ldf, pitchc = sizeof(double) * slice;
    const int64_t rowsf = (int64_t)NSt * ldf, rowsc = (int64_t)NSt * slice;
    struct Scratch {
        std::vector<void*> p;
        ~Scratch() { for (void* q : p) cudaFree(q); }
    } sc;
    auto alloc = [&](double** q, int64_t n) {
        if (cudaMalloc((void**)q, sizeof(double) * n) != cudaSuccess) return false;
        sc.p.push_back(*q);
        return true;
    };
    // per Q^par level l >= 1: S z_{l-1} [M_l][NS][ld], tau_l (same), its slices' initial values [NS][ld];
    // coarsest level, per slice: S z, tau, y_{p,0} and the new end values
    std::vector<double*> SZl(L, nullptr), TAUl(L, nullptr), Y0l(L, nullptr);
    double *SZ = nullptr, *TAU = nullptr, *YIC = nullptr, *YOC = nullptr, *ytmp = nullptr;
    for (int l = 1; l < L - 1; ++l)
        if (!alloc(&SZl[l], (int64_t)M[l] * rowsf) || !alloc(&TAUl[l], (int64_t)M[l] * rowsf) ||
            !alloc(&Y0l[l], rowsf))
            return set_berr(fine, ESDC_ERR_NO_MEMORY, "multilevel scratch");
    if (!alloc(&SZ, (int64_t)P * Mc * rowsc) || !alloc(&TAU, (int64_t)P * Mc * rowsc) || !alloc(&YIC, rowsc) ||
        !alloc(&YOC, (int64_t)P * rowsc) || !alloc(&ytmp, rowsf))
        return set_berr(fine, ESDC_ERR_NO_MEMORY, "multilevel scratch");
    Y0l[0] = y_in;
    std::vector<double> tf(P);
    for (int p = 0; p < P; ++p) tf[p] = t0 + p * dt;
    std::vector<double> Im(Mc * Mc, 0.0), Ip(Mc * Mc, 0.0);     // -I and +I of the coarsest level
    for (int i = 0; i < Mc; ++i) { Im[i * Mc + i] = -1.0; Ip[i * Mc + i] = 1.0; }
    // the calls below alternate between kinds of step: record no graphs
    struct GraphsOff {
        std::vector<esdc_batch*> b;
        std::vector<char> was;
        ~GraphsOff() { for (size_t i = 0; i < b.size(); ++i) b[i]->use_graph = was[i] != 0; }
        void add(esdc_batch* x) { b.push_back(x); was.push_back(x->use_graph); x->use_graph = false; }
    } graphs_off;
    for (int l = 0; l < L - 1; ++l) graphs_off.add(levels[l]);
    for (int p = 0; p < P; ++p) graphs_off.add(coarse[p]);
    auto fail_cuda = [&](const char* what) { return set_berr(fine, ESDC_ERR_CUDA, what); };
    // y_{p,0} of slice p >= 1 := row M-1 of slice p-1 of the iterate Z (the Q^par coupling)
    auto shift_ends = [&](double* y0dst, const double* Z, int Ml) {
        return P > 1 && cudaMemcpy2DAsync(y0dst + slice, pitchf, Z + (int64_t)(Ml - 1) * rowsf, pitchf,
                                          sizeof(double) * slice * (P - 1), NSt, cudaMemcpyDeviceToDevice,
                                          s) != cudaSuccess;
    };
    std::vector<double*> Yl(L - 1, nullptr), Rl(L - 1, nullptr);
    int rc;
    // z^0 = 1 (x) y0 in every slice: y_in[p] = y0, Y_j = y0
    for (int p = 1; p < P; ++p)
        if (cudaMemcpy2DAsync(y_in + p * slice, pitchf, y_in, pitchf, pitchc, NSt, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return fail_cuda("slice copy failed");
    // K = 0 calls allocate the residual buffers and give the iterate pointers
    for (int l = 0; l < L - 1; ++l) {
        if ((rc = esdc_batch_sweep_ex(levels[l], y_in, ytmp, nullptr, tf.data(), dt, M[l], 0, 1, 1, stream)) !=
            ESDC_OK)
            return rc;
        esdc_batch_iterate(levels[l], &Yl[l], &Rl[l]);
    }
    for (int j = 0; j < M[0]; ++j)
        if (cudaMemcpyAsync(Yl[0] + (int64_t)j * rowsf, y_in, sizeof(double) * rowsf, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return fail_cuda("spread failed");
    for (int k = 0; k < iters; ++k) {
        // finest level: its residual vectors at the iterate (tau_1 = 0)
        if ((rc = esdc_batch_sweep_ex(fine, y_in, ytmp, nullptr, tf.data(), dt, M[0], 0, 1, 1, stream)) != ESDC_OK)
            return rc;
        // down: tau_l = S R_{l-1}(z_{l-1}; tau_{l-1}) - R_l(S z_{l-1}); one Q^par sweep from S z_{l-1} with tau_l
        for (int l = 1; l < L - 1; ++l) {
            esdc_batch* b = levels[l];
            if ((rc = esdc_interp(Yl[l - 1], M[l - 1], ldf, SZl[l], M[l], ldf, NSt, ldf, Sm[l - 1].data(), 0.0,
                                  stream)) != ESDC_OK)
                return set_berr(fine, rc, "restriction failed");
            if (cudaMemcpyAsync(Yl[l], SZl[l], sizeof(double) * M[l] * rowsf, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return fail_cuda("iterate copy failed");
            if ((rc = esdc_batch_sweep_ex(b, Y0l[l - 1], ytmp, nullptr, tf.data(), dt, M[l], 0, 1, 1, stream)) !=
                ESDC_OK)
                return rc;
            if ((rc = esdc_interp(Rl[l - 1], M[l - 1], ldf, TAUl[l], M[l], ldf, NSt, ldf, Sm[l - 1].data(), 0.0,
                                  stream)) != ESDC_OK)
                return set_berr(fine, rc, "tau failed");
            {
                std::vector<double> Iml(M[l] * M[l], 0.0);
                for (int i = 0; i < M[l]; ++i) Iml[i * M[l] + i] = -1.0;
                if ((rc = esdc_interp(Rl[l], M[l], ldf, TAUl[l], M[l], ldf, NSt, ldf, Iml.data(), 1.0, stream)) !=
                    ESDC_OK)
                    return set_berr(fine, rc, "tau failed");
            }
            // the sweep: slice p starts from the end of slice p-1 of S z_{l-1}; it keeps R_l(z_l; tau_l)
            if (cudaMemcpy2DAsync(Y0l[l], pitchf, y_in, pitchf, pitchc, NSt, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess ||
                shift_ends(Y0l[l], SZl[l], M[l]))
                return fail_cuda("slice shift failed");
            if ((rc = esdc_batch_sweep_ex(b, Y0l[l], ytmp, TAUl[l], tf.data(), dt, M[l], 1, 1, 1, stream)) != ESDC_OK)
                return rc;
        }
        // coarsest level, per slice: S z, tau = S R_{L-1} - R_L(S z)
        const int lp = L - 2;                                      // the level above the coarsest
        for (int p = 0; p < P; ++p) {
            esdc_batch* c = coarse[p];
            double *Yc = nullptr, *Rc = nullptr;
            double* SZp = SZ + (int64_t)p * Mc * rowsc;
            double* TAUp = TAU + (int64_t)p * Mc * rowsc;
            const double tp = tf[p];
            if ((rc = esdc_interp(Yl[lp] + p * slice, M[lp], ldf, SZp, Mc, slice, NSt, slice, Sm[lp].data(), 0.0,
                                  stream)) != ESDC_OK)
                return set_berr(fine, rc, "restriction failed");
            if (cudaMemcpy2DAsync(YIC, pitchc, Y0l[lp] + p * slice, pitchf, pitchc, NSt, cudaMemcpyDeviceToDevice,
                                  s) != cudaSuccess)
                return fail_cuda("slice copy failed");
            esdc_batch_iterate(c, &Yc, nullptr);
            if (cudaMemcpyAsync(Yc, SZp, sizeof(double) * Mc * rowsc, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return fail_cuda("iterate copy failed");
            if ((rc = esdc_batch_sweep_ex(c, YIC, YOC + p * rowsc, nullptr, &tp, dt, Mc, 0, 1, 1, stream)) != ESDC_OK)
                return rc;
            esdc_batch_iterate(c, nullptr, &Rc);
            if ((rc = esdc_interp(Rl[lp] + p * slice, M[lp], ldf, TAUp, Mc, slice, NSt, slice, Sm[lp].data(), 0.0,
                                  stream)) != ESDC_OK ||
                (rc = esdc_interp(Rc, Mc, slice, TAUp, Mc, slice, NSt, slice, Im.data(), 1.0, stream)) != ESDC_OK)
                return set_berr(fine, rc, "tau failed");
        }
        // coarsest Q^seq sweep (slice p starts from the new end value of slice p-1), then the
        // coarse-grid correction of level L-1: z += T (z_L - S z)
        for (int p = 0; p < P; ++p) {
            esdc_batch* c = coarse[p];
            double *Yc = nullptr, *Rc = nullptr;
            esdc_batch_iterate(c, &Yc, &Rc);
            if (p == 0) {
                if (cudaMemcpy2DAsync(YIC, pitchc, y_in, pitchf, pitchc, NSt, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    return fail_cuda("slice copy failed");
            } else if (cudaMemcpyAsync(YIC, YOC + (p - 1) * rowsc, sizeof(double) * rowsc, cudaMemcpyDeviceToDevice,
                                       s) != cudaSuccess) {
                return fail_cuda("slice copy failed");
            }
            if (cudaMemcpyAsync(Yc, SZ + (int64_t)p * Mc * rowsc, sizeof(double) * Mc * rowsc,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return fail_cuda("iterate copy failed");
            const double tp = tf[p];
            if ((rc = esdc_batch_sweep_ex(c, YIC, YOC + p * rowsc, TAU + (int64_t)p * Mc * rowsc, &tp, dt, Mc, 1, 1, 0,
                                          stream)) != ESDC_OK)
                return rc;
            double* SZp = SZ + (int64_t)p * Mc * rowsc;
            if ((rc = esdc_interp(Yc, Mc, slice, SZp, Mc, slice, NSt, slice, Ip.data(), -1.0, stream)) != ESDC_OK ||
                (rc = esdc_interp(SZp, Mc, slice, Yl[lp] + p * slice, M[lp], ldf, NSt, slice, Tm[lp].data(), 1.0,
                                  stream)) != ESDC_OK)
                return set_berr(fine, rc, "correction failed");
        }
        // up: one Q^par sweep of level l from its corrected iterate (slice p starts from
        // that iterate's end of slice p-1), then the correction of level l-1
        for (int l = L - 2; l >= 0; --l) {
            esdc_batch* b = levels[l];
            if (l > 0 && cudaMemcpy2DAsync(Y0l[l], pitchf, y_in, pitchf, pitchc, NSt, cudaMemcpyDeviceToDevice, s) !=
                             cudaSuccess)
                return fail_cuda("slice copy failed");
            if (shift_ends(Y0l[l], Yl[l], M[l])) return fail_cuda("slice shift failed");
            if ((rc = esdc_batch_sweep_ex(b, Y0l[l], l == 0 ? y_out : ytmp, l == 0 ? nullptr : TAUl[l], tf.data(), dt,
                                          M[l], 1, 1, 0, stream)) != ESDC_OK)
                return rc;
            if (l > 0) {
                // z_{l-1} += T (z_l - S z_{l-1}): the difference in place of S z_{l-1}
                std::vector<double> Ipl(M[l] * M[l], 0.0);
                for (int i = 0; i < M[l]; ++i) Ipl[i * M[l] + i] = 1.0;
                if ((rc = esdc_interp(Yl[l], M[l], ldf, SZl[l], M[l], ldf, NSt, ldf, Ipl.data(), -1.0, stream)) !=
                        ESDC_OK ||
                    (rc = esdc_interp(SZl[l], M[l], ldf, Yl[l - 1], M[l - 1], ldf, NSt, ldf, Tm[l - 1].data(), 1.0,
                                      stream)) != ESDC_OK)
                    return set_berr(fine, rc, "correction failed");
            }
        }
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? ESDC_OK : set_berr(fine, ESDC_ERR_CUDA, "multilevel run failed");
}

int esdc_hsdc2(esdc_batch* fine, esdc_batch* const* coarse, double* y_in, double* y_out, double t0, double dt, int M1,
               int M2, int iters, void* stream)
{
    if (!fine) return ESDC_ERR_INVALID_ARG;
    esdc_batch* levels[1] = {fine};
    const int M[2] = {M1, M2};
    return esdc_hsdc(levels, coarse, M, 2, y_in, y_out, t0, dt, iters, stream);
}

}  // extern "C"
