// Grid-wide building blocks of the persistent CG kernels: a bounded grid
// barrier and deterministic block / grid reductions.  Shared by the scalar
// (one node per thread) and the quad (four x-consecutive nodes per thread)
// kernels.
#pragma once
#include "esdc_internal.h"

namespace {

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // give up a barrier wait after 1 s

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct CgArgs {
    MeshDev m;
    double g;
    double dinv[7];          // inverse diagonal of I - g L by neighbour count
    const double* b;
    double* x;
    double *r, *p, *q, *z;
    double* part;            // [6][nblocks]: setup r.z, r.r, b.b | p.q | r.z, r.r
    unsigned* bar;           // barrier arrival counter
    int* status;             // [0] iterations, [1] flags
    int* iter_log;
    int* flags;
    double tol2;
    int maxit;
    int precond;
};

// Grid barrier on one monotonic arrival counter bar[0] (zeroed before the
// launch): barrier number b is passed once the counter reaches b * gridDim.x.
// Thread 0 of each block adds its arrival and polls with acquire loads,
// tightly at first, then with short sleeps; after 1 s of waiting it raises
// TIMEOUT and returns false, and the caller must return from the kernel.
// bar[2] and bar[3] are zero in use.  esdc_debug_barrier sets them to make the
// waits of a solve run out on purpose (the failure path, tested on the host's
// side): bar[2] = 1 + the index of a block that does not arrive at the
// kernel's first barrier, bar[3] = the wait limit in microseconds (0: 1 s).
// bar[2] is read at the first barrier only and bar[3] only once a wait is long.
__device__ bool grid_barrier(unsigned* bar, unsigned& target, int* flags)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        const bool skip = target == gridDim.x && __ldcg(bar + 2) == blockIdx.x + 1;
        __threadfence();
        if (!skip) atomicAdd(bar, 1u);
        int ok = 1;
        if (load_acquire(bar) < target) {
            const unsigned long long t0 = global_ns();
            unsigned long long limit = 0;
            unsigned spins = 0;
            while (load_acquire(bar) < target) {
                if (++spins > 32) __nanosleep(32);
                if ((spins & 255u) == 0) {
                    if (!limit) {
                        const unsigned us = __ldcg(bar + 3);
                        limit = us ? 1000ull * us : kWaitLimitNs;
                    }
                    if (global_ns() - t0 > limit) {
                        ok = 0;
                        atomicOr(flags, ESDC_FLAG_TIMEOUT);
                        break;
                    }
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Block sum of up to three values in a fixed order: every thread stores its
// value, lane l of warp 0 adds the values of lane l of all warps (in warp
// order), then warp 0 reduces its 32 sums with a shuffle tree.  Few FP64 adds
// per thread: the FP64 pipe is the scarce unit.
// One reduction buffer per kernel, whatever the number of block_sum<NV>
// instantiations it uses.
__device__ __forceinline__ double (*red_buf())[32][33]
{
    __shared__ double sh[3][32][33];
    return sh;
}

template <int NV>
__device__ void block_sum(double (&v)[NV], double* out)
{
    static_assert(NV <= 3, "block_sum reduces at most three values");
    double (*sh)[32][33] = red_buf();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][lane][wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = sh[k][lane][0];
            for (int w = 1; w < nw; ++w) s += sh[k][lane][w];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) out[k] = s;
        }
    }
    __syncthreads();
}

// Every block sums the partials of all blocks: lane l of warp 0 adds partials
// l, l+32, ... in order, then a shuffle tree; the result is broadcast through
// shared memory, so every block obtains the same bits.  The partials were
// written by other blocks before the last barrier; __ldcg reads them from L2,
// past this SM's L1.
template <int NV>
__device__ void grid_total(const double* part, int off0, double (&tot)[NV])
{
    __shared__ double res[NV];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double* pk = part + (size_t)(off0 + k) * gridDim.x;
            double s = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(pk + b);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) res[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = res[k];
    __syncthreads();
}

// grid_total, plus one quotient computed once per block by lane 0 and
// broadcast with the sums: q = num / tot[0] (MODE 1) or q = tot[0] / num
// (MODE 2).  An FP64 division is a few dozen FP64-pipe operations; repeated by
// every thread of every block it costs as much as a stencil pass on small meshes.
template <int NV, int MODE>
__device__ void grid_total_q(const double* part, int off0, double (&tot)[NV], double num, double& q)
{
    __shared__ double res[NV + 1];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double* pk = part + (size_t)(off0 + k) * gridDim.x;
            double s = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(pk + b);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) res[k] = s;
        }
        if (lane == 0) res[NV] = MODE == 1 ? num / res[0] : res[0] / num;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = res[k];
    q = res[NV];
    __syncthreads();
}

struct NodeIdx { int ix, iy, iz; };

__device__ __forceinline__ NodeIdx node_idx(const MeshDev& m, int p)
{
    NodeIdx n;
    int r = p / m.nx;
    n.ix = p - r * m.nx;
    n.iz = r / m.ny;
    n.iy = r - n.iz * m.ny;
    return n;
}

}  // namespace
