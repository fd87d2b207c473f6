// Allocation-free diffusion solve.
//
// Some callers cannot allocate device memory at all: code running where
// cudaMalloc is forbidden or unavailable (inside a custom allocator or memory
// pool callback, in a process whose device memory is fully reserved up front by
// another framework, or in embedded/real-time loops that must not call into
// the allocator after start-up).  They cannot create a handle, because
// esdc_create allocates the workspace.  esdc_diffusion_solve_static gives them
// the diffusion solve (I - g L) x = b with all of its scratch -- the CG
// vectors, the block partial sums and the grid-barrier counter -- placed in one
// file-scope device array of fixed size, compiled into the library.
//
// Consequences a caller must know:
//  * Every GPU that loads the library holds ESDC_STATIC_SCRATCH_BYTES of device
//    memory for this array until the process exits.
//  * Meshes with more than ESDC_STATIC_MAX_NODES nodes are rejected with
//    ESDC_ERR_TOO_LARGE.
//  * All calls share the array.  Two calls whose work overlaps on the GPU (on
//    different streams, or from different host threads without ordering) race
//    on it and give wrong results; serialise them.
//  * The first call on each device looks up the array's device address (see
//    below).  Make that first call before any stream capture starts.
#include <cstring>
#include <mutex>

#include "esdc_internal.h"

namespace {

// Layout of the scratch array (in doubles):
//   r, p, q, z        4 x ESDC_STATIC_MAX_NODES
//   partial sums      8 x kMaxBlocks (the slots CgWork::part provides; the FP64
//                     CG kernels this entry point runs use the first six)
//   control words     32 doubles' worth: the grid barrier's four words (two
//                     doubles), the status words, the flags
constexpr int kMaxBlocks = 1024;
constexpr long long kVec = ESDC_STATIC_MAX_NODES;
constexpr long long kDoubles = 4 * kVec + 8LL * kMaxBlocks + 32;
static_assert(kDoubles * 8 == ESDC_STATIC_SCRATCH_BYTES, "ESDC_STATIC_SCRATCH_BYTES (esdc.h) states the array's size");

static __device__ __align__(256) double g_static_scratch[kDoubles];

std::mutex g_mu;
double* g_addr[64] = {nullptr};      // device address of g_static_scratch, per device

// Device address of the array on the current device.  In host code the name
// g_static_scratch is only a host-side stand-in, never a device address, so
// the address is looked up once per device with that device current.
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int esdc_diffusion_solve_static(const esdc_mesh* mesh, double g, const double* b, double* x,
                                           double tol, int maxit, int precond, int* iters, void* stream)
{
    if (!mesh || !b || !x) return ESDC_ERR_INVALID_ARG;
    if (mesh->dim < 1 || mesh->dim > 3 || mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->h > 0.0))
        return ESDC_ERR_INVALID_ARG;
    if ((mesh->dim < 3 && mesh->nz != 1) || (mesh->dim < 2 && mesh->ny != 1)) return ESDC_ERR_INVALID_ARG;
    if (!(g >= 0.0) || !(tol >= 0.0) || maxit < 1) return ESDC_ERR_INVALID_ARG;
    const long long N = (long long)mesh->nx * mesh->ny * mesh->nz;
    if (N > ESDC_STATIC_MAX_NODES) return ESDC_ERR_TOO_LARGE;

    double* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return ESDC_ERR_CUDA;

    MeshDev m{};                                  // scalar conductivity only
    m.nx = mesh->nx; m.ny = mesh->ny; m.nz = mesh->nz;
    m.N = (int)N;
    m.ld = N;
    m.ih2 = 1.0 / (mesh->h * mesh->h);

    CgWork w{};
    w.r = base;
    w.p = base + kVec;
    w.q = base + 2 * kVec;
    w.z = base + 3 * kVec;
    w.part = base + 4 * kVec;
    double* ctl = base + 4 * kVec + 8LL * kMaxBlocks;
    w.bar = reinterpret_cast<unsigned*>(ctl);              // [4]: barrier counter, spare, test words (zero)
    w.status = reinterpret_cast<int*>(ctl + 2);            // [0] iterations, [1] spare
    int* flags = reinterpret_cast<int*>(ctl + 3);          // error flags
    w.threads = ESDC_CG_THREADS;
    w.max_blocks = esdc_cg_blocks(m, w.threads);
    if (w.max_blocks < 1) return ESDC_ERR_CUDA;
    if (w.max_blocks > kMaxBlocks) w.max_blocks = kMaxBlocks;

    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps the previous call's contents: clear the control words
    // (barrier, status, flags), so that a solve that stops early reports no
    // stale iteration count.  The CG vectors and partial sums are fully written
    // before they are read.
    if (cudaMemsetAsync(ctl, 0, 4 * sizeof(double), s) != cudaSuccess) return ESDC_ERR_CUDA;
    if (esdc_cg_launch(m, w, g, b, x, tol, maxit, precond != 0, 1, nullptr, flags, s) != cudaSuccess)
        return ESDC_ERR_CUDA;
    int st[2] = {0, 0}, fl = 0;
    if (cudaMemcpyAsync(st, w.status, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&fl, flags, sizeof fl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ESDC_ERR_CUDA;
    if (iters) *iters = st[0];
    if (fl & ESDC_FLAG_TIMEOUT) return ESDC_ERR_DEVICE_TIMEOUT;
    if (fl & ESDC_FLAG_NONFINITE) return ESDC_ERR_NONFINITE;
    if (fl & ESDC_FLAG_CG_MAXIT) return ESDC_ERR_CG_NOT_CONVERGED;
    return ESDC_OK;
}
