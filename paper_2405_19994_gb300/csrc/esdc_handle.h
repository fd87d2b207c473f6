// Internal: the handle and the per-launch argument block shared by the
// translation units of the step (FP64 and precision-form instantiations).
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "esdc_internal.h"

struct StepArgs {
    MeshDev m;
    StimDev st;
    ModelDev mp;
    ModelDevF mpf;         // FP32 parameters (precision form)
    int i;                 // collocation node 1..M (k_node), M+1: evaluate G at node M only
    int k;                 // sweep index (0-based)
    int fuse1;             // k_setup, and k_node at i = M+1 (M >= 2): also node 1 of the next sweep
    double rho;            // warm-start extrapolation weight for node i
    double* Vprev;         // [ld] V_{i-1}^k, saved before node i-1 was solved
    double dt, t_n, D, inv_Cm;
    double dS0[ESDC_MMAX][ESDC_MMAX];   // dt * (a_ij(0) - a_{i-1,j}(0))
    double dtB[ESDC_MMAX][ESDC_MMAX][ESDC_MMAX];   // dt * B_ijk (set-up: dt a_ij = sum_k dt B_ijk phi_k)
    const double* ztab;                 // set-up coefficient table for (M, dt) (esdc_ztab.cpp), or nullptr
    double dtd[ESDC_MMAX + 1];          // dt * d_i
    unsigned stim_on[ESDC_MMAX + 1];    // boxes active at t_{n,j}, j = 0..M (bit b = box b)
    const double* yn;
    double* yout;          // residual kernel: destination of y_{n+1}
    double* Y;
    const double* Gold;
    double* Gnew;
    double* FI;
    double* S;
    double* PHI;
    double* LAMN;
    double* rhs;
    double* R;             // residual vectors (optional)
    unsigned long long* rmax;   // [NS] per-state max |r| (as ordered bits), [NS] max |y|
    int* flags;
    // ragged batches (batched kernels only)
    const TissueDev* tis;
    const int* tile_tissue;     // [tiles] tissue of each tile
    const unsigned* tis_on;     // [tissues][ESDC_MMAX + 1] stimulus window bits per collocation time
    const double* tau;          // FAS correction [M][NS][ld] (batched kernels; nullptr: none)
};

struct esdc_handle {
    int device = 0, sms = 152;
    int model = 0, NS = 0, NA = 0, NG = 0;
    ColloData col[ESDC_MMAX];
    MeshDev mesh{};
    StimDev stim{};
    ModelDev mp{};
    ModelDevF mpf{};
    double sigma = 0, chi = 0, Cm = 0, D = 0;
    double* vtab = nullptr;                    // the gate table of the model (SYN19), see ModelDev
    ZtabSlots zt;                              // set-up coefficient tables per (M, dt)
    double vtab_err[2] = {0, 0};               // its build-time errors (b / |Lambda| absolute, Lambda relative)
    double *lay = nullptr, *wdiag = nullptr;   // layered conductivity (see MeshDev)
    double* sigf = nullptr;                    // conductivity field (see MeshDev)
    float* layf = nullptr;
    esdc_options opt{};
    // workspace
    double *Y = nullptr, *G0 = nullptr, *G1 = nullptr, *FI = nullptr, *S = nullptr, *PHI = nullptr,
           *LAMN = nullptr, *rhs = nullptr, *R = nullptr, *ydev = nullptr, *Vprev = nullptr;
    CgWork cg{};
    DctDev dct{};                         // options.solver = 2
    // adjoint recording (set only inside esdc_adjoint_backward): Y^{1..K},
    // G^{0..K}, FI^{0..K} of one step, each block [M][NS][ld] or [M][ld]
    double *tapeY = nullptr, *tapeG = nullptr, *tapeFI = nullptr;
    unsigned long long* rmax = nullptr;   // [2*NS]
    int* flags = nullptr;                 // [1]
    int* cg_log = nullptr;                // [K_log] iteration counts of the last step
    int cg_log_len = 0;
    // state of the most recent sweep
    int last_M = 0, last_K = 0;
    double last_dt = 0.0;
    const double* last_Gfinal = nullptr;
    cudaStream_t last_stream = nullptr;
    // kernel-class timing (esdc_profile): event pairs around each launch
    bool prof_on = false;
    cudaEvent_t prof_ev[2 * 512] = {};
    int prof_cls[512] = {};
    int prof_used = 0;
    double prof_ms[ESDC_PROF_CLASSES] = {};
    long long prof_cnt[ESDC_PROF_CLASSES] = {};
    char err[256] = {0};
};
// (Re)builds the handle's gate table for its current parameters (esdc_step.cu).
cudaError_t esdc_vtab_upload(esdc_handle* h);



// Records a formatted message on the handle and returns code.
__attribute__((format(printf, 3, 4))) inline int set_err(esdc_handle* h, int code, const char* fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CUDA_TRY(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_err((h), e_ == cudaErrorMemoryAllocation ? ESDC_ERR_NO_MEMORY : ESDC_ERR_CUDA, \
                           "%s: %s", #call, cudaGetErrorString(e_));                           \
    } while (0)

// Kernel-class timing (esdc_profile).
// Folds the recorded event pairs into the per-class totals (synchronises them).
inline cudaError_t prof_flush(esdc_handle* h)
{
    for (int k = 0; k < h->prof_used; ++k) {
        cudaError_t e = cudaEventSynchronize(h->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return e;
        h->prof_ms[h->prof_cls[k]] += ms;
        h->prof_cnt[h->prof_cls[k]] += 1;
    }
    h->prof_used = 0;
    return cudaSuccess;
}

inline void prof_begin(esdc_handle* h, int cls, cudaStream_t s)
{
    if (!h->prof_on) return;
    if (h->prof_used == 512) prof_flush(h);
    h->prof_cls[h->prof_used] = cls;
    cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
}

inline void prof_end(esdc_handle* h, cudaStream_t s)
{
    if (!h->prof_on) return;
    cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
    h->prof_used++;
}


// Launches one HSDC step of the precision form (defined in esdc_step_mixed.cu).
cudaError_t esdc_dispatch_mixed(esdc_handle* h, StepArgs& a, double* y, int M, int K, cudaStream_t s);
