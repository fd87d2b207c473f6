// The precision form of the HSDC step: the same kernels as esdc_step.cu with
// the ionic model evaluated in FP32 (MIXED = true).  A separate translation
// unit, so that the two sets of instantiations compile in parallel.
#include <mutex>

#include "esdc_kernels.cuh"

namespace {
std::mutex g_mu;
bool g_done[64] = {false};
}  // namespace

cudaError_t esdc_dispatch_mixed(esdc_handle* h, StepArgs& a, double* y, int M, int K, cudaStream_t s)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaError_t e = upload_constants_local(g_done, h->device);
        if (e != cudaSuccess) return e;
    }
    return h->model == ESDC_MODEL_HH1952 ? dispatch_M<esdc::HH1952, true>(h, a, y, M, K, s)
                                         : dispatch_M<esdc::SYN19, true>(h, a, y, M, K, s);
}
