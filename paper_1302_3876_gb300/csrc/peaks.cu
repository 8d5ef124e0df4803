// CUDA-core multiply-add throughput of this GPU, FP32 and FP64: the denominators
// of the ALU rooflines (the FP32 panel sweeps, the on-chip batch, the plain FP64
// path).  Each thread runs kChains independent multiply-add chains of `iters`
// steps in registers, so the count of issued FMAs is known exactly and nothing
// but the FMA pipe is exercised; the caller times the launch with CUDA events.
#include <cuda_runtime.h>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace enkf {
namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T mul, T add, T* sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], mul, add);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    // the chains converge to add / (1 - mul) > 0; the store never happens but the
    // compiler cannot prove it, so the chains are kept
    if (s < (T)-1) *sink = s;
}

enkf_status peak_fail(enkf_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

}  // namespace
}  // namespace enkf

extern "C" enkf_status enkf_fma_peak_launch(int32_t precision, int32_t iters, int32_t ctas_per_sm, void* sink,
                                           void* stream, double* flops) {
    using namespace enkf;
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return peak_fail(ENKF_ERR_ARG, "enkf_fma_peak_launch: precision must be ENKF_FP64 or ENKF_FP32");
    if (iters < 1 || ctas_per_sm < 1 || ctas_per_sm > 8 || !sink || !flops)
        return peak_fail(ENKF_ERR_ARG, "enkf_fma_peak_launch: bad iters, ctas_per_sm, sink or flops");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return peak_fail(ENKF_ERR_CUDA, "enkf_fma_peak_launch: device query failed");
    const int grid = sms * ctas_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == ENKF_FP32)
        fma_chain_kernel<float><<<grid, kThreads, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink);
    else
        fma_chain_kernel<double><<<grid, kThreads, 0, s>>>(iters, 0.999, 1e-3, (double*)sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) return peak_fail(ENKF_ERR_CUDA, cudaGetErrorString(e));
    *flops = 2.0 * (double)grid * kThreads * kChains * (double)iters;
    return ENKF_OK;
}
