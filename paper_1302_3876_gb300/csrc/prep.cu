// Observation-space preparation of the SMEnKF (Sec. 2 and Sec. 3):
//   xbar = X_B 1 / Nens                      (eq. ensemble-background-mean)
//   dX_B = X_B - xbar 1^T                    (numerator of eq. EnSM:Matrix-member-deviations)
//   V    = H dX_B / sqrt(Nens - 1)           (eq. EnKSM:member-observations)
//   D    = Y - H X_B                         (eq. EnKSM:system-rhs)
// with H selecting state rows 0, stride, 2 stride, ...  One thread per state row
// (centering pass) or per observation row; member loops are coalesced across
// threads because consecutive threads own consecutive rows of every column.
#include <math.h>

#include "internal.h"

namespace enkf {
namespace {

template <typename T>
__global__ void center_observe_kernel(int64_t nstate, int64_t nobs, int n, int stride, const T* __restrict__ XB,
                                      int64_t ldb, T* __restrict__ dXB, int64_t ldx, const T* __restrict__ Y,
                                      int64_t ldy, T* __restrict__ V, int64_t ldv, T* __restrict__ D, int64_t ldd,
                                      double scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nstate;
         i += (int64_t)gridDim.x * blockDim.x) {
        // unrolled so that several member loads are in flight (a small problem is bound by
        // their latency); the sum runs in member order
        double s = 0.0;
#pragma unroll 8
        for (int e = 0; e < n; ++e) s += (double)XB[(int64_t)e * ldb + i];
        const double mean = s / (double)n;
        const bool observed = (i % stride == 0) && (i / stride < nobs);
        const int64_t j = i / stride;
#pragma unroll 8
        for (int e = 0; e < n; ++e) {
            const T x = XB[(int64_t)e * ldb + i];
            const T d = (T)((double)x - mean);
            dXB[(int64_t)e * ldx + i] = d;
            if (observed) {
                V[(int64_t)e * ldv + j] = (T)((double)d * scale);
                if (Y) D[(int64_t)e * ldd + j] = Y[(int64_t)e * ldy + j] - x;
            }
        }
    }
}

// One member column per blockIdx.y; each thread takes kObsU observations kObsT apart, so
// that kObsU independent strided loads are in flight per thread (a strided gather reads
// every DRAM sector of the rows it spans and is bound by the loads in flight).
constexpr int kObsT = 256, kObsU = 8;

template <typename T>
__global__ void __launch_bounds__(kObsT) observe_kernel(int64_t nobs, int n, int stride, const T* __restrict__ XB,
                                                        int64_t ldb, const T* __restrict__ dXB, int64_t ldx,
                                                        const T* __restrict__ Y, int64_t ldy, T* __restrict__ V,
                                                        int64_t ldv, T* __restrict__ D, int64_t ldd, double scale) {
    const int e = blockIdx.y;
    const T* dx = dXB + (int64_t)e * ldx;
    for (int64_t j0 = blockIdx.x * (int64_t)(kObsT * kObsU) + threadIdx.x; j0 < nobs;
         j0 += (int64_t)gridDim.x * (kObsT * kObsU)) {
        T d[kObsU];
#pragma unroll
        for (int u = 0; u < kObsU; ++u) {
            const int64_t j = j0 + (int64_t)u * kObsT;
            d[u] = j < nobs ? __ldcs(dx + j * stride) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kObsU; ++u) {
            const int64_t j = j0 + (int64_t)u * kObsT;
            if (j >= nobs) break;
            // FP32 storage scales in FP32 (one extra rounding of 1/sqrt(N-1)): FP64 arithmetic per
            // element would run on GB300's narrow FP64 pipe
            if (sizeof(T) == 4)
                V[(int64_t)e * ldv + j] = d[u] * (T)scale;
            else
                V[(int64_t)e * ldv + j] = (T)((double)d[u] * scale);
            if (Y) D[(int64_t)e * ldd + j] = Y[(int64_t)e * ldy + j] - XB[(int64_t)e * ldb + j * stride];
        }
    }
}

}  // namespace

cudaError_t obs_prep(bool fp64, int64_t nstate, int64_t nobs, int32_t nens, int32_t stride, int32_t center,
                     const void* XB, int64_t ldb, void* dXB, int64_t ldx, const void* Y, int64_t ldy, void* V,
                     int64_t ldv, void* D, int64_t ldd, cudaStream_t s) {
    const double scale = 1.0 / sqrt((double)(nens - 1));
    if (center) {
        const int blocks = (int)((nstate + 255) / 256);
        if (fp64)
            center_observe_kernel<double><<<blocks, 256, 0, s>>>(nstate, nobs, nens, stride, (const double*)XB, ldb,
                                                                 (double*)dXB, ldx, (const double*)Y, ldy, (double*)V,
                                                                 ldv, (double*)D, ldd, scale);
        else
            center_observe_kernel<float><<<blocks, 256, 0, s>>>(nstate, nobs, nens, stride, (const float*)XB, ldb,
                                                                (float*)dXB, ldx, (const float*)Y, ldy, (float*)V, ldv,
                                                                (float*)D, ldd, scale);
    } else {
        int64_t bx = (nobs + kObsT * kObsU - 1) / (kObsT * kObsU);
        if (bx > 4096) bx = 4096;
        dim3 grid((unsigned)bx, (unsigned)nens);
        if (fp64)
            observe_kernel<double><<<grid, kObsT, 0, s>>>(nobs, nens, stride, (const double*)XB, ldb, (const double*)dXB,
                                                        ldx, (const double*)Y, ldy, (double*)V, ldv, (double*)D, ldd,
                                                        scale);
        else
            observe_kernel<float><<<grid, kObsT, 0, s>>>(nobs, nens, stride, (const float*)XB, ldb, (const float*)dXB, ldx,
                                                       (const float*)Y, ldy, (float*)V, ldv, (float*)D, ldd, scale);
    }
    return cudaGetLastError();
}

}  // namespace enkf
