// Block-diagonal observation-error covariance R = diag(R_1, ..., R_nblk) (Sec. 3.1:
// R^{-1} is applied block by block in Step 1), with the C-ABI entry points
// enkf_rblock_factor, enkf_rblock_whiten and enkf_rblock_unwhiten (declared in
// include/enkf_ism.h).
//
// The analysis kernels take a diagonal R.  A block-diagonal R reaches them through
// its block Cholesky factor R = L L^T:
//   (R + V V^T) Z = D   <=>   (I + V~ V~^T) Z~ = D~,  V~ = L^{-1} V,  D~ = L^{-1} D,  Z = L^{-T} Z~.
// Every level of the recurrence maps one to one (u_k = L^{-T} u~_k, h_k = L^{-T} h~_k,
// gamma_k = 1 + v~_k^T u~_k is unchanged), and V^T Z = V~^T Z~, so M and X_A come out
// of the unchanged analysis run on (r = 1, V~, D~).
//
// enkf_rblock_factor: one warp per block, right-looking Cholesky in shared memory
// (FP64), lane q owning row q.  enkf_rblock_whiten / enkf_rblock_unwhiten: one lane per
// column of a block, forward (L y = b) or backward (L^T x = y) substitution in
// registers with the factor and its reciprocal diagonal broadcast from shared memory,
// in the storage precision (FP32 or FP64).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace enkf {
namespace {

constexpr int kRbMax = 32;        // largest block
constexpr int kRbPitch = kRbMax + 1;
constexpr int kFactorWarps = 4;
constexpr int kSolveWarps = 8;

enkf_status rfail(enkf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

enkf_status rcuda(cudaError_t e, const char* what) {
    return rfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

__global__ void __launch_bounds__(kFactorWarps * 32) rblock_factor_kernel(int64_t nobs, int bs, int64_t nblk,
                                                                          const double* __restrict__ R,
                                                                          double* __restrict__ L) {
    __shared__ double As[kFactorWarps][kRbMax * kRbPitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * kFactorWarps + warp;
    if (b >= nblk) return;
    const int64_t r0 = b * bs;
    const int m = (int)((nobs - r0) < bs ? (nobs - r0) : bs);
    const double* Rb = R + b * (int64_t)bs * bs;
    double* Lb = L + b * (int64_t)bs * bs;
    double* A = As[warp];                                  // A[row * pitch + col], lower triangle used
    for (int c = 0; c < m; ++c) A[lane * kRbPitch + c] = lane < m ? Rb[(int64_t)c * bs + lane] : 0.0;
    __syncwarp();
    bool ok = true;
    for (int c = 0; c < m; ++c) {
        const double d = A[c * kRbPitch + c];
        if (!(d > 0.0) || !isfinite(d)) ok = false;
        const double lcc = sqrt(d);
        __syncwarp();
        if (lane == c) A[c * kRbPitch + c] = lcc;
        if (lane > c && lane < m) A[lane * kRbPitch + c] /= lcc;
        __syncwarp();
        if (lane > c && lane < m) {
            const double lqc = A[lane * kRbPitch + c];
            for (int s = c + 1; s <= lane; ++s) A[lane * kRbPitch + s] -= lqc * A[s * kRbPitch + c];
        }
        __syncwarp();
    }
    // a block that is not positive definite yields NaN factors: the whitened rows become NaN and
    // the analysis reports them through its finiteness checks
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int c = 0; c < bs; ++c)
        if (lane < bs) Lb[(int64_t)c * bs + lane] = !ok ? nan : (lane >= c && lane < m && c < m) ? A[lane * kRbPitch + c] : 0.0;
}

// blockIdx.x = block of R; warp w of CTA blockIdx.y owns columns (blockIdx.y * kSolveWarps + w) * 32 + lane
// (first ncol0 of A0, then A1), one column per lane.  A warp stages its 32 columns of the block
// through shared memory (column loads are contiguous runs of the block's rows), substitutes in
// registers with L and the reciprocal diagonal broadcast from shared memory, and stores back the
// same way.  Arithmetic in the storage type (FP32 or FP64); the factors are FP64 in memory.
template <typename T>
constexpr int solve_warps() { return sizeof(T) == 8 ? kSolveWarps / 2 : kSolveWarps; }   // static smem <= 48 KB

template <typename T, bool kForward>
__global__ void __launch_bounds__(solve_warps<T>() * 32) rblock_solve_kernel(int64_t nobs, int bs,
                                                                        const double* __restrict__ L, T* A0,
                                                                        int64_t ld0, int ncol0, T* A1, int64_t ld1,
                                                                        int ncol1) {
    __shared__ T Ls[kRbMax * kRbPitch];                    // Ls[row * pitch + col], zero outside m x m
    __shared__ T inv[kRbMax];
    constexpr int W = solve_warps<T>();
    __shared__ T tile[W][32 * kRbPitch];                   // tile[column * pitch + row]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.x;
    const int64_t r0 = b * bs;
    const int m = (int)((nobs - r0) < bs ? (nobs - r0) : bs);
    const double* Lb = L + b * (int64_t)bs * bs;
    for (int idx = threadIdx.x; idx < kRbMax * kRbMax; idx += W * 32) {
        const int row = idx % kRbMax, col = idx / kRbMax;
        Ls[row * kRbPitch + col] = (row < m && col < m) ? (T)Lb[(int64_t)col * bs + row] : T(0);
    }
    if (threadIdx.x < kRbMax) inv[threadIdx.x] = threadIdx.x < m ? (T)(1.0 / Lb[(int64_t)threadIdx.x * bs + threadIdx.x]) : T(0);
    __syncthreads();
    const int ncol = ncol0 + ncol1;
    const int cbase = (blockIdx.y * W + warp) * 32;
    if (cbase >= ncol) return;
    T* tw = tile[warp];
    // stage: column cc of the warp, rows r0 .. r0 + m - 1 (lane = row)
    for (int cc = 0; cc < 32; ++cc) {
        const int col = cbase + cc;
        T v = T(0);
        if (col < ncol && lane < m) {
            const T* x = col < ncol0 ? A0 + (int64_t)col * ld0 : A1 + (int64_t)(col - ncol0) * ld1;
            v = x[r0 + lane];
        }
        tw[cc * kRbPitch + lane] = v;
    }
    __syncwarp();
    T y[kRbMax];
    if (kForward) {
#pragma unroll
        for (int c = 0; c < kRbMax; ++c) {
            T acc = tw[lane * kRbPitch + c];
#pragma unroll
            for (int p = 0; p < c; ++p) acc -= Ls[c * kRbPitch + p] * y[p];
            y[c] = acc * inv[c];                           // rows >= m: L and inv are zero, y = 0
        }
    } else {
#pragma unroll
        for (int c = kRbMax - 1; c >= 0; --c) {
            T acc = tw[lane * kRbPitch + c];
#pragma unroll
            for (int p = c + 1; p < kRbMax; ++p) acc -= Ls[p * kRbPitch + c] * y[p];
            y[c] = acc * inv[c];
        }
    }
#pragma unroll
    for (int c = 0; c < kRbMax; ++c) tw[lane * kRbPitch + c] = y[c];
    __syncwarp();
    for (int cc = 0; cc < 32; ++cc) {
        const int col = cbase + cc;
        if (col < ncol && lane < m) {
            T* x = col < ncol0 ? A0 + (int64_t)col * ld0 : A1 + (int64_t)(col - ncol0) * ld1;
            x[r0 + lane] = tw[cc * kRbPitch + lane];
        }
    }
}

template <bool kForward>
cudaError_t rblock_solve(bool fp64, int64_t nobs, int bs, const double* L, void* A0, int64_t ld0, int ncol0, void* A1,
                         int64_t ld1, int ncol1, cudaStream_t s) {
    const int64_t nblk = (nobs + bs - 1) / bs;
    const int cols = ncol0 + ncol1;
    if (fp64) {
        constexpr int W = solve_warps<double>();
        dim3 grid((unsigned)nblk, (unsigned)((cols + 32 * W - 1) / (32 * W)));
        rblock_solve_kernel<double, kForward><<<grid, W * 32, 0, s>>>(nobs, bs, L, (double*)A0, ld0, ncol0,
                                                                     (double*)A1, ld1, ncol1);
    } else {
        constexpr int W = solve_warps<float>();
        dim3 grid((unsigned)nblk, (unsigned)((cols + 32 * W - 1) / (32 * W)));
        rblock_solve_kernel<float, kForward><<<grid, W * 32, 0, s>>>(nobs, bs, L, (float*)A0, ld0, ncol0,
                                                                    (float*)A1, ld1, ncol1);
    }
    return cudaGetLastError();
}

enkf_status check_sizes(const char* who, int64_t nobs, int32_t bs) {
    if (nobs < 1 || bs < 1 || bs > kRbMax) return rfail(ENKF_ERR_SHAPE, "%s: need nobs >= 1 and 1 <= bs <= %d", who, kRbMax);
    if ((nobs + bs - 1) / bs > 0x7fffffffll) return rfail(ENKF_ERR_SHAPE, "%s: too many blocks", who);
    return ENKF_OK;
}

}  // namespace
}  // namespace enkf

using namespace enkf;

extern "C" enkf_status enkf_rblock_factor(int64_t nobs, int32_t bs, const double* Rblk, double* Lblk, void* stream) {
    if (!Rblk || !Lblk) return rfail(ENKF_ERR_ARG, "enkf_rblock_factor: NULL Rblk or Lblk");
    enkf_status st = check_sizes("enkf_rblock_factor", nobs, bs);
    if (st != ENKF_OK) return st;
    const int64_t nblk = (nobs + bs - 1) / bs;
    const size_t bytes = sizeof(double) * (size_t)nblk * bs * bs;
    const char *pr = (const char*)Rblk, *pl = (const char*)Lblk;
    if (pr < pl + bytes && pl < pr + bytes) return rfail(ENKF_ERR_ARG, "enkf_rblock_factor: Rblk and Lblk overlap");
    if (((uintptr_t)Rblk | (uintptr_t)Lblk) & 7) return rfail(ENKF_ERR_ARG, "enkf_rblock_factor: unaligned pointer");
    const int64_t grid = (nblk + kFactorWarps - 1) / kFactorWarps;
    rblock_factor_kernel<<<(unsigned)grid, kFactorWarps * 32, 0, (cudaStream_t)stream>>>(nobs, bs, nblk, Rblk, Lblk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rcuda(e, "enkf_rblock_factor: launch");
    return ENKF_OK;
}

extern "C" enkf_status enkf_rblock_whiten(int64_t nobs, int32_t nens, int32_t precision, int32_t bs,
                                          const double* Lblk, void* V, int64_t ldv, void* D, int64_t ldd,
                                          void* stream) {
    if (!Lblk || !V) return rfail(ENKF_ERR_ARG, "enkf_rblock_whiten: NULL Lblk or V");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return rfail(ENKF_ERR_ARG, "enkf_rblock_whiten: precision must be ENKF_FP64 or ENKF_FP32");
    enkf_status st = check_sizes("enkf_rblock_whiten", nobs, bs);
    if (st != ENKF_OK) return st;
    if (nens < 1 || nens > 65535 * 16) return rfail(ENKF_ERR_SHAPE, "enkf_rblock_whiten: bad nens");
    if (ldv < nobs || (D && ldd < nobs)) return rfail(ENKF_ERR_SHAPE, "enkf_rblock_whiten: ld smaller than nobs");
    const uintptr_t wmask = precision == ENKF_FP64 ? 7 : 3;
    if ((((uintptr_t)V | (uintptr_t)D) & wmask) || ((uintptr_t)Lblk & 7))
        return rfail(ENKF_ERR_ARG, "enkf_rblock_whiten: pointer not aligned to the element size");
    cudaError_t e = rblock_solve<true>(precision == ENKF_FP64, nobs, bs, Lblk, V, ldv, nens, D, ldd, D ? nens : 0,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return rcuda(e, "enkf_rblock_whiten: launch");
    return ENKF_OK;
}

extern "C" enkf_status enkf_rblock_unwhiten(int64_t nobs, int32_t ncols, int32_t precision, int32_t bs,
                                            const double* Lblk, void* Z, int64_t ldz, void* stream) {
    if (!Lblk || !Z) return rfail(ENKF_ERR_ARG, "enkf_rblock_unwhiten: NULL Lblk or Z");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return rfail(ENKF_ERR_ARG, "enkf_rblock_unwhiten: precision must be ENKF_FP64 or ENKF_FP32");
    enkf_status st = check_sizes("enkf_rblock_unwhiten", nobs, bs);
    if (st != ENKF_OK) return st;
    if (ncols < 1 || ncols > 65535 * 32) return rfail(ENKF_ERR_SHAPE, "enkf_rblock_unwhiten: bad ncols");
    if (ldz < nobs) return rfail(ENKF_ERR_SHAPE, "enkf_rblock_unwhiten: ldz smaller than nobs");
    if (((uintptr_t)Z & (precision == ENKF_FP64 ? 7 : 3)) || ((uintptr_t)Lblk & 7))
        return rfail(ENKF_ERR_ARG, "enkf_rblock_unwhiten: pointer not aligned to the element size");
    cudaError_t e = rblock_solve<false>(precision == ENKF_FP64, nobs, bs, Lblk, Z, ldz, ncols, nullptr, 0, 0,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return rcuda(e, "enkf_rblock_unwhiten: launch");
    return ENKF_OK;
}
