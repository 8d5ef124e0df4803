// Whole analysis of a small problem in one CTA (the latency-bound Lorenz-96 case):
// Step 1 (eq. SM-step-1), the levels of Step 2 (eqs. SM-step-2-h/Z/u), M = V^T Z /
// sqrt(Nens - 1) and X_A = X_B + dX_B M (Sec. 3.1), with V, U and Z resident in shared
// memory for the whole solve.  One launch per analysis; no grid barrier, no workspace
// traffic beyond the status word and gamma.
//
// The dots of a level are formed by groups of 8 lanes (each lane sums every 8th row in
// ascending order, then a fixed xor butterfly), 32 dots per pass of 256 threads, and the
// updates by one thread per element.  In FP64 the cost is set by GB300's narrow FP64 pipe
// (about 1.7 FMA per clock per SM): 4 Nobs Nens^2 + 2 Nstate Nens^2 FMAs in all.
#include <math.h>

#include "internal.h"

namespace enkf {
namespace {

constexpr int kST = 256;     // threads
constexpr int kG = 8;        // lanes per dot

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ double tol_gamma();
template <>
__device__ __forceinline__ double tol_gamma<float>() { return 64.0 * 1.1920928955078125e-07; }
template <>
__device__ __forceinline__ double tol_gamma<double>() { return 64.0 * 2.220446049250313e-16; }

template <typename T>
__global__ void __launch_bounds__(kST) small_analysis_kernel(SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.nobs, N = a.nens, tid = threadIdx.x;
    const int ld = n;                                  // column stride of the resident arrays
    T* sV = reinterpret_cast<T*>(smem_raw);            // [N][n]
    T* sU = sV + (size_t)N * ld;                       // [N][n]
    T* sZ = sU + (size_t)N * ld;                       // [N][n]
    T* sh = sZ + (size_t)N * ld;                       // [n]  r, then h_k
    T* cf = sh + n;                                    // [2N] level dots; [2N] = 1 / gamma_k
    T* sM = cf + 2 * N + 2;                            // [N][N] M, column-major (k + e N)
    const T* r = static_cast<const T*>(a.r);
    const T* V = static_cast<const T*>(a.V);
    const T* D = static_cast<const T*>(a.D);

    // ---- Step 1: U = R^-1 V, Z = R^-1 D (divisions, as the equation reads)
    for (int j = tid; j < n; j += kST) {
        const T rj = r[j];
        if (a.check && !(rj > T(0) && isfinite(rj))) {
            set_status(a.ctl, kErrNumeric);
            a.ctl->fail_level = 0;
        }
        sh[j] = rj;
    }
    __syncthreads();
    for (int e = tid; e < N * n; e += kST) {
        const int c = e / n, j = e - c * n;
        const T v = V[(int64_t)c * a.ldv + j];
        const T d = D[(int64_t)c * a.ldd + j];
        if (a.check && !(isfinite(v) && isfinite(d))) {
            set_status(a.ctl, kErrNumeric);
            a.ctl->fail_level = 0;
        }
        sV[c * ld + j] = v;
        sU[c * ld + j] = v / sh[j];
        sZ[c * ld + j] = d / sh[j];
    }
    __syncthreads();

    // ---- Step 2: levels k = 0 .. N-1; the dots of level k are with v_k: every z_i (i < N)
    // and u_i for i >= k (i = k gives gamma_k - 1)
    const int grp = tid / kG, gl = tid % kG, ngrp = kST / kG;
    for (int k = 0; k < N; ++k) {
        const T* vk = sV + k * ld;
        const int ndots = N + (N - k);
        for (int d0 = 0; d0 < ndots; d0 += ngrp) {
            const int d = d0 + grp;
            T acc = T(0);
            if (d < ndots) {
                const T* x = d < N ? sZ + d * ld : sU + (k + d - N) * ld;
                for (int j = gl; j < n; j += kG) acc = fma(vk[j], x[j], acc);
            }
            acc = group_sum(acc);
            if (d < ndots && gl == 0) cf[d] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            // gamma_k and its reciprocal by one thread (one FP64 division per level)
            const T gam = T(1) + cf[N];
            cf[2 * N] = T(1) / gam;
            a.gamma[k] = (double)gam;
            if (a.check && (!(gam >= T(1) - (T)tol_gamma<T>() * (T(1) + fabs(gam - T(1)))) || !isfinite(gam))) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = k + 1;
            }
        }
        __syncthreads();
        // h_k = u_k / gamma_k
        const T ginv = cf[2 * N];
        for (int j = tid; j < n; j += kST) sh[j] = sU[k * ld + j] * ginv;
        __syncthreads();
        // x <- x - h_k c_x for every z_i and every u_i, i > k
        const int nupd = N + (N - 1 - k);
        for (int e = tid; e < nupd * n; e += kST) {
            const int c = e / n, j = e - c * n;
            T* x = c < N ? sZ + c * ld : sU + (k + 1 + c - N) * ld;
            const T ci = c < N ? cf[c] : cf[N + 1 + (c - N)];
            x[j] = fma(-sh[j], ci, x[j]);
        }
        __syncthreads();
    }

    // ---- Z out, M = V^T Z / sqrt(N - 1), X_A = X_B + dX_B M
    if (a.Z) {
        T* Zo = static_cast<T*>(a.Z);
        for (int e = tid; e < N * n; e += kST) {
            const int c = e / n, j = e - c * n;
            Zo[(int64_t)c * a.ldz + j] = sZ[c * ld + j];
        }
    }
    if (N >= 2 && (a.M || a.dXB)) {
        const T scale = T(1) / sqrt(T(N - 1));
        for (int d0 = 0; d0 < N * N; d0 += ngrp) {
            const int d = d0 + grp;            // entry (kk, e), kk fastest
            T acc = T(0);
            if (d < N * N) {
                const int kk = d % N, e = d / N;
                for (int j = gl; j < n; j += kG) acc = fma(sV[kk * ld + j], sZ[e * ld + j], acc);
            }
            acc = group_sum(acc);
            if (d < N * N && gl == 0) sM[d] = acc * scale;
        }
        __syncthreads();
        if (a.M) {
            T* Mo = static_cast<T*>(a.M);
            for (int e = tid; e < N * N; e += kST) Mo[e] = sM[e];
        }
        if (a.dXB) {
            const T* dX = static_cast<const T*>(a.dXB);
            const T* XB = static_cast<const T*>(a.XB);
            T* XA = static_cast<T*>(a.XA);
            for (int64_t q = tid; q < a.nstate * N; q += kST) {
                const int e = (int)(q / a.nstate);
                const int64_t i = q - (int64_t)e * a.nstate;
                T acc = XB[(int64_t)e * a.ldb + i];
                for (int kk = 0; kk < N; ++kk) acc = fma(dX[(int64_t)kk * a.ldx + i], sM[kk + e * N], acc);
                XA[(int64_t)e * a.lda + i] = acc;
            }
        }
    }
}

template <typename T>
size_t smem_bytes(int64_t nobs, int32_t nens) {
    return sizeof(T) * ((size_t)3 * nens * nobs + nobs + 2 * (size_t)nens + 2 + (size_t)nens * nens);
}

}  // namespace

bool small_fits(bool fp64, int64_t nobs, int32_t nens) {
    const size_t b = fp64 ? smem_bytes<double>(nobs, nens) : smem_bytes<float>(nobs, nens);
    return nobs >= 1 && nens >= 1 && nobs * (int64_t)nens <= 4096 && b <= 100 * 1024;
}

cudaError_t small_launch(bool fp64, const SmallArgs& a, cudaStream_t s) {
    const size_t smem = fp64 ? smem_bytes<double>(a.nobs, a.nens) : smem_bytes<float>(a.nobs, a.nens);
    const void* fn = fp64 ? (const void*)small_analysis_kernel<double> : (const void*)small_analysis_kernel<float>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (fp64)
        small_analysis_kernel<double><<<1, kST, smem, s>>>(a);
    else
        small_analysis_kernel<float><<<1, kST, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enkf
