// Analysis assembly of the SMEnKF (Sec. 3.1): M = V^T Z / sqrt(Nens - 1) and
// X_A = X_B + dX_B M.
//
// M is assembled from the recurrence's own quantities rather than from a direct
// product V^T Z, which cancels catastrophically when gamma_k >> 1 (the part of Z
// in range(V) is damped by 1/gamma and dominated by rounding).  From eqs.
// SM-step-2-Z, for k < m:  v_k^T Z^(m) = v_k^T Z^(m-1) - (v_k^T h_m) c_m, and
// v_k^T Z^(k) = c_k / gamma_k, so with Q_km = v_k^T u_m^(m-1) (the final, frozen
// columns of U) and chat_m = c_m / gamma_m:
//     V^T Z = (I - triu(Q, 1)) chat,
// an identity in exact arithmetic.  Q is a strictly-upper Gram matrix of V and the
// final U, computed here split over rows with double partials.
#include <math.h>

#include <cuda_bf16.h>

#include "internal.h"

namespace enkf {
namespace {

// ---------------------------------------------------------------------------
// Q[k][m] = sum_j A[j,k] B[j,m], k < m.  64 x 64 output tile per CTA, 256 threads
// with 4 x 4 outputs each, rows in sub-blocks of 32 staged transposed in smem.
// ---------------------------------------------------------------------------
constexpr int GT = 64;   // tile edge
constexpr int GR = 32;   // rows per smem stage

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(sizeof(T)),
                 "r"(valid ? (int)sizeof(T) : 0)
                 : "memory");
}

template <typename T>
__global__ void __launch_bounds__(256, 2) gram_upper_kernel(int64_t nrows, int n, const T* __restrict__ A, int64_t lda,
                                                         const T* __restrict__ B, int64_t ldb, int64_t rows_per_split,
                                                         double* __restrict__ Qpart, int full) {
    // two stages of SR rows x 64 columns of A and B, [row][column] (pitch GT + 4) so that a
    // thread's four columns are one 16-byte load
    constexpr int SR = sizeof(T) == 8 ? GR / 2 : GR;
    constexpr int CP = GT + 4;
    __shared__ __align__(16) T As[2][SR][CP];
    __shared__ __align__(16) T Bs[2][SR][CP];
    // map blockIdx.x to a tile: every (kb, mb) when full, else the upper tiles (kb <= mb)
    const int nt = (n + GT - 1) / GT;
    int kb = 0, mb = 0;
    if (full) {
        kb = blockIdx.x / nt;
        mb = blockIdx.x % nt;
    } else {
        int t = blockIdx.x;
        while (t >= nt - kb) {
            t -= nt - kb;
            ++kb;
        }
        mb = kb + t;
    }
    const int split = blockIdx.y;
    const int64_t j0 = (int64_t)split * rows_per_split;
    const int64_t j1 = min(j0 + rows_per_split, nrows);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double accd[4][4];
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) accd[i][q] = 0.0, acc[i][q] = T(0);
    // asynchronous copies of one stage: lane -> row (coalesced), warp and step -> column
    auto stage = [&](int64_t jb, int buf) {
        const int lr = tid % SR;
        const int64_t j = jb + lr;
        for (int c = tid / SR; c < GT; c += 256 / SR) {
            const int ka = kb * GT + c, mbc = mb * GT + c;
            const bool va = j < j1 && ka < n, vb = j < j1 && mbc < n;
            cp_async_elem(&As[buf][lr][c], va ? A + (int64_t)ka * lda + j : A, va);
            cp_async_elem(&Bs[buf][lr][c], vb ? B + (int64_t)mbc * ldb + j : B, vb);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    int stage_no = 0;
    if (j0 < j1) stage(j0, 0);
    for (int64_t jb = j0; jb < j1; jb += SR) {
        const int buf = (int)(((jb - j0) / SR) & 1);
        if (jb + SR < j1) {
            stage(jb + SR, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < SR; ++j) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][j][ty * 4 + i];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[buf][j][tx * 4 + q];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] += a[i] * b[q];
        }
        __syncthreads();     // the buffer is refilled by the next iteration's prefetch
        // fold the working-precision accumulators into double every 512 rows
        if (++stage_no == 512 / SR) {
            stage_no = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) accd[i][q] += (double)acc[i][q], acc[i][q] = T(0);
        }
    }
    double* out = Qpart + (int64_t)split * n * n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = kb * GT + ty * 4 + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = mb * GT + tx * 4 + q;
            if (k < n && m < n && (full || k < m)) out[(int64_t)k * n + m] = accd[i][q] + (double)acc[i][q];
        }
    }
}

__global__ void gram_reduce_kernel(int n, int nsplit, const double* __restrict__ Qpart, double* __restrict__ Q,
                                   int full) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), m = (int)(e % n);
        double s = 0.0;
        if (full || k < m)
            for (int p = 0; p < nsplit; ++p) s += Qpart[(int64_t)p * nn + e];
        Q[e] = s;
    }
}

// Row k of (I - triu(Q,1)) diag(1/gamma) C at column i: chat[k][i] - sum_{m>k} Q[k][m] chat[m][i],
// chat[m][i] = C[m][i] / gamma_m, summed in ascending m.  A thread owns one (k, i); the
// threads of a warp share k (Q[k][m] is one broadcast load) and take consecutive i (C[m][i]
// coalesced).  Eight terms' loads are issued before their multiply-adds, so that the chain
// of L2 round trips is an eighth as long; the order of the sum is unchanged.
__device__ __forceinline__ double identity_row_term(int n, int k, int i, const double* __restrict__ Q,
                                                    const double* __restrict__ C, const double* ginv) {
    const double* q = Q + (int64_t)k * n;
    double s = C[(int64_t)k * n + i] * ginv[k];
    int m = k + 1;
    for (; m + 8 <= n; m += 8) {
        double qa[8], ca[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            qa[u] = q[m + u];
            ca[u] = C[(int64_t)(m + u) * n + i];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s -= qa[u] * (ca[u] * ginv[m + u]);
    }
    for (; m < n; ++m) s -= q[m] * (C[(int64_t)m * n + i] * ginv[m]);
    return s;
}

// M[k + i n] = (row k of the identity at column i) / sqrt(n - 1).
template <typename T>
__global__ void assemble_M_kernel(int n, const double* __restrict__ Q, const double* __restrict__ C,
                                  const double* __restrict__ gamma, T* __restrict__ M, double* __restrict__ M64) {
    extern __shared__ double ginv[];     // 1 / gamma_m, one division per level per CTA
    for (int m = threadIdx.x; m < n; m += blockDim.x) ginv[m] = 1.0 / gamma[m];
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int k = (int)(e / n), i = (int)(e % n);
    const double s = identity_row_term(n, k, i, Q, C, ginv) * (1.0 / sqrt((double)(n - 1)));
    const int64_t o = k + (int64_t)i * n;
    if (M) M[o] = (T)s;
    if (M64) M64[o] = s;
}

// P = V^T Z by the same identity, unscaled and row-major (P[k n + i] = v_k^T z_i).
__global__ void assemble_P_kernel(int n, const double* __restrict__ Q, const double* __restrict__ C,
                                  const double* __restrict__ gamma, double* __restrict__ P) {
    extern __shared__ double ginv[];     // 1 / gamma_m, one division per level per CTA
    for (int m = threadIdx.x; m < n; m += blockDim.x) ginv[m] = 1.0 / gamma[m];
    __syncthreads();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int k = (int)(e / n), i = (int)(e % n);
    P[e] = identity_row_term(n, k, i, Q, C, ginv);
}

// ---------------------------------------------------------------------------
// XA = XB + dXB * M.  CTA tile 128 rows x 64 columns, 256 threads; lane -> 4 rows
// (lane + 32 r), warp -> 8 columns.  The 64 needed columns of M sit in smem for
// the whole K = n; dXB is staged 32 columns (of K) at a time.
// ---------------------------------------------------------------------------
constexpr int XBM = 128, XBN = 64, XBK = 32;

template <typename T>
__global__ void __launch_bounds__(256) xa_update_kernel(int64_t nstate, int n, const T* XB, int64_t ldb,
                                                        const T* __restrict__ dXB, int64_t ldx,
                                                        const T* __restrict__ M, T* XA, int64_t lda) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ms = reinterpret_cast<T*>(smem_raw);          // [n][XBN]  Ms[k*XBN + c] = M[k + (e0+c) n]
    T* As = Ms + (size_t)n * XBN;                    // [XBK][XBM]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * XBM;
    const int e0 = blockIdx.y * XBN;
    for (int idx = tid; idx < n * XBN; idx += 256) {
        const int k = idx / XBN, c = idx % XBN;
        Ms[idx] = (e0 + c < n) ? M[k + (int64_t)(e0 + c) * n] : T(0);
    }
    T acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = T(0);
    for (int k0 = 0; k0 < n; k0 += XBK) {
        __syncthreads();
        for (int idx = tid; idx < XBK * XBM; idx += 256) {
            const int kk = idx / XBM, rr = idx % XBM;
            const int64_t i = i0 + rr;
            As[idx] = (k0 + kk < n && i < nstate) ? dXB[(int64_t)(k0 + kk) * ldx + i] : T(0);
        }
        __syncthreads();
        const int kmax = min(XBK, n - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            T a[4], b[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk * XBM + lane + 32 * r];
#pragma unroll
            for (int c = 0; c < 8; ++c) b[c] = Ms[(k0 + kk) * XBN + warp * 8 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] += a[r] * b[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int e = e0 + warp * 8 + c;
        if (e >= n) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = i0 + lane + 32 * r;
            if (i < nstate) XA[(int64_t)e * lda + i] = XB[(int64_t)e * ldb + i] + acc[r][c];
        }
    }
}

}  // namespace

int32_t gram_upper_nsplit(int64_t nrows, int32_t n) {
    const int nt = (n + GT - 1) / GT;
    const int tiles = nt * (nt + 1) / 2;
    int64_t want = (152 * 4 + tiles - 1) / tiles;          // about four waves of CTAs
    int64_t by_rows = (nrows + 1023) / 1024;               // at least 1024 rows per split
    int64_t s = want < by_rows ? want : by_rows;
    if (s < 1) s = 1;
    if (s > 1024) s = 1024;
    return (int32_t)s;
}

static cudaError_t gram_tc_reduce(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B,
                                  int64_t ldb, double* Qpart, int32_t nsplit, double* Q, int full, Control* ctl,
                                  uint64_t timeout_ns, cudaStream_t s) {
    int32_t used = 0;
    // Every 32 rows (one chunk per stage).  Folding every 128 rows made the Gram 20 % faster
    // at Nobs = 2^19 but raised the relative error of Q from 1.8e-7 to 8e-7: the error of M
    // against FP64 grew from 6.3e-5 to 8.0e-5, and one refinement step contracted M's error
    // by 0.47 instead of 0.1.
    const int stage_chunks = 1;
    cudaError_t e = gram_tc05(nrows, n, A, lda, B, ldb, Qpart, nsplit, full, stage_chunks, ctl, timeout_ns, s, &used);
    if (e == cudaErrorNotSupported) e = gram_tc(nrows, n, A, lda, B, ldb, Qpart, nsplit, full, s, &used);
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    gram_reduce_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, used, Qpart, Q, full);
    return cudaGetLastError();
}

static cudaError_t gram_launch(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B,
                               int64_t ldb, double* Qpart, int32_t nsplit, double* Q, int full, Control* ctl,
                               uint64_t timeout_ns, cudaStream_t s) {
    const int nt = (n + GT - 1) / GT;
    const int tiles = full ? nt * nt : nt * (nt + 1) / 2;
    int64_t rps = (nrows + nsplit - 1) / nsplit;
    rps = (rps + GR - 1) / GR * GR;
    dim3 grid(tiles, nsplit);
    if (fp64)
        gram_upper_kernel<double><<<grid, 256, 0, s>>>(nrows, n, (const double*)A, lda, (const double*)B, ldb, rps, Qpart,
                                                       full);
    else
        return gram_tc_reduce(nrows, n, (const float*)A, lda, (const float*)B, ldb, Qpart, nsplit, Q, full, ctl,
                              timeout_ns, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    gram_reduce_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, nsplit, Qpart, Q, full);
    return cudaGetLastError();
}

cudaError_t gram_upper(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                       double* Qpart, int32_t nsplit, double* Q, Control* ctl, uint64_t timeout_ns, cudaStream_t s) {
    return gram_launch(fp64, nrows, n, A, lda, B, ldb, Qpart, nsplit, Q, 0, ctl, timeout_ns, s);
}

cudaError_t gram_full(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                      double* Qpart, int32_t nsplit, double* Q, Control* ctl, uint64_t timeout_ns, cudaStream_t s) {
    return gram_launch(fp64, nrows, n, A, lda, B, ldb, Qpart, nsplit, Q, 1, ctl, timeout_ns, s);
}

cudaError_t assemble_M(bool fp64, int32_t nens, const double* Q, const double* C, const double* gamma, void* M,
                       double* M64, cudaStream_t s) {
    const int64_t nn = (int64_t)nens * nens;
    const int blocks = (int)((nn + 255) / 256);
    if (fp64)
        assemble_M_kernel<double><<<blocks, 256, sizeof(double) * nens, s>>>(nens, Q, C, gamma, (double*)M, M64);
    else
        assemble_M_kernel<float><<<blocks, 256, sizeof(double) * nens, s>>>(nens, Q, C, gamma, (float*)M, M64);
    return cudaGetLastError();
}

cudaError_t assemble_P(int32_t nens, const double* Q, const double* C, const double* gamma, double* P,
                       cudaStream_t s) {
    const int64_t nn = (int64_t)nens * nens;
    assemble_P_kernel<<<(int)((nn + 255) / 256), 256, sizeof(double) * nens, s>>>(nens, Q, C, gamma, P);
    return cudaGetLastError();
}

cudaError_t xa_update(bool fp64, int64_t nstate, int32_t nens, const void* XB, int64_t ldb, const void* dXB,
                      int64_t ldx, const void* M, void* XA, int64_t lda, cudaStream_t s) {
    const size_t w = fp64 ? 8 : 4;
    const size_t smem = w * ((size_t)nens * XBN + (size_t)XBK * XBM);
    dim3 grid((unsigned)((nstate + XBM - 1) / XBM), (unsigned)((nens + XBN - 1) / XBN));
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(xa_update_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        xa_update_kernel<double><<<grid, 256, smem, s>>>(nstate, nens, (const double*)XB, ldb, (const double*)dXB, ldx,
                                                         (const double*)M, (double*)XA, lda);
    } else {
        e = cudaFuncSetAttribute(xa_update_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        xa_update_kernel<float><<<grid, 256, smem, s>>>(nstate, nens, (const float*)XB, ldb, (const float*)dXB, ldx,
                                                        (const float*)M, (float*)XA, lda);
    }
    return cudaGetLastError();
}

}  // namespace enkf
