// One step of iterative refinement of the panel solve (mixed-precision modes).
//
// With Z1 the solve's result and P = V^T Z1 (N x N):
//   delta0 = R^{-1} (D - (R + V V^T) Z1) = (D - r o Z1 - V P) / r,
// the stored panel factors are applied to delta0 (refinement sweep of the panel
// kernel) giving delta, and
//   Z = Z1 + delta,   M = (V^T Z1 + V^T delta) / sqrt(N - 1).
//
// M = V^T Z is ill-conditioned for a direct product: the part of Z in range(V) is
// damped by 1/gamma (gamma ~ 10^4 at Nobs = 2^19), so an error e relative to
// |v||z| in the Nobs-long sums becomes about gamma * e relative in M.  The Grams
// here are therefore formed with exact products (TwoProd by FMA) and compensated
// (Kahan) FP32 sums over blocks of 512 rows, the block sums and compensations
// folded into FP64 -- about 2^-40 relative to |v||z| instead of 2^-24 sqrt(512).
// The N-term sums V[j,:] P[:,i] of the residual use the same exact products and
// compensated FP32 sums (P split into hi + lo floats).  FP64 arithmetic for either
// would run on GB300's narrow FP64 pipe.  V^T delta needs no compensation: delta is
// the small correction, so the plain Gram's relative error is scaled by |delta|/|Z|.
#include <math.h>

#include "internal.h"

namespace enkf {
namespace {

constexpr int RCOL = 8;     // residual columns per CTA
constexpr int RPT = 4;      // rows per thread
constexpr int RM = 128;     // rows of P staged at a time

// ---------------------------------------------------------------------------
// Compensated Gram P[k][m] = sum_j A[j,k] B[j,m] (every k, m).  64 x 64 output tile
// per CTA, 256 threads with 4 x 4 outputs, 32 rows per shared-memory stage; the
// rows are split over blockIdx.y and the FP64 partials reduced in a fixed order.
// ---------------------------------------------------------------------------
constexpr int GT = 64;
constexpr int GR = 32;

__global__ void __launch_bounds__(256) gram_comp_kernel(int64_t nrows, int n, const float* __restrict__ A,
                                                        int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                        int64_t rows_per_split, double* __restrict__ part) {
    __shared__ float As[GT][GR + 1];
    __shared__ float Bs[GT][GR + 1];
    const int nt = (n + GT - 1) / GT;
    const int kb = blockIdx.x / nt, mb = blockIdx.x % nt;
    const int64_t j0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t j1 = min(j0 + rows_per_split, nrows);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
    float sum[4][4], cmp[4][4], err[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.0, sum[i][q] = 0.f, cmp[i][q] = 0.f, err[i][q] = 0.f;
    int stage = 0;
    for (int64_t jb = j0; jb < j1; jb += GR) {
        __syncthreads();
        const int lr = tid & 31;
        for (int c = tid >> 5; c < GT; c += 8) {
            const int64_t j = jb + lr;
            const int ka = kb * GT + c, mbc = mb * GT + c;
            As[c][lr] = (j < j1 && ka < n) ? A[(int64_t)ka * lda + j] : 0.f;
            Bs[c][lr] = (j < j1 && mbc < n) ? B[(int64_t)mbc * ldb + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < GR; ++j) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][j];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[tx * 4 + q][j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float p = __fmul_rn(a[i], b[q]);
                    err[i][q] = __fadd_rn(err[i][q], __fmaf_rn(a[i], b[q], -p));   // exact product error
                    const float y = __fsub_rn(p, cmp[i][q]);
                    const float t = __fadd_rn(sum[i][q], y);
                    cmp[i][q] = __fsub_rn(__fsub_rn(t, sum[i][q]), y);
                    sum[i][q] = t;
                }
        }
        if (++stage == 16) {   // fold every 512 rows
            stage = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[i][q] += ((double)sum[i][q] - (double)cmp[i][q]) + (double)err[i][q];
                    sum[i][q] = 0.f, cmp[i][q] = 0.f, err[i][q] = 0.f;
                }
        }
    }
    double* out = part + (int64_t)blockIdx.y * n * n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = kb * GT + ty * 4 + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = mb * GT + tx * 4 + q;
            if (k < n && m < n)
                out[(int64_t)k * n + m] = acc[i][q] + (((double)sum[i][q] - (double)cmp[i][q]) + (double)err[i][q]);
        }
    }
}

__global__ void gram_comp_reduce_kernel(int n, int nsplit, const double* __restrict__ part, double* __restrict__ P) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < nsplit; ++p) s += part[(int64_t)p * nn + e];
        P[e] = s;
    }
}

// Each thread forms RPT rows (j = row0 + t + 256 q) of RCOL residual columns; the
// CTAs of one row block differ in blockIdx.x (the column group), so they run close
// together and share V through L2.
__global__ void __launch_bounds__(256) residual_kernel(int64_t nobs, int n, const float* __restrict__ r,
                                                       const float* __restrict__ V, int64_t ldv,
                                                       const float* __restrict__ D, int64_t ldd,
                                                       const float* __restrict__ Z, int64_t ldz,
                                                       const double* __restrict__ P, float* __restrict__ out,
                                                       int64_t ldo) {
    __shared__ __align__(16) float Ph[RM][RCOL];
    __shared__ __align__(16) float Pl[RM][RCOL];
    const int i0 = blockIdx.x * RCOL;
    const int64_t row0 = (int64_t)blockIdx.y * (256 * RPT) + threadIdx.x;
    // running sums of V[j,:] P[:,i]: sh (FP32, Kahan-compensated by sc) + sl (product
    // errors and the lo part of P)
    float sh[RPT][RCOL], sc[RPT][RCOL], sl[RPT][RCOL];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int c = 0; c < RCOL; ++c) sh[q][c] = 0.f, sc[q][c] = 0.f, sl[q][c] = 0.f;
    for (int m0 = 0; m0 < n; m0 += RM) {
        __syncthreads();
        for (int e = threadIdx.x; e < RM * RCOL; e += blockDim.x) {
            const int m = e / RCOL, c = e % RCOL;
            // P[m][i] = v_m^T z_i, row-major (m * n + i)
            const double pv = (m0 + m < n && i0 + c < n) ? P[(int64_t)(m0 + m) * n + (i0 + c)] : 0.0;
            const float h = (float)pv;
            Ph[m][c] = h;
            Pl[m][c] = (float)(pv - (double)h);
        }
        __syncthreads();
        const int mmax = min(RM, n - m0);
        for (int m = 0; m < mmax; ++m) {
            float v[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int64_t j = row0 + 256 * q;
                v[q] = j < nobs ? V[(int64_t)(m0 + m) * ldv + j] : 0.f;
            }
#pragma unroll
            for (int c = 0; c < RCOL; ++c) {
                const float ph = Ph[m][c], pl = Pl[m][c];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const float p = __fmul_rn(v[q], ph);
                    const float pe = __fmaf_rn(v[q], ph, -p);      // exact error of the product (TwoProd)
                    const float y = __fsub_rn(p, sc[q][c]);
                    const float t = __fadd_rn(sh[q][c], y);
                    sc[q][c] = __fsub_rn(__fsub_rn(t, sh[q][c]), y);
                    sh[q][c] = t;
                    sl[q][c] = __fmaf_rn(v[q], pl, __fadd_rn(sl[q][c], pe));
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t j = row0 + 256 * q;
        if (j >= nobs) break;
        const double rj = (double)r[j];
#pragma unroll
        for (int c = 0; c < RCOL; ++c) {
            const int i = i0 + c;
            if (i >= n) break;
            const double vp = ((double)sh[q][c] - (double)sc[q][c]) + (double)sl[q][c];
            const double res = (double)D[(int64_t)i * ldd + j] - rj * (double)Z[(int64_t)i * ldz + j] - vp;
            out[(int64_t)i * ldo + j] = (float)(res / rj);
        }
    }
}

// Z += delta;  M[k + i n] = (P[k][i] + Pd[k][i]) / sqrt(n - 1)  (P, Pd row-major).
__global__ void refine_apply_kernel(int64_t nobs, int n, float* Z, int64_t ldz, const float* __restrict__ delta,
                                    int64_t ldd, const double* __restrict__ P, const double* __restrict__ Pd,
                                    double* M64, float* M) {
    const int64_t total = nobs * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / nobs);
        const int64_t j = q % nobs;
        Z[(int64_t)i * ldz + j] += delta[(int64_t)i * ldd + j];
    }
    const int64_t nn = (int64_t)n * n;
    const double scale = 1.0 / sqrt((double)(n - 1));
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q % n), i = (int)(q / n);
        const double v = (P[(int64_t)k * n + i] + Pd[(int64_t)k * n + i]) * scale;
        if (M64) M64[q] = v;
        if (M) M[q] = (float)v;
    }
}

}  // namespace

cudaError_t gram_comp(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                      double* part, int32_t nsplit, double* P, cudaStream_t s) {
    const int nt = (n + GT - 1) / GT;
    int64_t rps = (nrows + nsplit - 1) / nsplit;
    rps = (rps + GR - 1) / GR * GR;
    if (rps < GR) rps = GR;
    const int64_t used = (nrows + rps - 1) / rps;           // splits that hold rows
    dim3 grid(nt * nt, (unsigned)(used > 0 ? used : 1));
    gram_comp_kernel<<<grid, 256, 0, s>>>(nrows, n, A, lda, B, ldb, rps, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    gram_comp_reduce_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, (int)grid.y, part, P);
    return cudaGetLastError();
}

cudaError_t refine_residual(int64_t nobs, int32_t n, const float* r, const float* V, int64_t ldv, const float* D,
                            int64_t ldd, const float* Z, int64_t ldz, const double* P, float* delta, int64_t ldo,
                            cudaStream_t s) {
    dim3 grid((unsigned)((n + RCOL - 1) / RCOL), (unsigned)((nobs + 256 * RPT - 1) / (256 * RPT)));
    residual_kernel<<<grid, 256, 0, s>>>(nobs, n, r, V, ldv, D, ldd, Z, ldz, P, delta, ldo);
    return cudaGetLastError();
}

cudaError_t refine_apply(int64_t nobs, int32_t n, float* Z, int64_t ldz, const float* delta, int64_t ldd,
                         const double* P, const double* Pd, double* M64, float* M, cudaStream_t s) {
    int64_t blocks = (nobs * n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    refine_apply_kernel<<<(int)blocks, 256, 0, s>>>(nobs, n, Z, ldz, delta, ldd, P, Pd, M64, M);
    return cudaGetLastError();
}

}  // namespace enkf
