// One step of iterative refinement of the panel solve (mixed-precision modes).
//
// With Z1 the solve's result and P = V^T Z1 (N x N):
//   delta0 = R^{-1} (D - (R + V V^T) Z1) = (D - r o Z1 - V P) / r,
// the stored panel factors are applied to delta0 (refinement sweep of the panel
// kernel) giving delta, and
//   Z = Z1 + delta,   M = (V^T Z1 + V^T delta) / sqrt(N - 1) = (P + V^T delta) / sqrt(N - 1).
//
// P must be accurate: the part of Z in range(V) is damped by 1/gamma (gamma ~ 10^4 at
// Nobs = 2^19), so |P| is about 10^-6 of sum_j |v_j||z_j|, and an error e relative to that
// sum becomes about 10^6 e relative in M.  The Gram P is therefore formed from
// fixed-point BF16 digits on the tensor cores (gram_exact, ~2^-32 of that sum) or, when V
// or Z is not TMA-aligned, here with exact products (TwoProd by FMA) and compensated
// (Kahan) FP32 sums over blocks of 512 rows, the block sums and compensations folded into
// FP64 (~2^-40).
//
// The residual's N-term sums V P need no such care.  The same P enters the residual
// and M = P + V^T delta, so an error E in the product V P changes M only by
// (I + V^T R^-1 V)^-1 V^T R^-1 E, damped by 1/gamma; it changes Z by R^-1 E-sized
// amounts, so Z keeps its accuracy when E is ~1e-7 of sum |v||p|.  So T = D - r o Z1 is
// one FP32 fused multiply-add per element, and (T - V P) / r runs on the tensor cores as
// the X_A update (three BF16 pieces, six products, FP32 accumulation) with -P in place
// of M and a divisor r per row.
// V^T delta needs no compensation either: delta is the small correction, so the plain
// Gram's relative error is scaled by |delta|/|Z|.
#include <math.h>
#include <stdint.h>

#include <initializer_list>

#include "internal.h"

namespace enkf {
namespace {

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

// The element-wise passes over Nobs x N column blocks below take one member column per
// blockIdx.y (stepping by gridDim.y) and the rows of that column grid-stride along x, as
// float4 accesses when Nobs, every leading dimension and every base are multiples of 4
// floats (16 bytes), else one element per thread.  No per-element index division.
inline bool vec4_ok(int64_t nobs, std::initializer_list<const void*> ptrs, std::initializer_list<int64_t> lds) {
    if (nobs % 4 != 0) return false;
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16 != 0) return false;
    for (int64_t ld : lds)
        if (ld % 4 != 0) return false;
    return true;
}

// Grid of the element-wise passes: about 16 CTAs of 256 threads per SM in all, no more
// x-blocks than a column has 256-unit rows.
inline dim3 ew_grid(int64_t nobs, int n, bool vec) {
    const int64_t units = vec ? nobs / 4 : nobs;
    const int gy = n < 65535 ? (n > 0 ? n : 1) : 65535;
    int64_t gx = (152 * 16 + gy - 1) / gy;
    const int64_t need = (units + 255) / 256;
    if (gx > need) gx = need;
    if (gx < 1) gx = 1;
    return dim3((unsigned)gx, (unsigned)gy);
}

// T = D - r o Z1, one FP32 fused multiply-add per element (one rounding).
template <bool VEC>
__global__ void __launch_bounds__(256) residual_prep_kernel(int64_t nobs, int n, const float* __restrict__ r,
                                                            const float* __restrict__ D, int64_t ldd,
                                                            const float* __restrict__ Z, int64_t ldz,
                                                            float* __restrict__ out, int64_t ldo) {
    const int64_t units = VEC ? nobs / 4 : nobs;
    const int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, qs = (int64_t)gridDim.x * blockDim.x;
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        const float* d = D + (int64_t)i * ldd;
        const float* z = Z + (int64_t)i * ldz;
        float* o = out + (int64_t)i * ldo;
        for (int64_t q = q0; q < units; q += qs) {
            if (VEC) {
                const float4 rv = __ldg(reinterpret_cast<const float4*>(r) + q);
                const float4 dv = __ldcs(reinterpret_cast<const float4*>(d) + q);
                const float4 zv = __ldcs(reinterpret_cast<const float4*>(z) + q);
                float4 ov;
                ov.x = __fmaf_rn(-rv.x, zv.x, dv.x);
                ov.y = __fmaf_rn(-rv.y, zv.y, dv.y);
                ov.z = __fmaf_rn(-rv.z, zv.z, dv.z);
                ov.w = __fmaf_rn(-rv.w, zv.w, dv.w);
                reinterpret_cast<float4*>(o)[q] = ov;
            } else {
                o[q] = __fmaf_rn(-r[q], z[q], d[q]);
            }
        }
    }
}

// Mneg[k + i n] = -P[k][i] rounded to FP32 (P row-major FP64).
__global__ void neg_p_kernel(int n, const double* __restrict__ P, float* __restrict__ Mneg) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q % n), i = (int)(q / n);
        Mneg[q] = (float)(-P[(int64_t)k * n + i]);
    }
}

constexpr int kNormBlocks = 512;

// Per-CTA FP64 sums of delta^2 and (D / r)^2 over a fixed share of the elements.
__global__ void __launch_bounds__(256) resid_norm_kernel(int64_t nobs, int n, const float* __restrict__ delta,
                                                         int64_t ldd, const float* __restrict__ r,
                                                         const float* __restrict__ D, int64_t ldD,
                                                         double* __restrict__ part) {
    __shared__ double red[2][256];
    const int64_t total = nobs * n;
    double a = 0.0, b = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / nobs);
        const int64_t j = q % nobs;
        const double x = (double)delta[(int64_t)i * ldd + j];
        const double y = (double)D[(int64_t)i * ldD + j] / (double)r[j];
        a += x * x;
        b += y * y;
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[2 * blockIdx.x] = red[0][0], part[2 * blockIdx.x + 1] = red[1][0];
}

__global__ void resid_norm_final_kernel(const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kNormBlocks; ++q) a += part[2 * q], b += part[2 * q + 1];
        out[0] = b > 0.0 ? sqrt(a / b) : 0.0;
    }
}

// Z += delta;  M[k + i n] = (P[k][i] + Pd[k][i]) / sqrt(n - 1)  (P, Pd row-major).
template <bool VEC>
__global__ void __launch_bounds__(256) refine_apply_kernel(int64_t nobs, int n, float* Z, int64_t ldz,
                                                           const float* __restrict__ delta, int64_t ldd,
                                                           const double* __restrict__ P, const double* __restrict__ Pd,
                                                           double* M64, float* M) {
    const int64_t units = VEC ? nobs / 4 : nobs;
    const int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, qs = (int64_t)gridDim.x * blockDim.x;
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        float* z = Z + (int64_t)i * ldz;
        const float* dl = delta + (int64_t)i * ldd;
        for (int64_t q = q0; q < units; q += qs) {
            if (VEC) {
                float4 zv = __ldcs(reinterpret_cast<const float4*>(z) + q);
                const float4 dv = __ldcs(reinterpret_cast<const float4*>(dl) + q);
                zv.x += dv.x;
                zv.y += dv.y;
                zv.z += dv.z;
                zv.w += dv.w;
                reinterpret_cast<float4*>(z)[q] = zv;
            } else {
                z[q] += dl[q];
            }
        }
    }
    const int64_t nn = (int64_t)n * n;
    const double scale = 1.0 / sqrt((double)(n - 1));
    const int64_t nthreads = (int64_t)gridDim.x * gridDim.y * blockDim.x;
    for (int64_t q = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; q < nn;
         q += nthreads) {
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
                            int64_t ldd, const float* Z, int64_t ldz, const double* P, float* Mneg, void* msplit,
                            float* delta, int64_t ldo, Control* ctl, uint64_t timeout_ns, cudaStream_t s) {
    const bool vec = vec4_ok(nobs, {r, D, Z, delta}, {ldd, ldz, ldo});
    const dim3 grid = ew_grid(nobs, n, vec);
    if (vec)
        residual_prep_kernel<true><<<grid, 256, 0, s>>>(nobs, n, r, D, ldd, Z, ldz, delta, ldo);
    else
        residual_prep_kernel<false><<<grid, 256, 0, s>>>(nobs, n, r, D, ldd, Z, ldz, delta, ldo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    neg_p_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, P, Mneg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // delta = (T + V (-P)) / r on the tensor cores, written over T
    return xa_update_tc05(nobs, n, delta, ldo, V, ldv, Mneg, msplit, delta, ldo, r, 3, ctl, timeout_ns, s);
}

cudaError_t refine_resid_norm(int64_t nobs, int32_t n, const float* delta, int64_t ldd, const float* r,
                              const float* D, int64_t ldD, double* part, double* out, cudaStream_t s) {
    resid_norm_kernel<<<kNormBlocks, 256, 0, s>>>(nobs, n, delta, ldd, r, D, ldD, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resid_norm_final_kernel<<<1, 32, 0, s>>>(part, out);
    return cudaGetLastError();
}

cudaError_t refine_apply(int64_t nobs, int32_t n, float* Z, int64_t ldz, const float* delta, int64_t ldd,
                         const double* P, const double* Pd, double* M64, float* M, cudaStream_t s) {
    const bool vec = vec4_ok(nobs, {Z, delta}, {ldz, ldd});
    const dim3 grid = ew_grid(nobs, n, vec);
    if (vec)
        refine_apply_kernel<true><<<grid, 256, 0, s>>>(nobs, n, Z, ldz, delta, ldd, P, Pd, M64, M);
    else
        refine_apply_kernel<false><<<grid, 256, 0, s>>>(nobs, n, Z, ldz, delta, ldd, P, Pd, M64, M);
    return cudaGetLastError();
}

}  // namespace enkf
