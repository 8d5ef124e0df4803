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
__global__ void __launch_bounds__(256) gram_upper_kernel(int64_t nrows, int n, const T* __restrict__ A, int64_t lda,
                                                         const T* __restrict__ B, int64_t ldb, int64_t rows_per_split,
                                                         double* __restrict__ Qpart, int full) {
    __shared__ T As[GT][GR + 1];
    __shared__ T Bs[GT][GR + 1];
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
    int stage = 0;
    for (int64_t jb = j0; jb < j1; jb += GR) {
        __syncthreads();
        // load 32 rows x 64 columns of A and B: lane -> row, warp and step -> column
        const int lr = tid & 31;
        for (int c = tid >> 5; c < GT; c += 8) {
            const int64_t j = jb + lr;
            const int ka = kb * GT + c, mbc = mb * GT + c;
            As[c][lr] = (j < j1 && ka < n) ? A[(int64_t)ka * lda + j] : T(0);
            Bs[c][lr] = (j < j1 && mbc < n) ? B[(int64_t)mbc * ldb + j] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < GR; ++j) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][j];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[tx * 4 + q][j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] += a[i] * b[q];
        }
        // fold the working-precision accumulators into double every 16 stages (512 rows)
        if (++stage == 16) {
            stage = 0;
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

// M[k + i n] = (chat[k][i] - sum_{m>k} Q[k][m] chat[m][i]) / sqrt(n - 1), chat[m][i] = C[m][i] / gamma_m.
template <typename T>
__global__ void assemble_M_kernel(int n, const double* __restrict__ Q, const double* __restrict__ C,
                                  const double* __restrict__ gamma, T* __restrict__ M, double* __restrict__ M64) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int k = (int)(e % n), i = (int)(e / n);
    double s = C[(int64_t)k * n + i] / gamma[k];
    for (int m = k + 1; m < n; ++m) s -= Q[(int64_t)k * n + m] * (C[(int64_t)m * n + i] / gamma[m]);
    s *= 1.0 / sqrt((double)(n - 1));
    if (M) M[e] = (T)s;
    if (M64) M64[e] = s;
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

// ---------------------------------------------------------------------------
// XA = XB + dXB * M on BF16 tensor cores with split operands (FP32 storage):
// dXB = A_hi + A_lo and M = M_hi + M_lo (BF16 each), XA = XB + A_hi M_hi + A_hi M_lo
// + A_lo M_hi (the dropped A_lo M_lo term is below FP32 rounding), FP32 accumulation
// (mma.sync m16n8k16).  CTA tile 128 rows x 128 columns, 8 warps of 32 x 64, K in
// chunks of 32; A chunks are staged [k][row] (fragments by ldmatrix.trans), M is
// pre-split into [col][k] hi/lo (ldmatrix).  X_B initialises the accumulators.
// ---------------------------------------------------------------------------
constexpr int TR = 128, TC = 128, KC = 32;
constexpr int APITCH = TR + 8;     // bf16, [k][row]
constexpr int BPITCH = KC + 8;     // bf16, [col][k]

__global__ void split_M_kernel(const float* __restrict__ M, int n, int kpad, __nv_bfloat16* __restrict__ Mhi,
                               __nv_bfloat16* __restrict__ Mlo) {
    // Mhi/Mlo[e][k] = split of M[k + e n] (k < n), zero for k >= n
    const int64_t total = (int64_t)n * kpad;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(q / kpad), k = (int)(q % kpad);
        const float v = k < n ? M[k + (int64_t)e * n] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16(v);
        Mhi[q] = h;
        Mlo[q] = __float2bfloat16(v - __bfloat162float(h));
    }
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) xa_update_tc_kernel(int64_t nstate, int n, int kpad, const float* XB,
                                                           int64_t ldb, const float* __restrict__ dXB, int64_t ldx,
                                                           const __nv_bfloat16* __restrict__ Mhi,
                                                           const __nv_bfloat16* __restrict__ Mlo, float* XA,
                                                           int64_t lda, int vec_a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(smem_raw);   // [KC][APITCH]
    __nv_bfloat16* Alo = Ahi + KC * APITCH;
    __nv_bfloat16* Bhi = Alo + KC * APITCH;                              // [TC][BPITCH]
    __nv_bfloat16* Blo = Bhi + TC * BPITCH;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 3) * 32, wn = (warp >> 2) * 64;
    const int e0 = blockIdx.y * TC;
    const int64_t ntiles = (nstate + TR - 1) / TR;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i0 = tile * TR;
        float acc[2][8][4];
        // accumulators start at X_B
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int64_t i = i0 + wm + mt * 16 + (lane >> 2) + (h >> 1) * 8;
                    const int e = e0 + wn + nt * 8 + (lane & 3) * 2 + (h & 1);
                    acc[mt][nt][h] = (i < nstate && e < n) ? XB[(int64_t)e * ldb + i] : 0.f;
                }
        for (int k0 = 0; k0 < kpad; k0 += KC) {
            __syncthreads();
            // A chunk: dXB rows i0.., members k0..k0+31 -> [k][row] hi/lo
            for (int q = tid; q < KC * (TR / 4); q += 256) {
                const int k = q / (TR / 4), r4 = (q % (TR / 4)) * 4;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                if (k0 + k < n) {
                    const float* src = dXB + (int64_t)(k0 + k) * ldx + i0 + r4;
                    if (vec_a && i0 + r4 + 3 < nstate) {
                        const float4 f = *reinterpret_cast<const float4*>(src);
                        v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
                    } else {
                        for (int u = 0; u < 4; ++u)
                            if (i0 + r4 + u < nstate) v[u] = src[u];
                    }
                }
                __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    h[u] = __float2bfloat16(v[u]);
                    l[u] = __float2bfloat16(v[u] - __bfloat162float(h[u]));
                }
                *reinterpret_cast<uint2*>(Ahi + k * APITCH + r4) = *reinterpret_cast<const uint2*>(h);
                *reinterpret_cast<uint2*>(Alo + k * APITCH + r4) = *reinterpret_cast<const uint2*>(l);
            }
            // B chunk: [col][k] hi/lo for columns e0.., k0..k0+31 (16-byte copies)
            for (int q = tid; q < TC * (KC / 8); q += 256) {
                const int c = q / (KC / 8), k8 = (q % (KC / 8)) * 8;
                uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
                if (e0 + c < n) {
                    vh = *reinterpret_cast<const uint4*>(Mhi + (int64_t)(e0 + c) * kpad + k0 + k8);
                    vl = *reinterpret_cast<const uint4*>(Mlo + (int64_t)(e0 + c) * kpad + k0 + k8);
                }
                *reinterpret_cast<uint4*>(Bhi + c * BPITCH + k8) = vh;
                *reinterpret_cast<uint4*>(Blo + c * BPITCH + k8) = vl;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; kk += 16) {
                uint32_t ah[2][4], al[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    // matrices (m 0-7,k 0-7) (m 8-15,k 0-7) (m 0-7,k 8-15) (m 8-15,k 8-15) from [k][row]
                    const int j = lane >> 3;
                    const int kr = kk + (j >> 1) * 8 + (lane & 7);
                    const int mr = wm + mt * 16 + (j & 1) * 8;
                    ldsm_x4_t(ah[mt], Ahi + kr * APITCH + mr);
                    ldsm_x4_t(al[mt], Alo + kr * APITCH + mr);
                }
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    // two n-tiles: matrices (n 0-7,k 0-7) (n 0-7,k 8-15) (n 8-15,k 0-7) (n 8-15,k 8-15)
                    const int j = lane >> 3;
                    const int nr = wn + np * 16 + (j >> 1) * 8 + (lane & 7);
                    const int kc = kk + (j & 1) * 8;
                    uint32_t bh[4], bl[4];
                    ldsm_x4(bh, Bhi + nr * BPITCH + kc);
                    ldsm_x4(bl, Blo + nr * BPITCH + kc);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            float* d = acc[mt][np * 2 + hh];
                            mma16816(d, al[mt], bh[2 * hh], bh[2 * hh + 1]);
                            mma16816(d, ah[mt], bl[2 * hh], bl[2 * hh + 1]);
                            mma16816(d, ah[mt], bh[2 * hh], bh[2 * hh + 1]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int64_t i = i0 + wm + mt * 16 + (lane >> 2) + (h >> 1) * 8;
                    const int e = e0 + wn + nt * 8 + (lane & 3) * 2 + (h & 1);
                    if (i < nstate && e < n) XA[(int64_t)e * lda + i] = acc[mt][nt][h];
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

static cudaError_t gram_launch(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B,
                               int64_t ldb, double* Qpart, int32_t nsplit, double* Q, int full, cudaStream_t s) {
    const int nt = (n + GT - 1) / GT;
    const int tiles = full ? nt * nt : nt * (nt + 1) / 2;
    int64_t rps = (nrows + nsplit - 1) / nsplit;
    rps = (rps + GR - 1) / GR * GR;
    dim3 grid(tiles, nsplit);
    if (fp64)
        gram_upper_kernel<double><<<grid, 256, 0, s>>>(nrows, n, (const double*)A, lda, (const double*)B, ldb, rps, Qpart,
                                                       full);
    else
        gram_upper_kernel<float><<<grid, 256, 0, s>>>(nrows, n, (const float*)A, lda, (const float*)B, ldb, rps, Qpart,
                                                      full);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    gram_reduce_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, nsplit, Qpart, Q, full);
    return cudaGetLastError();
}

cudaError_t gram_upper(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                       double* Qpart, int32_t nsplit, double* Q, cudaStream_t s) {
    return gram_launch(fp64, nrows, n, A, lda, B, ldb, Qpart, nsplit, Q, 0, s);
}

cudaError_t gram_full(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                      double* Qpart, int32_t nsplit, double* Q, cudaStream_t s) {
    return gram_launch(fp64, nrows, n, A, lda, B, ldb, Qpart, nsplit, Q, 1, s);
}

cudaError_t assemble_M(bool fp64, int32_t nens, const double* Q, const double* C, const double* gamma, void* M,
                       double* M64, cudaStream_t s) {
    const int64_t nn = (int64_t)nens * nens;
    const int blocks = (int)((nn + 255) / 256);
    if (fp64)
        assemble_M_kernel<double><<<blocks, 256, 0, s>>>(nens, Q, C, gamma, (double*)M, M64);
    else
        assemble_M_kernel<float><<<blocks, 256, 0, s>>>(nens, Q, C, gamma, (float*)M, M64);
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

namespace enkf {

int32_t xa_tc_kpad(int32_t nens) { return (nens + KC - 1) / KC * KC; }

cudaError_t xa_update_tc(int64_t nstate, int32_t nens, const float* XB, int64_t ldb, const float* dXB, int64_t ldx,
                         const float* M, void* msplit, float* XA, int64_t lda, cudaStream_t s) {
    const int kpad = xa_tc_kpad(nens);
    __nv_bfloat16* Mhi = static_cast<__nv_bfloat16*>(msplit);
    __nv_bfloat16* Mlo = Mhi + (size_t)nens * kpad;
    split_M_kernel<<<(int)(((int64_t)nens * kpad + 255) / 256), 256, 0, s>>>(M, nens, kpad, Mhi, Mlo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(__nv_bfloat16) * (2 * KC * APITCH + 2 * TC * BPITCH);
    if ((e = cudaFuncSetAttribute(xa_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (nstate + TR - 1) / TR;
    const int ycols = (nens + TC - 1) / TC;
    int64_t gx = (int64_t)nsm * 3 / ycols;
    if (gx < 1) gx = 1;
    if (gx > ntiles) gx = ntiles;
    const int vec_a = ((uintptr_t)dXB % 16 == 0) && (ldx % 4 == 0);
    xa_update_tc_kernel<<<dim3((unsigned)gx, (unsigned)ycols), 256, smem, s>>>(nstate, nens, kpad, XB, ldb, dXB, ldx,
                                                                               Mhi, Mlo, XA, lda, vec_a);
    return cudaGetLastError();
}

}  // namespace enkf
