// Gram products Q[k][m] = sum_j A[j,k] B[j,m] of FP32 columns on the tensor cores, for
// the M assembly of the analysis (Sec. 3.1; Q = V^T U of the final U columns) and the
// refinement.  Each FP32 operand is split into three BF16 pieces (x = hi + mid + lo,
// kept to ~2^-25) and the six products a_i b_j with i + j < 3 are summed
// (mma.sync.m16n8k16, FP32 accumulation).  Tensor-core accumulation truncates, so each
// 32-row stage is summed from zero and added to an FP32 running sum, which is folded
// into FP64 every 512 rows -- the accumulation scheme of the CUDA-core Gram.
//
// CTA: one 64 x 64 output tile (kb, mb) over a slice of the rows (blockIdx.y); 8 warps
// of 16 (k) x 32 (m).  FP32 rows are staged by cp.async into [column][row] tiles (two
// stages), split into piece tiles [piece][column][row], and read by ldmatrix.
#include <cuda_bf16.h>

#include "internal.h"

namespace enkf {
namespace {

constexpr int QT = 64;          // output tile edge
constexpr int QR = 32;          // rows per stage
constexpr int RP = QR + 4;      // FP32 stage pitch (floats; 16-byte aligned rows)
constexpr int KP = QR + 8;      // piece pitch (16-bit; conflict-free ldmatrix rows)
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned short bf(float x) { return __bfloat16_as_ushort(__float2bfloat16(x)); }
__device__ __forceinline__ float fb(unsigned short h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

__device__ __forceinline__ void split3(float x, unsigned short& h, unsigned short& m, unsigned short& l) {
    h = bf(x);
    const float r = x - fb(h);
    m = bf(r);
    l = bf(r - fb(m));
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}

struct GramSmem {
    float raw[2][2][QT][RP];                 // [stage][A / B][column][row]
    unsigned short pc[2][3][QT][KP];         // [A / B][piece][column][row]
};

template <bool VEC>
__global__ void __launch_bounds__(kThreads) gram_tc_kernel(int64_t nrows, int n, const float* __restrict__ A,
                                                          int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                          int64_t rows_per_split, double* __restrict__ Qpart,
                                                          int full) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GramSmem& sm = *reinterpret_cast<GramSmem*>(smem_raw);
    const int nt = (n + QT - 1) / QT;
    int kb = 0, mb = 0;
    if (full) {
        kb = blockIdx.x / nt;
        mb = blockIdx.x % nt;
    } else {
        int t = blockIdx.x;
        while (t >= nt - kb) t -= nt - kb, ++kb;
        mb = kb + t;
    }
    const int64_t j0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t j1 = min(j0 + rows_per_split, nrows);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 32;

    // stage rows [jb, jb + 32) of the 64 columns of A and B: [column][row]
    auto stage = [&](int64_t jb, int buf) {
        if (VEC) {
            for (int e = tid; e < 2 * QT * (QR / 4); e += kThreads) {
                const int isb = e / (QT * (QR / 4)), r = e % (QT * (QR / 4));
                const int c = r / (QR / 4), j4 = (r % (QR / 4)) * 4;
                const int col = (isb ? mb : kb) * QT + c;
                const int64_t rem = j1 - (jb + j4);
                const int bytes = (col < n && rem > 0) ? (rem >= 4 ? 16 : 4 * (int)rem) : 0;
                const float* base = isb ? B : A;
                const int64_t ld = isb ? ldb : lda;
                const float* src = bytes ? base + (int64_t)col * ld + jb + j4 : base;
                cp_async16(&sm.raw[buf][isb][c][j4], src, bytes);
            }
        } else {
            for (int e = tid; e < 2 * QT * QR; e += kThreads) {
                const int isb = e / (QT * QR), r = e % (QT * QR);
                const int c = r / QR, j = r % QR;
                const int col = (isb ? mb : kb) * QT + c;
                const bool ok = col < n && jb + j < j1;
                const float* base = isb ? B : A;
                const int64_t ld = isb ? ldb : lda;
                cp_async4(&sm.raw[buf][isb][c][j], ok ? base + (int64_t)col * ld + jb + j : base, ok ? 4 : 0);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    float run[4][4];
    double accd[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 4; ++h) run[q][h] = 0.f, accd[q][h] = 0.0;
    int stage_no = 0;
    if (j0 < j1) stage(j0, 0);
    for (int64_t jb = j0; jb < j1; jb += QR) {
        const int buf = (int)(((jb - j0) / QR) & 1);
        if (jb + QR < j1) {
            stage(jb + QR, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        // split the stage into BF16 pieces: thread -> (operand, column, 4 rows)
        for (int e = tid; e < 2 * QT * (QR / 4); e += kThreads) {
            const int isb = e / (QT * (QR / 4)), r = e % (QT * (QR / 4));
            const int c = r / (QR / 4), j4 = (r % (QR / 4)) * 4;
            const float4 v = *reinterpret_cast<const float4*>(&sm.raw[buf][isb][c][j4]);
            unsigned short h[4], m[4], l[4];
            split3(v.x, h[0], m[0], l[0]);
            split3(v.y, h[1], m[1], l[1]);
            split3(v.z, h[2], m[2], l[2]);
            split3(v.w, h[3], m[3], l[3]);
            *reinterpret_cast<uint2*>(&sm.pc[isb][0][c][j4]) =
                make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16));
            *reinterpret_cast<uint2*>(&sm.pc[isb][1][c][j4]) =
                make_uint2((uint32_t)m[0] | ((uint32_t)m[1] << 16), (uint32_t)m[2] | ((uint32_t)m[3] << 16));
            *reinterpret_cast<uint2*>(&sm.pc[isb][2][c][j4]) =
                make_uint2((uint32_t)l[0] | ((uint32_t)l[1] << 16), (uint32_t)l[2] | ((uint32_t)l[3] << 16));
        }
        __syncthreads();
        float tile[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < 4; ++h) tile[q][h] = 0.f;
#pragma unroll
        for (int ks = 0; ks < QR; ks += 16) {
            uint32_t a[3][4], b[3][2][4];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                ldsm_x4(a[p], &sm.pc[0][p][wm + (lane & 15)][ks + (lane >> 4) * 8]);
#pragma unroll
                for (int np = 0; np < 2; ++np)
                    ldsm_x4(b[p][np], &sm.pc[1][p][wn + np * 16 + ((lane >> 4) << 3) + (lane & 7)]
                                            [ks + ((lane >> 3) & 1) * 8]);
            }
#pragma unroll
            for (int nt4 = 0; nt4 < 4; ++nt4) {
                const int np = nt4 >> 1, hh = nt4 & 1;
                // pieces (i, j) with i + j < 3, smallest first
#pragma unroll
                for (int sum = 2; sum >= 0; --sum)
#pragma unroll
                    for (int i = sum; i >= 0; --i)
                        mma_bf16(tile[nt4], a[i], b[sum - i][np][2 * hh], b[sum - i][np][2 * hh + 1]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < 4; ++h) run[q][h] += tile[q][h];
        if (++stage_no == 512 / QR) {
            stage_no = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int h = 0; h < 4; ++h) accd[q][h] += (double)run[q][h], run[q][h] = 0.f;
        }
        __syncthreads();   // the raw buffer and the pieces are rewritten next
    }
    double* out = Qpart + (int64_t)blockIdx.y * n * n;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = kb * QT + wm + (lane >> 2) + (h >> 1) * 8;
            const int m = mb * QT + wn + q * 8 + (lane & 3) * 2 + (h & 1);
            if (k < n && m < n && (full || k < m)) out[(int64_t)k * n + m] = accd[q][h] + (double)run[q][h];
        }
}

}  // namespace

cudaError_t gram_tc(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                    double* Qpart, int32_t nsplit, int full, cudaStream_t s, int32_t* used) {
    const int nt = (n + QT - 1) / QT;
    const int tiles = full ? nt * nt : nt * (nt + 1) / 2;
    const bool vec = ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && (lda % 4 == 0) && (ldb % 4 == 0);
    const void* fn = vec ? (const void*)gram_tc_kernel<true> : (const void*)gram_tc_kernel<false>;
    const int smem = (int)sizeof(GramSmem);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // One wave: a grid larger than the resident CTAs leaves a partial last wave (e.g. 609 CTAs
    // on 304 slots run as 304 + 304 + 1), so the rows are cut into at most slots / tiles slices.
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem)) != cudaSuccess) return e;
    const int64_t wave = (int64_t)sms * (per_sm > 0 ? per_sm : 1) / tiles;
    if (wave >= 1 && nsplit > wave) nsplit = (int32_t)wave;
    if (nsplit < 1) nsplit = 1;
    int64_t rps = (nrows + nsplit - 1) / nsplit;
    rps = (rps + QR - 1) / QR * QR;
    *used = nsplit;
    dim3 grid(tiles, nsplit);
    if (vec)
        gram_tc_kernel<true><<<grid, kThreads, smem, s>>>(nrows, n, A, lda, B, ldb, rps, Qpart, full);
    else
        gram_tc_kernel<false><<<grid, kThreads, smem, s>>>(nrows, n, A, lda, B, ldb, rps, Qpart, full);
    return cudaGetLastError();
}

}  // namespace enkf
