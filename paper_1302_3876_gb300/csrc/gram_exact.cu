// Accurate Gram P[k][m] = sum_j A[j,k] B[j,m] of FP32 columns on the fifth-generation tensor
// cores, for the refinement of the analysis (P = V^T Z1, whose entries are about 1e-6 of
// sum_j |a_j||b_j|: the refined M = (P + V^T delta) / sqrt(N - 1) needs P to ~2^-30 of that
// sum, where a float-split tensor-core Gram reaches ~2^-22 and truncates besides).
//
// Fixed-point digits.  For every 32-row chunk and every column, the converter takes the
// largest magnitude m of the chunk's 32 values and the power of two 2^E > m, scales the
// values to y = x 2^-E in (-1, 1) and writes three digits
//   d0 = rint(2^8 y) 2^-8,  d1 = rint(2^16 (y - d0)) 2^-16,  d2 = rint(2^24 (y - d0 - d1)) 2^-24,
// each an integer of at most 9 bits times a power of two (exact in BF16); y - d0 - d1 - d2
// is at most 2^-25.  The digit products of one level L = i + j lie on the grid 2^-(16 + 8L)
// and their sums over the chunk stay below 2^22 grid steps, so each level's 32-row sum is
// exact in the tensor core's FP32 accumulator whatever order it adds in.  Levels 0, 1 and 2
// (products d0 d0 | d0 d1, d1 d0 | d0 d2, d1 d1, d2 d0) accumulate separately in TMEM; the
// epilogue scales them back by 2^(E_k + E_m) (exact) and adds level 0 into a double-FP32
// running sum by TwoSum, levels 1 and 2 into its low word.  The error is that of the
// dropped digit products and remainders, about 2^-25 of the chunk's largest product per
// row, random in sign: ~2^-32 of sum |a||b| over 2^20 rows.
//
// CTA: one 128 x 64 tile (kb, mb) of P over a slice of the rows (blockIdx.y), one CTA per
// SM, warp-specialised:
//   warp 16     loader: TMA copies (128-byte swizzle) of the FP32 chunks, 32 rows x 128
//               members of A and 32 rows x 64 members of B, into a ring of raw stages.
//   warps 8-15  converters: thread (operand, member) reads its 32 values, writes the chunk
//               exponent to the scale ring and the three digits in the K-major canonical
//               layout of the MMA into a ring of digit stages.
//   warp 17     TMEM allocation and the MMA issue (one thread): per chunk 2 K-steps x 6
//               products (M = 128, N = 64) into the three level accumulators of one of
//               two TMEM buffers.
//   warps 0-7   epilogue: TMEM lane quarter w % 4, column half w / 4; after the last chunk
//               it writes hi + lo of its entries to the slice's partial Gram (FP64).
// TMEM columns: buffer b, level L at (3 b + L) * 64; hi at 384, lo at 448.  Every wait is
// bounded; on expiry the CTA latches ENKF_ERR_TIMEOUT, drains its copies and MMAs with
// bounded waits, frees TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"
#include "tc05.cuh"

namespace enkf {
namespace {

using namespace tc05;

constexpr int EA = 128;                        // A members per tile (MMA M)
constexpr int EB = 64;                         // B members per tile (MMA N)
constexpr int EK = 32;                         // rows per chunk (two K-steps)
constexpr int ERS = 3;                         // raw stages
constexpr int EPS = 2;                         // digit stages
constexpr int ESC = 4;                         // scale slots
constexpr int kEpi = 256, kConv = 256;
constexpr int kThreads = kEpi + kConv + 64;    // + loader warp + MMA warp
constexpr int kRawA = EA * EK * 4;             // 16 KB
constexpr int kRawB = EB * EK * 4;             // 8 KB
constexpr int kRawBytes = kRawA + kRawB;
constexpr int kStepA = EA * 16 * 2;            // one K-step of one digit of A (4 KB)
constexpr int kStepB = EB * 16 * 2;            // (2 KB)
constexpr int kDigA = 2 * kStepA;              // one digit of A for the chunk
constexpr int kDigB = 2 * kStepB;
constexpr int kDigBytes = 3 * kDigA + 3 * kDigB;
constexpr unsigned kTmemCols = 512;

struct ExactShared {
    uint64_t raw_full[ERS], raw_empty[ERS], pc_full[EPS], pc_empty[EPS], acc_full[2], acc_empty[2];
    uint64_t sc_full[ESC], sc_empty[ESC], drained;
    float sA[ESC][EA];
    float sB[ESC][EB];
    unsigned taddr;
    int err;
};

constexpr int kSmem = 1024 + ERS * kRawBytes + EPS * kDigBytes + (int)sizeof(ExactShared);

struct ExactParams {
    int64_t nrows, rows_per_split;
    int n, ntb;
    double* part;
    Control* ctl;
    uint64_t timeout_ns;
};

__device__ __forceinline__ unsigned short bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// The three digits of y (|y| < 1) as BF16 bit patterns.
__device__ __forceinline__ void digits3(float y, unsigned short* d) {
    const float d0 = rintf(y * 256.0f) * (1.0f / 256.0f);
    const float r1 = y - d0;
    const float d1 = rintf(r1 * 65536.0f) * (1.0f / 65536.0f);
    const float r2 = r1 - d1;
    const float d2 = rintf(r2 * 16777216.0f) * (1.0f / 16777216.0f);
    d[0] = bf(d0);
    d[1] = bf(d1);
    d[2] = bf(d2);
}

__global__ void __launch_bounds__(kThreads, 1) gram_exact_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB,
                                                                 ExactParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* raw = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // ERS x kRawBytes
    unsigned char* dgs = raw + ERS * kRawBytes;                                           // EPS x kDigBytes
    ExactShared* sh = reinterpret_cast<ExactShared*>(dgs + EPS * kDigBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int kb = blockIdx.x / p.ntb, mb = blockIdx.x % p.ntb;
    const int64_t j0 = (int64_t)blockIdx.y * p.rows_per_split;
    const int64_t j1 = min(j0 + p.rows_per_split, p.nrows);
    const int nchunks = j1 > j0 ? (int)((j1 - j0 + EK - 1) / EK) : 0;

    if (tid == 0) {
        for (int q = 0; q < ERS; ++q) mbar_init(&sh->raw_full[q], 1), mbar_init(&sh->raw_empty[q], kConv);
        for (int q = 0; q < EPS; ++q) mbar_init(&sh->pc_full[q], kConv), mbar_init(&sh->pc_empty[q], 1);
        for (int q = 0; q < 2; ++q) mbar_init(&sh->acc_full[q], 1), mbar_init(&sh->acc_empty[q], kEpi);
        for (int q = 0; q < ESC; ++q) mbar_init(&sh->sc_full[q], kConv), mbar_init(&sh->sc_empty[q], kEpi);
        mbar_init(&sh->drained, 1);
        sh->err = 0;
        mbar_init_fence();
    }
    if (warp == 17) tmem_alloc(&sh->taddr, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tbase = sh->taddr;

    if (warp == 16) {
        // ---------------- loader (TMA): chunk g of A and of B into raw stage g % ERS
        if (lane == 0) {
            int g = 0;
            for (; g < nchunks; ++g) {
                const int rs = g % ERS;
                if (g >= ERS &&
                    !mbar_wait(&sh->raw_empty[rs], (unsigned)((g / ERS - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                    break;
                mbar_expect_tx(&sh->raw_full[rs], kRawBytes);
                const int x = (int)(j0 + (int64_t)g * EK);
                tma_load_2d(raw + rs * kRawBytes, &tmA, x, kb * EA, &sh->raw_full[rs]);
                tma_load_2d(raw + rs * kRawBytes + kRawA, &tmB, x, mb * EB, &sh->raw_full[rs]);
            }
            // every issued copy has landed before the CTA may exit
            for (int f = g - 1; f >= 0 && f >= g - ERS; --f)
                mbar_drain(&sh->raw_full[f % ERS], (unsigned)((f / ERS) & 1), p.timeout_ns);
        }
    } else if (warp >= 8 && warp < 16) {
        // ---------------- converters: thread (operand op, member r) turns its 32 values into digits
        const int ct = tid - kEpi;
        const int op = ct >> 7, r = ct & 127;
        const bool active = op == 0 || r < EB;
        for (int g = 0; g < nchunks; ++g) {
            const int s = g % EPS, rs = g % ERS, sc = g % ESC;
            if (g >= EPS && !mbar_wait(&sh->pc_empty[s], (unsigned)((g / EPS - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                break;
            if (g >= ESC &&
                !mbar_wait(&sh->sc_empty[sc], (unsigned)((g / ESC - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                break;
            if (!mbar_wait(&sh->raw_full[rs], (unsigned)((g / ERS) & 1), &sh->err, p.ctl, p.timeout_ns)) break;
            float v[EK];
            if (active) {
                // member r's row of 128 bytes; 16-byte chunk c sits at c ^ (r % 8) (128-byte swizzle)
                const unsigned char* row = raw + rs * kRawBytes + (op ? kRawA : 0) + r * 128;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 q = *reinterpret_cast<const float4*>(row + ((c ^ (r & 7)) << 4));
                    v[4 * c] = q.x, v[4 * c + 1] = q.y, v[4 * c + 2] = q.z, v[4 * c + 3] = q.w;
                }
            }
            release_to_async(&sh->raw_empty[rs]);
            if (active) {
                float m = 0.f;
#pragma unroll
                for (int q = 0; q < EK; ++q) m = fmaxf(m, fabsf(v[q]));
                int E = 0;
                if (m > 0.f) frexpf(m, &E);          // m < 2^E
                const float sin = ldexpf(1.0f, -E);   // exact scalings by powers of two
                if (op == 0) sh->sA[sc][r] = ldexpf(1.0f, E);
                else sh->sB[sc][r] = ldexpf(1.0f, E);
                unsigned char* dst = dgs + s * kDigBytes + (op ? 3 * kDigA : 0) + (r >> 3) * 256 + (r & 7) * 16;
                const int dstride = op ? kDigB : kDigA, kstep = op ? kStepB : kStepA;
#pragma unroll
                for (int k8 = 0; k8 < 4; ++k8) {       // rows 8 k8 .. 8 k8 + 7: K-step k8 / 2, core k8 % 2
                    uint32_t w[3][4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        unsigned short a[3], b[3];
                        digits3(v[8 * k8 + 2 * q] * sin, a);
                        digits3(v[8 * k8 + 2 * q + 1] * sin, b);
#pragma unroll
                        for (int d = 0; d < 3; ++d) w[d][q] = a[d] | ((uint32_t)b[d] << 16);
                    }
                    const int off = (k8 >> 1) * kstep + (k8 & 1) * 128;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        *reinterpret_cast<uint4*>(dst + d * dstride + off) = make_uint4(w[d][0], w[d][1], w[d][2], w[d][3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(&sh->sc_full[sc]);
            mbar_arrive(&sh->pc_full[s]);
        }
    } else if (warp < 8) {
        // ---------------- epilogue: chunk sums of the three levels into hi + lo
        const int quarter = warp & 3, half = warp >> 2;
        const unsigned lanes = tbase + ((unsigned)(quarter * 32) << 16);
        const int kl = quarter * 32 + lane;   // this thread's A member within the tile
        bool ok = true;
        for (int g = 0; ok && g < nchunks; ++g) {
            const int b = g & 1, sc = g % ESC;
            if (!mbar_wait(&sh->acc_full[b], (unsigned)((g >> 1) & 1), &sh->err, p.ctl, p.timeout_ns) ||
                !mbar_wait(&sh->sc_full[sc], (unsigned)((g / ESC) & 1), &sh->err, p.ctl, p.timeout_ns)) {
                ok = false;
                break;
            }
            fence_after();
            const float sk = sh->sA[sc][kl];
#pragma unroll 1
            for (int c16 = 0; c16 < 2; ++c16) {
                const unsigned col = (unsigned)(half * 32 + c16 * 16);
                unsigned a0[16], a1[16], a2[16], hi[16], lo[16];
                tmem_ld16(lanes + (unsigned)((3 * b + 0) * EB) + col, a0);
                tmem_ld16(lanes + (unsigned)((3 * b + 1) * EB) + col, a1);
                tmem_ld16(lanes + (unsigned)((3 * b + 2) * EB) + col, a2);
                if (g > 0) {
                    tmem_ld16(lanes + 384u + col, hi);
                    tmem_ld16(lanes + 448u + col, lo);
                }
                tmem_wait_ld(a0);
                reg_fence16(a1);
                reg_fence16(a2);
                if (g > 0) {
                    reg_fence16(hi);
                    reg_fence16(lo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float scl = sk * sh->sB[sc][col + q];
                    const float t = __uint_as_float(a0[q]) * scl;
                    const float h = g > 0 ? __uint_as_float(hi[q]) : 0.f;
                    const float s = h + t;
                    const float tt = s - h;
                    const float e = (h - (s - tt)) + (t - tt);
                    float l = g > 0 ? __uint_as_float(lo[q]) : 0.f;
                    l = __fmaf_rn(__uint_as_float(a1[q]), scl, l);
                    l = __fmaf_rn(__uint_as_float(a2[q]), scl, l);
                    hi[q] = __float_as_uint(s);
                    lo[q] = __float_as_uint(l + e);
                }
                tmem_st16(lanes + 384u + col, hi);
                tmem_st16(lanes + 448u + col, lo);
                tmem_wait_st();   // before the next group's loads reuse the source registers
            }
            fence_before();
            mbar_arrive(&sh->acc_empty[b]);
            mbar_arrive(&sh->sc_empty[sc]);
        }
        if (ok) {
            double* out = p.part + (int64_t)blockIdx.y * p.n * p.n;
            const int k = kb * EA + kl;
#pragma unroll 1
            for (int c16 = 0; c16 < 2; ++c16) {
                const unsigned col = (unsigned)(half * 32 + c16 * 16);
                unsigned hi[16], lo[16];
                if (nchunks > 0) {
                    tmem_ld16(lanes + 384u + col, hi);
                    tmem_ld16(lanes + 448u + col, lo);
                    tmem_wait_ld(hi);
                    reg_fence16(lo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int m = mb * EB + (int)col + q;
                    if (k < p.n && m < p.n)
                        out[(int64_t)k * p.n + m] =
                            nchunks > 0 ? (double)__uint_as_float(hi[q]) + (double)__uint_as_float(lo[q]) : 0.0;
                }
            }
        }
    } else {
        // ---------------- MMA issue (warp 17, one thread)
        if (lane == 0) {
            const unsigned idesc = instr_desc(EA, EB);
            // digit products (i, j) by level i + j; the first of each level starts its accumulator
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0}, lv[6] = {0, 1, 1, 2, 2, 2};
            const int first_of[6] = {1, 1, 0, 1, 0, 0};
            for (int g = 0; g < nchunks; ++g) {
                const int b = g & 1, s = g % EPS;
                if (g >= 2 && !mbar_wait(&sh->acc_empty[b], (unsigned)(((g >> 1) - 1) & 1), &sh->err, p.ctl,
                                         p.timeout_ns))
                    break;
                if (!mbar_wait(&sh->pc_full[s], (unsigned)((g / EPS) & 1), &sh->err, p.ctl, p.timeout_ns)) break;
                fence_after();
                const unsigned char* da = dgs + s * kDigBytes;
                const unsigned char* db = da + 3 * kDigA;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        mma_bf16(tbase + (unsigned)((3 * b + lv[q]) * EB),
                                 smem_desc(da + pa[q] * kDigA + ks * kStepA),
                                 smem_desc(db + pb[q] * kDigB + ks * kStepB), idesc,
                                 (ks == 0 && first_of[q]) ? 0 : 1);
                mma_commit(&sh->pc_empty[s]);
                mma_commit(&sh->acc_full[b]);
            }
            // the commit arrives once every MMA issued above has completed
            mma_commit(&sh->drained);
            mbar_drain(&sh->drained, 0u, p.timeout_ns);
        }
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    if (warp == 17) {
        fence_after();
        tmem_dealloc(tbase, kTmemCols);
    }
}

__global__ void gram_exact_reduce_kernel(int n, int nsplit, const double* __restrict__ part, double* __restrict__ P) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nsplit; ++q) s += part[(int64_t)q * nn + e];
        P[e] = s;
    }
}

}  // namespace

cudaError_t gram_exact(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                       double* part, int32_t nsplit, double* P, Control* ctl, uint64_t timeout_ns, cudaStream_t s) {
    CUtensorMap tmA, tmB;
    memset(&tmA, 0, sizeof(tmA));
    memset(&tmB, 0, sizeof(tmB));
    if (nrows < 1 || n < 1 || !encode_f32_2d(&tmA, A, nrows, n, lda, EK, EA, true) ||
        !encode_f32_2d(&tmB, B, nrows, n, ldb, EK, EB, true))
        return cudaErrorNotSupported;
    const int nta = (n + EA - 1) / EA, ntb = (n + EB - 1) / EB;
    const int tiles = nta * ntb;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // one wave of one CTA per SM
    int64_t wave = sms / tiles;
    if (wave < 1) wave = 1;
    if (nsplit > wave) nsplit = (int32_t)wave;
    if (nsplit < 1) nsplit = 1;
    int64_t rps = (nrows + nsplit - 1) / nsplit;
    rps = (rps + EK - 1) / EK * EK;
    const int used = (int)((nrows + rps - 1) / rps);
    if ((e = cudaFuncSetAttribute(gram_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)) !=
        cudaSuccess)
        return e;
    ExactParams p;
    p.nrows = nrows;
    p.rows_per_split = rps;
    p.n = n;
    p.ntb = ntb;
    p.part = part;
    p.ctl = ctl;
    p.timeout_ns = timeout_ns;
    void* args[] = {&tmA, &tmB, &p};
    e = cudaLaunchKernel((const void*)gram_exact_kernel, dim3((unsigned)tiles, (unsigned)used), dim3(kThreads), args,
                         kSmem, s);
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    gram_exact_reduce_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(n, used, part, P);
    return cudaGetLastError();
}

}  // namespace enkf
