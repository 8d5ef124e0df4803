// Gram products Q[k][m] = sum_j A[j,k] B[j,m] of FP32 columns on the fifth-generation tensor
// cores, for the M assembly of the analysis (Sec. 3.1; Q = V^T U of the final U columns).
// The operands are split as in the mma.sync Gram -- three BF16 pieces per value (x = hi +
// mid + lo, kept to ~2^-25), the six products a_i b_j with i + j < 3, smallest first --
// so both give the same products; here they run as tcgen05.mma (M = N = 128, K = 16)
// with FP32 accumulators in TMEM.
//
// Tensor-core accumulation truncates, so the rows are summed in stages of stage_chunks
// 32-row chunks (12 MMAs per chunk): a stage starts from zero in one of two TMEM
// accumulators, and the epilogue adds it into a double-FP32 running sum (TwoSum: hi + lo)
// that also lives in TMEM.  The truncation error grows with the stage length (relative
// error of Q about 1.8e-7 with one chunk per stage, 8e-7 with four), and the fold is most
// of the kernel's instructions.  TMEM columns: [0,128) and [128,256) the stage
// accumulators, [256,384) hi, [384,512) lo.
//
// CTA: one 128 x 128 tile (kb, mb) of Q over a slice of the rows (blockIdx.y), one CTA per
// SM, warp-specialised:
//   warp 16     loader: TMA copies (128-byte swizzle) of the FP32 chunks of A and B,
//               32 rows x 128 members each, into a ring of raw stages.
//   warps 8-15  converters: thread (operand, member) reads its 32 values (conflict-free
//               through the swizzle) and writes the three BF16 pieces in the K-major
//               canonical layout of the MMA into a ring of piece stages.
//   warp 17     TMEM allocation and the MMA issue (one thread).
//   warps 0-7   epilogue: TMEM lane quarter w % 4, column half w / 4; after the last
//               stage it writes hi + lo of its entries to the slice's partial Gram (FP64).
// Every wait is bounded; on expiry the CTA latches ENKF_ERR_TIMEOUT, drains its copies
// and MMAs with bounded waits, frees TMEM and returns.
#include <cuda_bf16.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"
#include "tc05.cuh"

namespace enkf {
namespace {

using namespace tc05;

constexpr int GM = 128;                       // tile edge: MMA M = N = 128 members
constexpr int GK = 32;                        // rows per chunk (two K-steps)
constexpr int GRS = 3;                        // raw stages
constexpr int GPS = 2;                        // piece stages
constexpr int kEpi = 256, kConv = 256;
constexpr int kThreads = kEpi + kConv + 64;   // + loader warp + MMA warp
constexpr int kRawOp = GM * GK * 4;           // one operand's FP32 chunk (16 KB)
constexpr int kRawBytes = 2 * kRawOp;         // A and B
constexpr int kPieceOp = GM * GK * 2;         // one BF16 piece of one operand (8 KB)
constexpr int kPieceBytes = 2 * 3 * kPieceOp; // A and B, three pieces each
constexpr int kStepBytes = GM * 16 * 2;       // one K-step of one piece (4 KB)
constexpr unsigned kTmemCols = 512;

struct GramShared {
    uint64_t raw_full[GRS], raw_empty[GRS], pc_full[GPS], pc_empty[GPS], acc_full[2], acc_empty[2], drained;
    unsigned taddr;
    int err;
};

constexpr int kSmem = 1024 + GRS * kRawBytes + GPS * kPieceBytes + (int)sizeof(GramShared);

struct GramParams {
    int64_t nrows, rows_per_split;
    int n, nt, full, stage_chunks;
    double* Qpart;
    Control* ctl;
    uint64_t timeout_ns;
};

__device__ __forceinline__ unsigned short bf(float x) { return __bfloat16_as_ushort(__float2bfloat16(x)); }
__device__ __forceinline__ float fb(unsigned short h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

__global__ void __launch_bounds__(kThreads, 1) gram_tc05_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, GramParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* raw = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // GRS x kRawBytes
    unsigned char* pcs = raw + GRS * kRawBytes;                                           // GPS x kPieceBytes
    GramShared* sh = reinterpret_cast<GramShared*>(pcs + GPS * kPieceBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    int kb = 0, mb = 0;
    if (p.full) {
        kb = blockIdx.x / p.nt;
        mb = blockIdx.x % p.nt;
    } else {
        int t = blockIdx.x;
        while (t >= p.nt - kb) t -= p.nt - kb, ++kb;
        mb = kb + t;
    }
    const int64_t j0 = (int64_t)blockIdx.y * p.rows_per_split;
    const int64_t j1 = min(j0 + p.rows_per_split, p.nrows);
    const int nchunks = j1 > j0 ? (int)((j1 - j0 + GK - 1) / GK) : 0;
    const int nstages = (nchunks + p.stage_chunks - 1) / p.stage_chunks;

    if (tid == 0) {
        for (int q = 0; q < GRS; ++q) mbar_init(&sh->raw_full[q], 1), mbar_init(&sh->raw_empty[q], kConv);
        for (int q = 0; q < GPS; ++q) mbar_init(&sh->pc_full[q], kConv), mbar_init(&sh->pc_empty[q], 1);
        for (int q = 0; q < 2; ++q) mbar_init(&sh->acc_full[q], 1), mbar_init(&sh->acc_empty[q], kEpi);
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
        // ---------------- loader (TMA): chunk g of A and of B into raw stage g % GRS
        if (lane == 0) {
            int g = 0;
            for (; g < nchunks; ++g) {
                const int rs = g % GRS;
                if (g >= GRS &&
                    !mbar_wait(&sh->raw_empty[rs], (unsigned)((g / GRS - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                    break;
                mbar_expect_tx(&sh->raw_full[rs], kRawBytes);
                const int x = (int)(j0 + (int64_t)g * GK);
                tma_load_2d(raw + rs * kRawBytes, &tmA, x, kb * GM, &sh->raw_full[rs]);
                tma_load_2d(raw + rs * kRawBytes + kRawOp, &tmB, x, mb * GM, &sh->raw_full[rs]);
            }
            // every issued copy has landed before the CTA may exit
            for (int f = g - 1; f >= 0 && f >= g - GRS; --f)
                mbar_drain(&sh->raw_full[f % GRS], (unsigned)((f / GRS) & 1), p.timeout_ns);
        }
    } else if (warp >= 8 && warp < 16) {
        // ---------------- converters: thread (operand op, member r) splits its 32 values
        const int ct = tid - kEpi;
        const int op = ct >> 7, r = ct & (GM - 1);
        for (int g = 0; g < nchunks; ++g) {
            const int s = g % GPS, rs = g % GRS;
            if (g >= GPS && !mbar_wait(&sh->pc_empty[s], (unsigned)((g / GPS - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                break;
            if (!mbar_wait(&sh->raw_full[rs], (unsigned)((g / GRS) & 1), &sh->err, p.ctl, p.timeout_ns)) break;
            // member r's row of 128 bytes; 16-byte chunk c sits at c ^ (r % 8) (128-byte swizzle)
            const unsigned char* row = raw + rs * kRawBytes + op * kRawOp + r * 128;
            float v[GK];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 q = *reinterpret_cast<const float4*>(row + ((c ^ (r & 7)) << 4));
                v[4 * c] = q.x, v[4 * c + 1] = q.y, v[4 * c + 2] = q.z, v[4 * c + 3] = q.w;
            }
            release_to_async(&sh->raw_empty[rs]);
            unsigned char* dst = pcs + s * kPieceBytes + op * 3 * kPieceOp + (r >> 3) * 256 + (r & 7) * 16;
#pragma unroll
            for (int k8 = 0; k8 < 4; ++k8) {       // rows 8 k8 .. 8 k8 + 7: K-step k8 / 2, core k8 % 2
                uint32_t h[4], m[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    unsigned short hh[2], mm[2], ll[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float x = v[8 * k8 + 2 * q + e];
                        hh[e] = bf(x);
                        const float r1 = x - fb(hh[e]);
                        mm[e] = bf(r1);
                        ll[e] = bf(r1 - fb(mm[e]));
                    }
                    h[q] = hh[0] | ((uint32_t)hh[1] << 16);
                    m[q] = mm[0] | ((uint32_t)mm[1] << 16);
                    l[q] = ll[0] | ((uint32_t)ll[1] << 16);
                }
                const int off = (k8 >> 1) * kStepBytes + (k8 & 1) * 128;
                *reinterpret_cast<uint4*>(dst + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(dst + kPieceOp + off) = make_uint4(m[0], m[1], m[2], m[3]);
                *reinterpret_cast<uint4*>(dst + 2 * kPieceOp + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(&sh->pc_full[s]);
        }
    } else if (warp < 8) {
        // ---------------- epilogue: stage sums into hi + lo (TwoSum), then the partial Gram
        const int quarter = warp & 3, half = warp >> 2;
        const unsigned lanes = tbase + ((unsigned)(quarter * 32) << 16);
        // strict upper triangle of a diagonal tile: column groups left of this warp's 32 rows
        // (every m < every k) are not needed -- 12 of the 32 groups
        const int cskip = (!p.full && kb == mb) ? quarter * 32 : 0;
        bool ok = true;
        for (int g = 0; ok && g < nstages; ++g) {   // g: stage
            const int b = g & 1;
            if (!mbar_wait(&sh->acc_full[b], (unsigned)((g >> 1) & 1), &sh->err, p.ctl, p.timeout_ns)) {
                ok = false;
                break;
            }
            fence_after();
#pragma unroll 1
            for (int c16 = 0; c16 < 4; ++c16) {
                const unsigned col = (unsigned)(half * 64 + c16 * 16);
                if ((int)col + 16 <= cskip) continue;
                unsigned acc[16], hi[16], lo[16];
                tmem_ld16(lanes + (unsigned)(b * GM) + col, acc);
                if (g > 0) {
                    tmem_ld16(lanes + 256u + col, hi);
                    tmem_ld16(lanes + 384u + col, lo);
                }
                tmem_wait_ld(acc);
                if (g > 0) {
                    reg_fence16(hi);
                    reg_fence16(lo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float a = g > 0 ? __uint_as_float(hi[q]) : 0.f;
                    const float x = __uint_as_float(acc[q]);
                    const float s = a + x;
                    const float xx = s - a;
                    const float e = (a - (s - xx)) + (x - xx);
                    hi[q] = __float_as_uint(s);
                    lo[q] = __float_as_uint((g > 0 ? __uint_as_float(lo[q]) : 0.f) + e);
                }
                tmem_st16(lanes + 256u + col, hi);
                tmem_st16(lanes + 384u + col, lo);
                tmem_wait_st();   // before the next group's loads reuse the source registers
            }
            fence_before();
            mbar_arrive(&sh->acc_empty[b]);
        }
        if (ok) {
            // this thread's row k of the tile, columns half * 64 ..: Qpart[slice][k][m]
            double* out = p.Qpart + (int64_t)blockIdx.y * p.n * p.n;
            const int k = kb * GM + quarter * 32 + lane;
#pragma unroll 1
            for (int c16 = 0; c16 < 4; ++c16) {
                const unsigned col = (unsigned)(half * 64 + c16 * 16);
                if ((int)col + 16 <= cskip) continue;
                unsigned hi[16], lo[16];
                if (nstages > 0) {
                    tmem_ld16(lanes + 256u + col, hi);
                    tmem_ld16(lanes + 384u + col, lo);
                    tmem_wait_ld(hi);
                    reg_fence16(lo);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int m = mb * GM + (int)col + q;
                    if (k < p.n && m < p.n && (p.full || k < m))
                        out[(int64_t)k * p.n + m] =
                            nstages > 0 ? (double)__uint_as_float(hi[q]) + (double)__uint_as_float(lo[q]) : 0.0;
                }
            }
        }
    } else {
        // ---------------- MMA issue (warp 17, one thread)
        if (lane == 0) {
            const unsigned idesc = instr_desc(GM, GM);
            // products a_i b_j, i + j < 3, smallest first
            const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
            for (int g = 0; g < nchunks; ++g) {
                const int st = g / p.stage_chunks, first = (g % p.stage_chunks) == 0;
                const int b = st & 1, s = g % GPS;
                if (first && st >= 2 &&
                    !mbar_wait(&sh->acc_empty[b], (unsigned)(((st >> 1) - 1) & 1), &sh->err, p.ctl, p.timeout_ns))
                    break;
                if (!mbar_wait(&sh->pc_full[s], (unsigned)((g / GPS) & 1), &sh->err, p.ctl, p.timeout_ns)) break;
                fence_after();
                const unsigned char* pa0 = pcs + s * kPieceBytes;
                const unsigned char* pb0 = pa0 + 3 * kPieceOp;
                const unsigned d = tbase + (unsigned)(b * GM);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        mma_bf16(d, smem_desc(pa0 + pa[q] * kPieceOp + ks * kStepBytes),
                                 smem_desc(pb0 + pb[q] * kPieceOp + ks * kStepBytes), idesc, !first || (ks | q) != 0);
                mma_commit(&sh->pc_empty[s]);
                if (g % p.stage_chunks == p.stage_chunks - 1 || g == nchunks - 1) mma_commit(&sh->acc_full[b]);
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

}  // namespace

cudaError_t gram_tc05(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                      double* Qpart, int32_t nsplit, int full, int stage_chunks, Control* ctl, uint64_t timeout_ns,
                      cudaStream_t s, int32_t* used) {
    CUtensorMap tmA, tmB;
    memset(&tmA, 0, sizeof(tmA));
    memset(&tmB, 0, sizeof(tmB));
    if (nrows < 1 || n < 1 || !encode_f32_2d(&tmA, A, nrows, n, lda, GK, GM, true) ||
        !encode_f32_2d(&tmB, B, nrows, n, ldb, GK, GM, true))
        return cudaErrorNotSupported;
    const int nt = (n + GM - 1) / GM;
    const int tiles = full ? nt * nt : nt * (nt + 1) / 2;
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
    rps = (rps + GK - 1) / GK * GK;
    if ((e = cudaFuncSetAttribute(gram_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)) != cudaSuccess)
        return e;
    GramParams p;
    p.nrows = nrows;
    p.rows_per_split = rps;
    p.n = n;
    p.nt = nt;
    p.full = full;
    p.stage_chunks = stage_chunks < 1 ? 1 : stage_chunks;
    p.Qpart = Qpart;
    p.ctl = ctl;
    p.timeout_ns = timeout_ns;
    *used = nsplit;
    void* args[] = {&tmA, &tmB, &p};
    return cudaLaunchKernel((const void*)gram_tc05_kernel, dim3((unsigned)tiles, (unsigned)nsplit), dim3(kThreads),
                            args, kSmem, s);
}

}  // namespace enkf
