// X_A = X_B + dX_B M (the SMEnKF analysis update, Sec. 3.1) on the fifth-generation
// tensor cores (with an optional divisor per row -- a product by its reciprocal -- the same
// kernel forms the scaled refinement residual (T - V P) / r): tcgen05.mma with BF16 operands split into pieces,
// x = hi + lo (three products hi*hi + hi*lo + lo*hi; operands kept to ~2^-17) or
// x = hi + mid + lo (six products with i + j < 3; ~2^-25, FP32-class), FP32 accumulators in
// TMEM.
//
// Persistent, warp-specialised CTA, one per SM; a tile is 128 state rows x NB members:
//   warp 16     loader: TMA tensor copies of the FP32 dX_B chunk (128 rows x 32 members)
//               into a ring of raw slots (mbarrier transaction counts).
//   warps 8-15  converters: raw FP32 -> BF16 hi/lo in the K-major canonical layout of
//               the MMA (core matrices of 8 rows x 16 bytes; LBO 128 B along K, SBO 256 B
//               along rows) in a ring of operand slots.  Without TMA (unaligned dX_B)
//               they read dX_B from global memory themselves.
//   warp 17     TMEM allocation and the MMA issue (one thread): 2 K-steps x 3 products
//               per chunk; tcgen05.commit frees the operand slot, and after a tile's last
//               chunk marks its accumulator full.  Two accumulators in TMEM.
//   warps 0-7   epilogue: warp w reads TMEM lanes 32 (w % 4).. (its 32 rows) for one
//               half of the columns; X_A = X_B + acc with coalesced column accesses.
//   warp 18     X_B loader (a TMA-aligned X_B): TMA copies of the column block's X_B
//               chunks (128 rows x 32 members) of every tile, in order, into a four-slot
//               ring the epilogue reads, so the epilogue waits on no global load; the two
//               halves of the epilogue then take alternate chunks (one consumer per fill).
// M is pre-split into hi/lo images of the same layout; they stay in shared memory for
// the whole launch when they fit (Nens <= 128), else each chunk's part travels in the
// operand slot.  Every mbarrier wait is bounded (iteration count and %globaltimer); on
// expiry the CTA latches ENKF_ERR_TIMEOUT, drains its copies and MMAs with bounded
// waits, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"
#include "tc05.cuh"

namespace enkf {
namespace {

constexpr int XM = 128;     // rows per tile (MMA M)
constexpr int XKC = 32;     // K per chunk: two MMA K-steps of 16
constexpr int XRS = 4;      // raw (FP32) slots
constexpr int XBS = 4;      // X_B slots (one tile of Nens <= 128)
constexpr int XNMAX = 256;  // largest MMA N
constexpr int kEpi = 256, kConv = 256;
constexpr int kThreads = kEpi + kConv + 96;    // + loader warp + MMA warp + X_B loader warp
constexpr int kRawBytes = XM * XKC * 4;        // one raw chunk
__host__ __device__ constexpr int a_bytes(int np) { return np * XM * XKC * 2; }   // A pieces of one chunk
constexpr int kMaxSmem = 232448;

__host__ __device__ constexpr int b_chunk_bytes(int nb, int np) { return np * nb * XKC * 2; }   // B pieces of one chunk

struct XaShared {
    uint64_t raw_full[XRS], raw_empty[XRS], a_full[4], a_empty[4], acc_full[2], acc_empty[2], drained;
    uint64_t xb_full[XBS], xb_empty[XBS];
    unsigned taddr;
    int err;
};

using tc05::fence_after;
using tc05::fence_before;
using tc05::mbar_arrive;
using tc05::mbar_drain;
using tc05::mbar_expect_tx;
using tc05::mbar_init;
using tc05::smem_u32;
using tc05::tmem_ld16;
using tc05::tmem_wait_ld;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, XaShared* sh, Control* ctl,
                                          uint64_t timeout_ns) {
    return tc05::mbar_wait(bar, parity, &sh->err, ctl, timeout_ns);
}
__device__ __forceinline__ uint64_t smem_desc(const void* p) { return tc05::smem_desc(p); }
__device__ __forceinline__ unsigned instr_desc(int n) { return tc05::instr_desc(XM, n); }
__device__ __forceinline__ void mma_bf16(unsigned d, uint64_t a, uint64_t b, unsigned idesc, int acc) {
    tc05::mma_bf16(d, a, b, idesc, acc);
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) { tc05::mma_commit(bar); }
__device__ __forceinline__ void tc_fence_before() { fence_before(); }
__device__ __forceinline__ void tc_fence_after() { fence_after(); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// 8 consecutive k of one row -> the NP pieces' 16-byte rows of their core matrices: piece q
// is the BF16 rounding of what pieces 0..q-1 leave (the subtractions are exact in FP32).
template <int NP>
__device__ __forceinline__ void put_row8(unsigned char* ahi, int off, const float* v) {
    float rest[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rest[q] = v[q];
#pragma unroll
    for (int pc = 0; pc < NP; ++pc) {
        uint4 h;
        h.x = pack_bf16(rest[0], rest[1]);
        h.y = pack_bf16(rest[2], rest[3]);
        h.z = pack_bf16(rest[4], rest[5]);
        h.w = pack_bf16(rest[6], rest[7]);
        *reinterpret_cast<uint4*>(ahi + pc * XM * XKC * 2 + off) = h;
        if (pc + 1 < NP) {
            const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&h);
#pragma unroll
            for (int q = 0; q < 8; ++q) rest[q] = rest[q] - __bfloat162float(hb[q]);
        }
    }
}

struct XaParams {
    int64_t nstate;
    int nens, nb, nchunks, alloc_cols, nas, resident, xbt;
    const float* XB;
    int64_t ldb;
    const float* dXB;
    int64_t ldx;
    const uint4* Mimg;
    float* XA;
    int64_t lda;
    const float* rdiv;   // nullable: row i of the result is divided by rdiv[i]
    Control* ctl;
    uint64_t timeout_ns;
};

template <bool TMA, int NP>
__global__ void __launch_bounds__(kThreads, 1) xa_tc05_kernel(const __grid_constant__ CUtensorMap tmap,
                                                              const __grid_constant__ CUtensorMap tmapb, XaParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nb = p.nb, nchunks = p.nchunks, nas = p.nas;
    constexpr int kABytes = a_bytes(NP);
    const int aslot = kABytes + (p.resident ? 0 : b_chunk_bytes(nb, NP));
    // 1024-byte aligned working area (the launch reserves 1 KB of slack for this)
    unsigned char* raw = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // XRS x kRawBytes
    unsigned char* xbs = raw + XRS * kRawBytes;                      // XBS x kRawBytes when p.xbt
    unsigned char* aring = xbs + (p.xbt ? XBS * kRawBytes : 0);     // nas x aslot
    unsigned char* bres = aring + nas * aslot;                       // resident B images
    XaShared* sh = reinterpret_cast<XaShared*>(bres + (p.resident ? nchunks * b_chunk_bytes(nb, NP) : 0));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int yb = blockIdx.y;
    const int64_t ntiles = (p.nstate + XM - 1) / XM;

    if (tid == 0) {
        for (int q = 0; q < XRS; ++q) mbar_init(&sh->raw_full[q], 1), mbar_init(&sh->raw_empty[q], kConv);
        for (int q = 0; q < nas; ++q) mbar_init(&sh->a_full[q], kConv), mbar_init(&sh->a_empty[q], 1);
        for (int q = 0; q < 2; ++q) mbar_init(&sh->acc_full[q], 1), mbar_init(&sh->acc_empty[q], kEpi);
        for (int q = 0; q < XBS; ++q) mbar_init(&sh->xb_full[q], 1), mbar_init(&sh->xb_empty[q], kEpi / 2);
        mbar_init(&sh->drained, 1);
        sh->err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 17) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sh->taddr)),
                     "r"(p.alloc_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tbase = sh->taddr;

    if (warp == 16) {
        // ---------------- loader (TMA)
        if (TMA && lane == 0) {
            int64_t g = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int rs = (int)(g % XRS);
                    if (g >= XRS && !mbar_wait(&sh->raw_empty[rs], (unsigned)((g / XRS - 1) & 1), sh, p.ctl,
                                               p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&sh->raw_full[rs], kRawBytes);
                    const int x = (int)(tile * XM), y = c * XKC;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                        "{%2, %3}], [%4];\n" ::"r"(smem_u32(raw + rs * kRawBytes)),
                        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x), "r"(y), "r"(smem_u32(&sh->raw_full[rs]))
                        : "memory");
                }
            }
            // every issued copy has landed before the CTA may exit
            for (int64_t f = g - 1; f >= 0 && f >= g - XRS; --f)   // the last fill of each slot
                mbar_drain(&sh->raw_full[f % XRS], (unsigned)((f / XRS) & 1), p.timeout_ns);
        }
    } else if (warp >= 8 && warp < 16) {
        // ---------------- converters
        const int ct = tid - kEpi;
        const int r = ct & (XM - 1), kh = ct >> 7;     // row, half of the chunk's 32 k
        if (p.resident) {
            const uint4* src = p.Mimg + (int64_t)yb * nchunks * (b_chunk_bytes(nb, NP) / 16);
            uint4* dst = reinterpret_cast<uint4*>(bres);
            for (int q = ct; q < nchunks * b_chunk_bytes(nb, NP) / 16; q += kConv) dst[q] = __ldg(src + q);
        }
        int64_t g = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const int64_t i = tile * XM + r;
            for (int c = 0; c < nchunks; ++c, ++g) {
                const int s = (int)(g % nas), rs = (int)(g % XRS);
                if (g >= nas && !mbar_wait(&sh->a_empty[s], (unsigned)((g / nas - 1) & 1), sh, p.ctl, p.timeout_ns)) {
                    ok = false;
                    break;
                }
                float v[16];
                if (TMA) {
                    if (!mbar_wait(&sh->raw_full[rs], (unsigned)((g / XRS) & 1), sh, p.ctl, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const float* rw = reinterpret_cast<const float*>(raw + rs * kRawBytes);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = rw[(kh * 16 + q) * XM + r];
                    tc05::release_to_async(&sh->raw_empty[rs]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int k = c * XKC + kh * 16 + q;
                        v[q] = (i < p.nstate && k < p.nens) ? __ldg(p.dXB + (int64_t)k * p.ldx + i) : 0.f;
                    }
                }
                unsigned char* slot = aring + s * aslot;
                // K-step kh, k-groups 0 and 1: core (r / 8, kg), row r % 8
                const int off = kh * (XM * 32) + (r >> 3) * 256 + (r & 7) * 16;
                put_row8<NP>(slot, off, v);
                put_row8<NP>(slot, off + 128, v + 8);
                if (!p.resident) {
                    const uint4* src = p.Mimg + ((int64_t)yb * nchunks + c) * (b_chunk_bytes(nb, NP) / 16);
                    uint4* dst = reinterpret_cast<uint4*>(slot + kABytes);
                    for (int q = ct; q < b_chunk_bytes(nb, NP) / 16; q += kConv) dst[q] = __ldg(src + q);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(&sh->a_full[s]);
            }
        }
    } else if (warp < 8) {
        // ---------------- epilogue
        const int quarter = warp & 3, half = warp >> 2;
        const int ngroups = nb / 16;
        const int g0 = half ? (ngroups + 1) / 2 : 0, g1 = half ? ngroups : (ngroups + 1) / 2;
        const int nxc = (ngroups + 1) / 2;   // X_B chunks of a tile (two groups of 16 members each)
        int64_t t = 0;
        auto load_xb = [&](int64_t i, int gq, float* xb) {
            const int e0 = yb * nb + gq * 16;
#pragma unroll
            for (int q = 0; q < 16; ++q)
                xb[q] = (i < p.nstate && e0 + q < p.nens) ? p.XB[(int64_t)(e0 + q) * p.ldb + i] : 0.f;
        };
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            const int b = (int)(t & 1);
            const int64_t i = tile * XM + quarter * 32 + lane;
            if (p.xbt) {
                if (!mbar_wait(&sh->acc_full[b], (unsigned)((t >> 1) & 1), sh, p.ctl, p.timeout_ns)) break;
                tc_fence_after();
                const unsigned row_addr = tbase + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * nb);
                bool ok = true;
                for (int c = half; c < nxc; c += 2) {
                    // X_B chunk c: members yb nb + 32 c .., [member][row]; ring fill G
                    const int64_t G = t * nxc + c;
                    const int slot = (int)(G % XBS);
                    if (!mbar_wait(&sh->xb_full[slot], (unsigned)((G / XBS) & 1), sh, p.ctl, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const float* xs = reinterpret_cast<const float*>(xbs + slot * kRawBytes) + quarter * 32 + lane;
                    for (int h = 0; h < 2 && 2 * c + h < ngroups; ++h) {
                        const int gq = 2 * c + h;
                        unsigned acc[16];
                        tmem_ld16(row_addr + gq * 16, acc);
                        float xb[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) xb[q] = xs[(h * 16 + q) * XM];
                        tmem_wait_ld(acc);
                        const int e0 = yb * nb + gq * 16;
                        if (i < p.nstate) {
                            // one reciprocal per row; a product by exactly 1 when there is no divisor
                            const float rinv = p.rdiv ? 1.0f / p.rdiv[i] : 1.0f;
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                if (e0 + q < p.nens)
                                    p.XA[(int64_t)(e0 + q) * p.lda + i] = (xb[q] + __uint_as_float(acc[q])) * rinv;
                        }
                    }
                    tc05::release_to_async(&sh->xb_empty[slot]);
                }
                if (!ok) break;
                tc_fence_before();
                mbar_arrive(&sh->acc_empty[b]);
                continue;
            }
            // X_B does not depend on the MMAs: the first group's loads are issued before the wait,
            // and each later group's one group ahead of its use
            float xnext[16];
            if (g0 < g1) load_xb(i, g0, xnext);
            if (!mbar_wait(&sh->acc_full[b], (unsigned)((t >> 1) & 1), sh, p.ctl, p.timeout_ns)) break;
            tc_fence_after();
            const unsigned row_addr = tbase + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * nb);
            for (int gq = g0; gq < g1; ++gq) {
                float xb[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) xb[q] = xnext[q];
                if (gq + 1 < g1) load_xb(i, gq + 1, xnext);
                unsigned acc[16];
                tmem_ld16(row_addr + gq * 16, acc);
                tmem_wait_ld(acc);
                const int e0 = yb * nb + gq * 16;
                if (i < p.nstate) {
                    const float rinv = p.rdiv ? 1.0f / p.rdiv[i] : 1.0f;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (e0 + q < p.nens)
                            p.XA[(int64_t)(e0 + q) * p.lda + i] = (xb[q] + __uint_as_float(acc[q])) * rinv;
                }
            }
            tc_fence_before();
            mbar_arrive(&sh->acc_empty[b]);
        }
    } else if (warp == 18) {
        // ---------------- X_B loader (TMA): fill G = (tile count) x nxc + c into slot G % XBS
        if (TMA && p.xbt && lane == 0) {
            const int nxc = (nb / 16 + 1) / 2;
            int64_t G = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                for (int c = 0; c < nxc; ++c, ++G) {
                    const int slot = (int)(G % XBS);
                    if (G >= XBS && !mbar_wait(&sh->xb_empty[slot], (unsigned)((G / XBS - 1) & 1), sh, p.ctl,
                                               p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&sh->xb_full[slot], kRawBytes);
                    tc05::tma_load_2d(xbs + slot * kRawBytes, &tmapb, (int)(tile * XM), yb * nb + c * XKC,
                                      &sh->xb_full[slot]);
                }
            }
            // every issued copy has landed before the CTA may exit (the last fill of each slot)
            for (int64_t f = G - 1; f >= 0 && f >= G - XBS; --f)
                mbar_drain(&sh->xb_full[f % XBS], (unsigned)((f / XBS) & 1), p.timeout_ns);
        }
    } else {
        // ---------------- MMA issue (warp 17, one thread)
        if (lane == 0) {
            const unsigned idesc = instr_desc(nb);
            int64_t g = 0, t = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++t) {
                const int b = (int)(t & 1);
                if (t >= 2 && !mbar_wait(&sh->acc_empty[b], (unsigned)(((t >> 1) - 1) & 1), sh, p.ctl, p.timeout_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned dcol = tbase + (unsigned)(b * nb);
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int s = (int)(g % nas);
                    if (!mbar_wait(&sh->a_full[s], (unsigned)((g / nas) & 1), sh, p.ctl, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* a0 = aring + s * aslot;
                    const unsigned char* b0 = p.resident ? bres + c * b_chunk_bytes(nb, NP) : a0 + kABytes;
                    // products of pieces (i, j) with i + j < NP, smallest first
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const int aoff = ks * XM * 32, boff = ks * nb * 32;
                        const int first = (c == 0 && ks == 0);
                        int q = 0;
#pragma unroll
                        for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
                            for (int i = sum; i >= 0; --i, ++q)
                                mma_bf16(dcol, smem_desc(a0 + i * XM * XKC * 2 + aoff),
                                         smem_desc(b0 + (sum - i) * nb * XKC * 2 + boff), idesc,
                                         (first && q == 0) ? 0 : 1);
                    }
                    mma_commit(&sh->a_empty[s]);
                }
                if (!ok) break;
                mma_commit(&sh->acc_full[b]);
            }
            // the commit arrives once every MMA issued above has completed
            mma_commit(&sh->drained);
            mbar_drain(&sh->drained, 0u, p.timeout_ns);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 17) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(p.alloc_cols)
                     : "memory");
    }
}

// M (column-major [k + e n]) -> the per-chunk canonical images: for column block yb
// and chunk c, the np pieces in turn, each [ks][n / 8][kg][n % 8][8 k] of BF16.
__global__ void xa_tc05_image_kernel(const float* __restrict__ M, int n, int nb, int nblocks, int nchunks, int np,
                                     __nv_bfloat16* __restrict__ img) {
    const int64_t per = (int64_t)nb * XKC;               // elements of one hi (or lo) chunk
    const int64_t total = (int64_t)nblocks * nchunks * per;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = q / per;                     // yb * nchunks + c
        const int rem = (int)(q % per);
        const int yb = (int)(blk / nchunks), c = (int)(blk % nchunks);
        const int ks = rem / (nb * 16), r2 = rem % (nb * 16);
        const int ng = r2 / 128, r3 = r2 % 128;
        const int kg = r3 / 64, r4 = r3 % 64;
        const int rn = r4 / 8, kk = r4 % 8;
        const int e = yb * nb + ng * 8 + rn;             // member (column of X_A)
        const int k = c * XKC + ks * 16 + kg * 8 + kk;   // member of dX_B (row of M)
        float rest = (e < n && k < n) ? M[k + (int64_t)e * n] : 0.f;
        for (int pc = 0; pc < np; ++pc) {
            const __nv_bfloat16 h = __float2bfloat16(rest);
            img[blk * np * per + pc * per + rem] = h;
            rest = rest - __bfloat162float(h);
        }
    }
}

struct XaGeom {
    int nb, nblocks, nchunks, alloc, nas, resident, smem;
};

XaGeom xa_geom(int32_t nens, bool xbt, int np) {
    XaGeom g;
    const int nfirst = nens < XNMAX ? nens : XNMAX;
    g.nb = (nfirst + 15) / 16 * 16;
    g.nblocks = (nens + g.nb - 1) / g.nb;
    g.nchunks = (nens + XKC - 1) / XKC;
    int alloc = 32;
    while (alloc < 2 * g.nb) alloc *= 2;
    g.alloc = alloc;
    g.resident = g.nchunks * b_chunk_bytes(g.nb, np) <= 65536;
    const int aslot = a_bytes(np) + (g.resident ? 0 : b_chunk_bytes(g.nb, np));
    const int fixed = (XRS + (xbt ? XBS : 0)) * kRawBytes + (g.resident ? g.nchunks * b_chunk_bytes(g.nb, np) : 0) +
                      (int)sizeof(XaShared) + 1024;
    g.nas = (kMaxSmem - fixed) / aslot;
    if (g.nas > 4) g.nas = 4;
    g.smem = fixed + g.nas * aslot;
    // one CTA per SM (the two accumulators may take all 512 TMEM columns)
    if (g.smem < kMaxSmem / 2 + 1024) g.smem = kMaxSmem / 2 + 1024;
    return g;
}

}  // namespace

bool encode_f32_2d(CUtensorMap* map, const float* base, int64_t inner, int64_t outer, int64_t ld, int box_inner,
                   int box_outer, bool swizzle128) {
    if ((uintptr_t)base % 16 != 0 || (ld * 4) % 16 != 0 || inner >= (int64_t(1) << 31)) return false;
    // resolved through the runtime so the library has no link-time dependency on libcuda
    using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<EncodeTiled>(f);
    }
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t xa_split_bytes(int32_t nens) {
    const XaGeom g = xa_geom(nens, false, 3);   // room for the three-piece images
    return (size_t)g.nblocks * g.nchunks * b_chunk_bytes(g.nb, 3);
}

cudaError_t xa_update_tc05(int64_t nstate, int32_t nens, const float* XB, int64_t ldb, const float* dXB, int64_t ldx,
                           const float* M, void* msplit, float* XA, int64_t lda, const float* rdiv, int pieces,
                           Control* ctl, uint64_t timeout_ns, cudaStream_t s) {
    const int np = pieces == 3 ? 3 : 2;
    XaGeom g = xa_geom(nens, false, np);
    if (g.nas < 2) return cudaErrorInvalidConfiguration;
    {
        const int64_t total = (int64_t)g.nblocks * g.nchunks * g.nb * XKC;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        xa_tc05_image_kernel<<<blocks, 256, 0, s>>>(M, nens, g.nb, g.nblocks, g.nchunks, np,
                                                     static_cast<__nv_bfloat16*>(msplit));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // TMA tensor maps of dX_B and X_B (rows inner, members outer), box 128 rows x 32 members;
    // the rows and members past the end read as zeros.  Each needs a 16-byte aligned base and
    // stride; with an unaligned X_B (or no room for its ring) the epilogue loads it from global
    // memory.
    CUtensorMap tmap, tmapb;
    memset(&tmap, 0, sizeof(tmap));
    memset(&tmapb, 0, sizeof(tmapb));
    const bool tma = encode_f32_2d(&tmap, dXB, nstate, nens, ldx, XM, XKC, false);
    bool xbt = tma && encode_f32_2d(&tmapb, XB, nstate, nens, ldb, XM, XKC, false);
    if (xbt) {
        const XaGeom gx = xa_geom(nens, true, np);
        if (gx.nas >= 2) g = gx;
        else xbt = false;
    }
    const void* fn = np == 3 ? (tma ? (const void*)xa_tc05_kernel<true, 3> : (const void*)xa_tc05_kernel<false, 3>)
                             : (tma ? (const void*)xa_tc05_kernel<true, 2> : (const void*)xa_tc05_kernel<false, 2>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t ntiles = (nstate + XM - 1) / XM;
    int64_t gx = (int64_t)nsm / g.nblocks;
    if (gx < 1) gx = 1;
    if (gx > ntiles) gx = ntiles;
    XaParams p;
    p.nstate = nstate;
    p.nens = nens;
    p.nb = g.nb;
    p.nchunks = g.nchunks;
    p.alloc_cols = g.alloc;
    p.nas = g.nas;
    p.resident = g.resident;
    p.xbt = xbt ? 1 : 0;
    p.XB = XB;
    p.ldb = ldb;
    p.dXB = dXB;
    p.ldx = ldx;
    p.Mimg = static_cast<const uint4*>(msplit);
    p.XA = XA;
    p.lda = lda;
    p.rdiv = rdiv;
    p.ctl = ctl;
    p.timeout_ns = timeout_ns;
    void* args[] = {&tmap, &tmapb, &p};
    return cudaLaunchKernel(fn, dim3((unsigned)gx, (unsigned)g.nblocks), dim3(kThreads), args, g.smem, s);
}

}  // namespace enkf
