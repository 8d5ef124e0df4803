// Panel form of the iterative Sherman-Morrison solve with the trailing update and the
// panel dots on the fifth-generation tensor cores (tcgen05.mma, TMEM accumulators, TMA).
//
// The recurrence is that of the CUDA-core panel kernel (b levels of Step 2, eqs.
// SM-step-2-h/Z/u, regrouped): for a panel P = {k0..k0+b-1} with the dots A = V_P^T X of
// the trailing columns X = [u_{k0+b..N-1}, z_0..z_{N-1}] (reduced across CTAs) and the
// panel Gram G = V_P^T U_P, every CTA factors G (FP64-class gamma, as there), forms
// K = -W A and sweeps its rows:
//     X <- X + U_P K               (MMA1: M = 128 rows, N = 128 columns, K = b)
//     A' += V_{P'}^T X_new         (MMA2: M = 128 columns, N = b, K = 32 rows per slice)
//     u_m <- U_P beta_m (m in P)   (MMA3: the panel's own final columns, N = b)
// Every product is formed from three BF16 pieces per FP32 value (x = hi + mid + lo, kept
// to ~2^-25) as the six products with i + j < 3, smallest first, accumulated in FP32.
// Each MMA's sum starts from zero and is added to FP32 afterwards (the tensor cores'
// accumulation truncates): the update is added to X by the epilogue, the dots of every
// 128-row tile are folded into FP32 registers.
//
// Data flow of one sweep, per CTA (one per SM; the CTA owns a block of 128-row tiles):
//   column chunks of 128 trailing columns (U part and Z part apart), and within a chunk
//   every tile of the CTA:
//   - X: eight epilogue warps, warp (q, h) for the 32-row quarter q of the tile and the
//     column half h, each with two slots of 32 rows x 32 columns FP32 (TMA, 128-byte
//     swizzle), refilled with the next tile's block as soon as the warp is done with it.
//   - U_P pieces and V_{P'} pieces: 24 KB per tile each (one buffer each), laid out in
//     global memory in the canonical K-major order of the MMA operands (written once per
//     panel by the previous sweep, or by the Step-1 pass for V) and brought in by one
//     bulk copy.
//   - K (and beta) pieces: computed per chunk by the whole CTA.
//   - per tile the epilogue warp (1) adds MMA1's TMEM accumulator to its slots, writes
//     X_new back to the slots and stores them with TMA, and releases D1; (2) waits for
//     its A-slice buffer (three buffers rotate over the four quarters); (3) converts its
//     rows into the pieces of MMA2's A operand (K-major: each column's 8 consecutive rows
//     in 16 bytes) and refills its slots; then writes the panel's final columns (MMA3)
//     and folds the previous tile's dots (MMA2's TMEM accumulator) into registers.
//   - warp 8 issues MMA1 and MMA3 and loads U_P; warp 9 issues MMA2 as each A slice
//     fills and loads V; each with its own commits.
// TMEM: D1 (MMA1, two buffers of 128 columns) at 0 and 128, D2 (MMA2, two buffers of 32)
// at 256 and 288, D3 (MMA3) at 320.
//
// The refinement's correction sweep runs in the same kernel (Tc5Args::refine): the solve
// keeps the pieces of every panel's final columns u_m and diag(1/gamma) (I + L)^-1, and the
// correction applies them to the columns of Z alone, with no factor and no U part.
//
// Every wait is bounded (iteration count and %globaltimer); on expiry the CTA latches
// ENKF_ERR_TIMEOUT, drains its copies and MMAs with bounded waits, frees TMEM and returns;
// the other CTAs then leave at their next grid barrier.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"
#include "panel_factor.cuh"
#include "tc05.cuh"

namespace enkf {
namespace {

using namespace tc05;

constexpr int TR = 128;              // rows per tile (MMA1 M)
constexpr int CW = 128;              // columns per chunk (MMA1 N, MMA2 M)
constexpr int SWC = 32;              // columns per X slot
constexpr int NQ = 4;                // epilogue warps (row quarters)
constexpr int NS = CW / SWC;         // slots per epilogue warp
constexpr int PB = 32;               // panel width (MMA2 N, MMA1 K)
constexpr int NH = 2;                // column groups of the epilogue warps
constexpr int NEPI = NQ * NH;        // epilogue warps: row quarter w % 4, column group w / 4
constexpr int NSW = NS / NH;         // X slots per epilogue warp
constexpr int kMmaWarp = NEPI, kAllocWarp = NEPI + 1;
constexpr int kThreads = 32 * (NEPI + 2);
constexpr int kSlotBytes = SWC * 32 * 4;          // 32 columns x 32 rows FP32 (4 KB)
constexpr int kPiece = TR * PB * 2;               // one BF16 piece of a 128 x 32 operand (8 KB)
constexpr int kOp3 = 3 * kPiece;                  // the three pieces (24 KB)
constexpr int kBeta3 = 3 * PB * PB * 2;           // beta pieces (6 KB)
constexpr unsigned kTmemCols = 512;
// D2: per buffer three blocks of PB columns, block j the products with V's piece j
constexpr unsigned kD2W = 3 * PB;
constexpr unsigned kD1 = 0, kD2 = 256, kD3 = kD2 + 2 * kD2W;
static_assert(kD3 + PB <= kTmemCols, "TMEM columns");

// shared-memory map (offsets from the 1024-byte aligned base); the control block first,
// 256-byte guard bands between the regions (filled with a pattern and checked after every
// chunk: a copy or a store that overruns its region is reported, not silently absorbed)
constexpr int kGuard = 256;
constexpr int kOffMisc = 0;
constexpr int kMiscBytes = 1024;
constexpr int kOffSlots = 2048;                                // 16 x 4 KB (1024-aligned for the swizzle)
constexpr int kNAs = 3;                                             // A-slice buffers
static_assert(kNAs == 3 && NQ == 4, "the A-slice buffer rotation below assumes 3 buffers, 4 quarters");
constexpr int kOffAs = kOffSlots + NQ * NS * kSlotBytes + kGuard;   // 3 x 24 KB   MMA2 A slices
constexpr int kOffVp = kOffAs + kNAs * kOp3 + kGuard;               // 24 KB       V_{P'} pieces
constexpr int kOffUp = kOffVp + kOp3 + kGuard;                      // 24 KB       U_P pieces
constexpr int kOffKp = kOffUp + kOp3 + kGuard;                      // 24 KB       K pieces
constexpr int kOffBp = kOffKp + kOp3 + kGuard;                      // 6 KB        beta pieces
constexpr int kOffW = kOffBp + kBeta3 + kGuard;                     // 4 KB        W (float)
constexpr int kEnd = kOffW + PB * PB * 4 + kGuard;
constexpr int kNGuard = 8;
__host__ __device__ constexpr int guard_off(int g) {
    return g == 0 ? kMiscBytes
                  : g == 1 ? kOffAs - kGuard
                           : g == 2 ? kOffVp - kGuard
                                    : g == 3 ? kOffUp - kGuard
                                             : g == 4 ? kOffKp - kGuard
                                                      : g == 5 ? kOffBp - kGuard : g == 6 ? kOffW - kGuard : kEnd - kGuard;
}
constexpr unsigned kGuardWord = 0xA5A5A5A5u;
constexpr int kSmem = 1024 + kEnd;
static_assert(kSmem <= 232448, "shared memory of one CTA");

struct Tc5Shared {
    uint64_t slot_full[NQ * NS];
    uint64_t up_full[2], up_empty[2], vp_full, vp_empty;
    uint64_t d1_full[2], d1_empty[2], d2_full[2], d2_empty[2], d3_full, d3_empty;
    // one pair per epilogue warp (one waiter and one signaller each, so that parity waits stay
    // in step); the two A-slice buffers are shared by warps q and q + 2
    uint64_t as_full[NQ], as_empty[NQ], drained_a, drained_b;
    double gam[PB];
    double red[32];
    unsigned taddr;
    int err;
    int flag[4];
    int prog[NEPI];    // progress of each epilogue warp (diagnostic): 16 tile + stage
};
static_assert(sizeof(Tc5Shared) <= kMiscBytes, "misc block");

// factor temporaries (alias the X slots, which are idle between sweeps)
struct FactorView {
    float* Gh;
    float* Gl;
    float* Bt;
    float* cb;
    float* Lt;
    float* W;
    float* Bf;
    double* gam;
};

struct Tc5Args {
    int64_t nobs;
    int32_t nens;
    int32_t ntiles;             // 128-row tiles of the whole problem
    int32_t tiles_per_blk;      // tiles owned by one CTA
    const float* r;
    float* U;
    int64_t ldu;
    float* Z;
    int64_t ldz;
    const unsigned char* vpc;   // V pieces: [panel][tile][24 KB]
    unsigned char* upc;         // U_P pieces: [2][tile][24 KB]
    double* part;               // per-CTA partial dots [cta][part_stride]
    int64_t part_stride;
    double* coefg;              // reduced dots
    double* C;                  // [N][N] Z coefficients
    double* gamma;              // [N]
    Control* ctl;
    int32_t check;
    uint64_t timeout_ns;
    // stored factors for a later correction sweep (both null: not kept)
    unsigned char* ufc;         // pieces of the final U columns of every panel: [panel][tile][24 KB]
    float* wfin;                // per panel diag(1/gamma) (I + L)^-1: [panel][32][32]
    int32_t refine;             // 1: apply the stored factors to Z (the correction sweep)
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }


// The three BF16 pieces of 8 values as three 16-byte rows (each the rounding of what the
// previous pieces leave; the subtractions are exact in FP32).
__device__ __forceinline__ void pieces8(const float* v, uint4* out) {
    float rest[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rest[q] = v[q];
#pragma unroll
    for (int pc = 0; pc < 3; ++pc) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // two values per conversion; the low half holds the first
            const __nv_bfloat162 h = __floats2bfloat162_rn(rest[2 * i], rest[2 * i + 1]);
            w[i] = *reinterpret_cast<const unsigned*>(&h);
            if (pc < 2) {
                rest[2 * i] = rest[2 * i] - __uint_as_float(w[i] << 16);
                rest[2 * i + 1] = rest[2 * i + 1] - __uint_as_float(w[i] & 0xffff0000u);
            }
        }
        out[pc] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Byte offset of (m, k) in a K-major canonical operand of rows m (blocks of 8 rows 256 B
// apart) and K = 32 (two K-steps of 16, kstep bytes apart; two 8-wide K-groups 128 B
// apart), for the 16-byte row of 8 consecutive k starting at k8 * 8.
__device__ __forceinline__ int kmaj_off(int m, int k8, int kstep_bytes) {
    return (k8 >> 1) * kstep_bytes + (m >> 3) * 256 + (k8 & 1) * 128 + (m & 7) * 16;
}

// Address of (column c, row j) in a 32 x 32 FP32 X slot written by TMA with the 128-byte
// swizzle: column c's 128-byte row holds rows 0..31, 16-byte chunk j / 4 at (j / 4) ^ (c % 8).
__device__ __forceinline__ float* slot_at(unsigned char* slot, int c, int j) {
    return reinterpret_cast<float*>(slot + c * 128 + ((((j >> 2) ^ (c & 7))) << 4) + (j & 3) * 4);
}

// Pipeline counters, identical in every thread: tiles with MMA1 (g1), with MMA2 (g2),
// with MMA3 (g3), and every tile (gt, for the slot phases).
struct Counters {
    unsigned g1, g2, g3, gt;
};

struct SweepSpec {
    int k0, bp;        // panel being applied (bp = 0: dots only)
    int k1;            // first trailing U column (N: none)
    int kv, nb;        // next panel: V columns kv.., nb of them (0: no dots)
    int aoff;          // offset of the trailing columns among the previous sweep's columns
    int ncols_prev;    // row stride of the previous sweep's reduced dots
    int mat;           // write the panel's final columns (MMA3)
    int up_par;        // parity of the U_P piece buffer holding panel P
    const unsigned char* upb;   // MMA1's A pieces of panel P, tile 0 ([tile][24 KB])
};

__device__ __forceinline__ unsigned char* tile_piece(const unsigned char* base, int64_t index) {
    return const_cast<unsigned char*>(base) + index * (int64_t)kOp3;
}

// Checks the guard bands; a corrupted band is recorded in the control block's diagnostic
// words (bit mask of bands, first bad word and its place).
__device__ void check_guards(const unsigned char* sm, Control* ctl) {
    for (int g = 0; g < kNGuard; ++g) {
        const volatile unsigned* w = reinterpret_cast<const volatile unsigned*>(sm + guard_off(g));
        for (int i = 0; i < kGuard / 4; ++i)
            if (w[i] != kGuardWord) {
                atomicOr(reinterpret_cast<unsigned*>(&ctl->pad[42]), 1u << g);
                if (atomicCAS(&ctl->pad[43], 0, (int)w[i]) == 0) ctl->pad[44] = g * 1000 + i;
                break;
            }
    }
}

// Phase timers (built only with -DENKF_TC5_TIMERS, for profiling): SM-clock cycles summed
// per CTA in the unused bytes between the first guard band and the X slots, then into a
// device array read by enkf_tc5_timers_read.  Entries 0..15: time in the waits of each
// site (lane 0 of the waiting warp); 16..: phases timed by thread 0 and the MMA thread.
enum { kTmK = 16, kTmEpi = 17, kTmEnd = 18, kTmRed = 19, kTmFac = 20, kTmAll = 21, kTmChunks = 22, kTmMma = 23,
       kTmStep1 = 24, kTmXup = 25, kTmConv = 26, kTmMat = 27, kTmFold = 28 };
#ifdef ENKF_TC5_TIMERS
constexpr int kOffTimers = kMiscBytes + kGuard;
constexpr int kNTimers = (kOffSlots - kOffTimers) / 8;
__device__ unsigned long long g_tc5_timers[kNTimers];
__device__ __forceinline__ unsigned long long* tc5_tacc(const void* sm) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<uintptr_t>(sm) + kOffTimers);
}
#define TC5_T0(v) const long long v = clock64()
#define TC5_ADD(smb, i, t0) atomicAdd(tc5_tacc(smb) + (i), (unsigned long long)(clock64() - (t0)))
#define TC5_CNT(smb, i) atomicAdd(tc5_tacc(smb) + (i), 1ull)
#else
#define TC5_T0(v)
#define TC5_ADD(smb, i, t0)
#define TC5_CNT(smb, i)
#endif

// Bounded wait that, when it gives up first, records where (site id, CTA, tile, parity,
// thread) in the control block's diagnostic words, so that the host can report it.
__device__ __forceinline__ bool waitx(uint64_t* bar, unsigned parity, int site, int tile, Tc5Shared* sh,
                                      const Tc5Args& a) {
#ifdef ENKF_TC5_TIMERS
    TC5_T0(tw);
    const bool okw = mbar_wait(bar, parity, &sh->err, a.ctl, a.timeout_ns);
    if ((threadIdx.x & 31) == 0 && site < 16) TC5_ADD(sh, site, tw);
    if (okw) return true;
#else
    if (mbar_wait(bar, parity, &sh->err, a.ctl, a.timeout_ns)) return true;
#endif
    if (atomicCAS(&a.ctl->pad[0], 0, site) == 0) {
        a.ctl->pad[1] = blockIdx.x;
        a.ctl->pad[2] = tile;
        a.ctl->pad[3] = (int)parity;
        a.ctl->pad[4] = threadIdx.x;
        a.ctl->pad[5] = sh->flag[3];        // sweep and chunk: 1000 k0 + 100 bp + chunk
        for (int w = 0; w < 4; ++w) a.ctl->pad[30 + w] = ((volatile int*)sh->prog)[w];   // warps 0-3
        // raw barrier words (the phase bit is the top bit of the 64-bit state)
        a.ctl->pad[34] = (int)(((volatile uint64_t*)sh->as_full)[0] >> 32);
        a.ctl->pad[35] = (int)(((volatile uint64_t*)sh->as_full)[1] >> 32);
        a.ctl->pad[36] = (int)(((volatile uint64_t*)sh->as_empty)[0] >> 32);
        a.ctl->pad[37] = (int)(((volatile uint64_t*)sh->as_empty)[1] >> 32);
        a.ctl->pad[38] = (int)(((volatile uint64_t*)sh->d2_full)[0] >> 32);
        a.ctl->pad[39] = (int)(((volatile uint64_t*)sh->d2_full)[1] >> 32);
        a.ctl->pad[40] = (int)(*(volatile uint64_t*)bar >> 32);
        a.ctl->pad[41] = (int)(*(volatile uint64_t*)bar);
        check_guards(reinterpret_cast<const unsigned char*>(sh), a.ctl);
    }
    if (site < 16) atomicAdd(&a.ctl->pad[10 + site], 1);
    return false;
}

// One sweep over this CTA's tiles.  Returns false if a wait expired (the CTA must leave).
__device__ bool sweep_tc5(const Tc5Args& a, const CUtensorMap* tmU, const CUtensorMap* tmZ, unsigned char* sm,
                          Tc5Shared* sh, unsigned tbase, const SweepSpec& sp, Counters& cn) {
    const int N = a.nens, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T0 = blockIdx.x * a.tiles_per_blk;
    const int T1 = min(T0 + a.tiles_per_blk, a.ntiles);
    if (T1 <= T0) return true;
    const int ntl = T1 - T0;
    const int nU = N - sp.k1;                    // trailing U columns
    const int ncols = nU + N;                    // trailing columns in all
    const int nchunks_u = (nU + CW - 1) / CW, nchunks = nchunks_u + (N + CW - 1) / CW;
    const bool upd = sp.bp > 0, dots = sp.nb > 0;
    unsigned char* slots = sm + kOffSlots;
    unsigned char* as = sm + kOffAs;
    unsigned char* vp = sm + kOffVp;
    unsigned char* up = sm + kOffUp;
    unsigned char* kp = sm + kOffKp;
    unsigned char* bpc = sm + kOffBp;
    const float* W = reinterpret_cast<const float*>(sm + kOffW);
    const int pv = sp.kv / PB;                   // panel index of V_{P'}
    const int nbn = min(PB, N - sp.k1);          // width of the panel after P (its U_P pieces)

    for (int ch = 0; ch < nchunks; ++ch) {
        const bool zpart = ch >= nchunks_u;
        const int cc0 = zpart ? (ch - nchunks_u) * CW : ch * CW;          // first column in U or Z
        const int ncl = min(CW, (zpart ? N : nU) - cc0);
        const int gidx = zpart ? nU + cc0 : cc0;                         // first trailing column
        const int acol0 = zpart ? cc0 : sp.k1 + cc0;                      // first column in its array
        const CUtensorMap* tm = zpart ? tmZ : tmU;
        const bool mat = sp.mat && ch == 0 && upd;
        const bool writeup = ch == 0 && !zpart && upd && nbn > 0;      // next panel's U_P pieces
        TC5_T0(tk);
        __syncthreads();
        if (tid == 0) sh->flag[3] = 1000 * sp.k0 + 100 * (sp.bp > 0) + 10 * (sp.nb > 0) + ch;
        // ---- K = -W A for this chunk's columns (and beta once per sweep), as BF16 pieces
        if (upd) {
            for (int e = tid; e < CW * 4; e += kThreads) {
                const int c = e >> 2, t8 = e & 3;          // column, 8-wide group of t
                float kv8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) kv8[q] = 0.f;
                if (c < ncl) {
                    const double* acol = a.coefg + gidx + c + sp.aoff;
                    for (int u = 0; u < sp.bp; ++u) {
                        const float au = (float)__ldcg(acol + (int64_t)u * sp.ncols_prev);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int t = t8 * 8 + q;
                            if (t < sp.bp) kv8[q] = fmaf(-W[t * PB + u], au, kv8[q]);
                        }
                    }
                }
                uint4 pc[3];
                pieces8(kv8, pc);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    *reinterpret_cast<uint4*>(kp + q * kPiece + kmaj_off(c, t8, CW * 32)) = pc[q];
            }
            if (mat) {
                // beta[u][m] (u_m = U_P beta_m) as the B operand of MMA3: N = m, K = u
                const float* Bf = reinterpret_cast<const float*>(sm + kOffSlots) + 4 * PB * PB;
                for (int e = tid; e < PB * 4; e += kThreads) {
                    const int m = e >> 2, u8 = e & 3;
                    float bv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int u = u8 * 8 + q;
                        bv[q] = (u < sp.bp && m < sp.bp) ? Bf[u * PB + m] : 0.f;
                    }
                    uint4 pc[3];
                    pieces8(bv, pc);
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        *reinterpret_cast<uint4*>(bpc + q * (PB * PB * 2) + kmaj_off(m, u8, PB * 32)) = pc[q];
                }
            }
        }
        fence_async_smem();
        __syncthreads();
#ifdef ENKF_TC5_TIMERS
        if (tid == 0) TC5_ADD(sm, kTmK, tk), TC5_CNT(sm, kTmChunks);
#endif
        TC5_T0(te);
        bool ok = true;
        if (warp < NEPI) {
            // ---------------- epilogue warp (q, h): rows 32 q .. 32 q + 31 of every tile, columns
            // 32 NSW h .. of the chunk (slots s = NSW h ..), dots and final columns t = HT h .. HT h + HT - 1
            const int q = warp & 3, h = warp >> 2;
            constexpr int HT = PB / NH;
            static_assert(HT == 8 || HT == 16, "TMEM loads of the dots and final columns");
            float acc2[HT];
#pragma unroll
            for (int t = 0; t < HT; ++t) acc2[t] = 0.f;
            const unsigned lanes = tbase + ((unsigned)(q * 32) << 16);
            unsigned char* myslots = slots + q * NS * kSlotBytes;
            const int s0 = NSW * h, s1 = NSW * h + NSW;
            // prefetch the first tile's blocks
            if (lane == 0)
                for (int s = s0; s < s1; ++s) {
                    mbar_expect_tx(&sh->slot_full[q * NS + s], kSlotBytes);
                    tma_load_2d(myslots + s * kSlotBytes, tm, T0 * TR + q * 32, acol0 + s * SWC,
                                &sh->slot_full[q * NS + s]);
                }
            Counters c = cn;
            auto fold_d2 = [&](unsigned g2) -> bool {
                if (!waitx(&sh->d2_full[g2 & 1], (g2 >> 1) & 1, 2, (int)g2, sh, a)) return false;
                fence_after();
                // the three blocks (products with V's pieces 0, 1, 2), added smallest first
                unsigned v0[HT], v1[HT], v2[HT];
                const unsigned d2a = lanes + kD2 + (g2 & 1) * kD2W + h * HT;
                if constexpr (HT == 8) {
                    tmem_ld8(d2a, v0);
                    tmem_ld8(d2a + PB, v1);
                    tmem_ld8(d2a + 2 * PB, v2);
                    tmem_wait_ld8(v0);
                    tmem_wait_ld8(v1);
                    tmem_wait_ld8(v2);
                } else {
                    tmem_ld16(d2a, v0);
                    tmem_ld16(d2a + PB, v1);
                    tmem_ld16(d2a + 2 * PB, v2);
                    tmem_wait_ld(v0);
                    reg_fence16(v1);
                    reg_fence16(v2);
                }
#pragma unroll
                for (int t = 0; t < HT; ++t)
                    acc2[t] += (__uint_as_float(v2[t]) + __uint_as_float(v1[t])) + __uint_as_float(v0[t]);
                fence_before();
                mbar_arrive(&sh->d2_empty[g2 & 1]);
                return true;
            };
            for (int it = 0; ok && it < ntl; ++it) {
                const int T = T0 + it;
                const int64_t row = (int64_t)T * TR + q * 32 + lane;
                const unsigned sig = 4u * c.g2 + (unsigned)q;          // this warp's MMA2 slice
                unsigned char* asb = as + (sig % kNAs) * kOp3;
                if (lane == 0) ((volatile int*)sh->prog)[warp] = 16 * (int)c.gt + 1;
                if (upd && !waitx(&sh->d1_full[c.g1 & 1], (c.g1 >> 1) & 1, 3, it, sh, a)) {
                    ok = false;
                    break;
                }
                fence_after();
                // (1) X_new = X + D1 for both slots: written back to the slot (for the transposed
                // reads below) and stored; the next panel's U_P pieces from chunk 0
                TC5_T0(tx);
                static_assert(NSW == 2, "the X update below loads two slots' D1 columns at once");
                for (int s = s0; s < s1; ++s)
                    if (!waitx(&sh->slot_full[q * NS + s], c.gt & 1, 4, it, sh, a)) {
                        ok = false;
                        break;
                    }
                if (!ok) break;
                unsigned dv0[16], dv1[16], dv2[16], dv3[16];
                if (upd) {
                    // every D1 column of this warp's slots in one round trip
                    const unsigned d1a = lanes + kD1 + (c.g1 & 1) * CW + s0 * SWC;
                    tmem_ld16(d1a, dv0);
                    tmem_ld16(d1a + 16, dv1);
                    tmem_ld16(d1a + SWC, dv2);
                    tmem_ld16(d1a + SWC + 16, dv3);
                    tmem_wait_ld(dv0);
                    reg_fence16(dv1);
                    reg_fence16(dv2);
                    reg_fence16(dv3);
                }
                if (upd) {
                    unsigned char* sl0 = myslots + s0 * kSlotBytes;
                    unsigned char* sl1 = sl0 + kSlotBytes;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float* p0 = slot_at(sl0, j, lane);
                        float* p1 = slot_at(sl0, 16 + j, lane);
                        float* p2 = slot_at(sl1, j, lane);
                        float* p3 = slot_at(sl1, 16 + j, lane);
                        *p0 = *p0 + __uint_as_float(dv0[j]);
                        *p1 = *p1 + __uint_as_float(dv1[j]);
                        *p2 = *p2 + __uint_as_float(dv2[j]);
                        *p3 = *p3 + __uint_as_float(dv3[j]);
                    }
                    // X_new to global memory from the slots by TMA (rows past nobs and columns past
                    // N lie outside the tensor and are not written)
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        for (int s = s0; s < s1; ++s)
                            tma_store_2d(tm, T * TR + q * 32, acol0 + s * SWC, myslots + s * kSlotBytes);
                        bulk_commit();
                    }
                    if (writeup && s0 == 0) {
                        // pieces of the next panel's U_P (trailing columns 0 .. nbn-1) for this row,
                        // read back from slot 0 (this lane's own row)
                        unsigned char* ub = tile_piece(a.upc, (int64_t)(sp.up_par ^ 1) * a.ntiles + T);
                        const int m = q * 32 + lane;
#pragma unroll
                        for (int t8 = 0; t8 < 4; ++t8) {
                            float v8[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                v8[e] = (t8 * 8 + e < nbn && row < a.nobs) ? *slot_at(sl0, t8 * 8 + e, lane) : 0.f;
                            uint4 pc[3];
                            pieces8(v8, pc);
#pragma unroll
                            for (int pq = 0; pq < 3; ++pq)
                                *reinterpret_cast<uint4*>(ub + pq * kPiece + kmaj_off(m, t8, TR * 32)) = pc[pq];
                        }
                    }
                }
                if (!ok) break;
#ifdef ENKF_TC5_TIMERS
                if (tid == 0) TC5_ADD(sm, kTmXup, tx);
#endif
                if (upd) {
                    // D1 has been read: MMA1 of tile it + 2 may overwrite it
                    fence_before();
                    mbar_arrive(&sh->d1_empty[c.g1 & 1]);
                }
                // (2) slice sig goes to buffer sig % 3, free once MMA2 has read slice sig - 3 (row
                // quarter q + 1 of the previous tile, or quarter 0 of this one for q = 3), whose
                // commit arrives on this warp's as_empty.  MMA2 takes the slices in order, so that
                // completion cannot be overtaken by the next one before this warp has waited for it.
                if (dots && sig >= kNAs) {
                    const unsigned k = q == NQ - 1 ? c.g2 : c.g2 - 1;
                    if (!waitx(&sh->as_empty[q], k & 1, 12, it, sh, a)) {
                        ok = false;
                        break;
                    }
                }
                // (3) the slots' 32 columns x this quarter's 32 rows -> pieces of MMA2's A operand
                // (M = chunk column, K = row): lane = column, four 8-row groups; then the slot
                // takes the next tile's block
                TC5_T0(tcv);
                if (dots) __syncwarp();       // the other lanes' rows of the slots are written
                for (int s = s0; s < s1; ++s) {
                    unsigned char* slot = myslots + s * kSlotBytes;
                    if (dots) {
                        const int cm = s * SWC + lane;
#pragma unroll
                        for (int g4 = 0; g4 < 4; ++g4) {
                            const float4 lo4 = *reinterpret_cast<const float4*>(slot + lane * 128 +
                                                                                (((2 * g4) ^ (lane & 7)) << 4));
                            const float4 hi4 = *reinterpret_cast<const float4*>(slot + lane * 128 +
                                                                                (((2 * g4 + 1) ^ (lane & 7)) << 4));
                            float v8[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
                            if (row - lane + g4 * 8 >= a.nobs) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v8[e] = 0.f;
                            }
                            uint4 pc[3];
                            pieces8(v8, pc);
#pragma unroll
                            for (int pq = 0; pq < 3; ++pq)
                                *reinterpret_cast<uint4*>(asb + pq * kPiece + kmaj_off(cm, g4, CW * 32)) = pc[pq];
                        }
                    }
                }
                // the pieces are read by MMA2 and the slots rewritten by TMA (async proxy)
                fence_async_smem();
                __syncwarp();
                if (lane == 0 && it + 1 < ntl) {
                    if (upd) bulk_wait_read0();       // the slots' stores have read them
                    for (int s = s0; s < s1; ++s) {
                        mbar_expect_tx(&sh->slot_full[q * NS + s], kSlotBytes);
                        tma_load_2d(myslots + s * kSlotBytes, tm, (T + 1) * TR + q * 32, acol0 + s * SWC,
                                    &sh->slot_full[q * NS + s]);
                    }
                }
                if (dots) mbar_arrive(&sh->as_full[q]);
#ifdef ENKF_TC5_TIMERS
                if (tid == 0) TC5_ADD(sm, kTmConv, tcv);
#endif
                TC5_T0(tmt);
                if (lane == 0) ((volatile int*)sh->prog)[warp] = 16 * (int)c.gt + 2;
                if (mat) {
                    // the panel's final columns u_{k0+m} = U_P beta_m for these rows
                    if (!waitx(&sh->d3_full, c.g3 & 1, 5, it, sh, a)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    unsigned u0[HT];
                    if constexpr (HT == 8) {
                        tmem_ld8(lanes + kD3 + h * HT, u0);
                        tmem_wait_ld8(u0);
                    } else {
                        tmem_ld16(lanes + kD3 + h * HT, u0);
                        tmem_wait_ld(u0);
                    }
                    if (row < a.nobs) {
#pragma unroll
                        for (int m = 0; m < HT; ++m)
                            if (h * HT + m < sp.bp)
                                a.U[(int64_t)(sp.k0 + h * HT + m) * a.ldu + row] = __uint_as_float(u0[m]);
                    }
                    if (a.ufc) {
                        // their pieces in MMA1's A order, for the correction sweep
                        unsigned char* fb = tile_piece(a.ufc, (int64_t)(sp.k0 / PB) * a.ntiles + T);
#pragma unroll
                        for (int g = 0; g < HT / 8; ++g) {
                            float v8[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int m = h * HT + g * 8 + e;
                                v8[e] = (m < sp.bp && row < a.nobs) ? __uint_as_float(u0[g * 8 + e]) : 0.f;
                            }
                            uint4 pc[3];
                            pieces8(v8, pc);
#pragma unroll
                            for (int pq = 0; pq < 3; ++pq)
                                *reinterpret_cast<uint4*>(fb + pq * kPiece +
                                                          kmaj_off(q * 32 + lane, (HT / 8) * h + g, TR * 32)) = pc[pq];
                        }
                    }
                    fence_before();
                    mbar_arrive(&sh->d3_empty);
                }
#ifdef ENKF_TC5_TIMERS
                if (tid == 0) TC5_ADD(sm, kTmMat, tmt);
#endif
                TC5_T0(tfd);
                if (lane == 0) ((volatile int*)sh->prog)[warp] = 16 * (int)c.gt + 3;
                if (dots && it > 0 && !fold_d2(c.g2 - 1)) {
                    ok = false;
                    break;
                }
#ifdef ENKF_TC5_TIMERS
                if (tid == 0) TC5_ADD(sm, kTmFold, tfd);
#endif
                c.gt++;
                if (upd) c.g1++;
                if (dots) c.g2++;
                if (mat) c.g3++;
            }
            if (lane == 0) ((volatile int*)sh->prog)[warp] = 16 * (int)c.gt + 4;
            if (ok && dots && !fold_d2(c.g2 - 1)) ok = false;
            if (lane == 0) ((volatile int*)sh->prog)[warp] = 16 * (int)c.gt + 5;
            if (ok && dots) {
                // this CTA's partial dots of the chunk's columns: part[t * ncols + column]
                const int cm = q * 32 + lane;
                if (cm < ncl) {
#pragma unroll
                    for (int t = 0; t < HT; ++t)
                        if (h * HT + t < sp.nb)
                            __stcg(&a.part[(int64_t)blockIdx.x * a.part_stride + (int64_t)(h * HT + t) * ncols + gidx +
                                           cm],
                                   (double)acc2[t]);
                }
            }
            // this chunk's X stores complete (their writes are read by TMA in later sweeps)
            if (lane == 0 && upd) bulk_wait0();
            if (!ok && lane == 0) {
                // copies still in flight land before the CTA may leave
                for (int s = s0; s < s1; ++s) mbar_drain(&sh->slot_full[q * NS + s], c.gt & 1, a.timeout_ns);
            }
        } else if (warp == kMmaWarp) {
            // ---------------- MMA1 and MMA3, one thread.  Step i: MMA1 of tile i (once its U_P pieces
            // have landed and the epilogue has released the D1 buffer of tile i - 2), then MMA3 of tile
            // i; U_P(i + 1) is loaded once those have read the (single) buffer, which is more than a
            // tile before MMA1(i + 1) can start (the epilogue still holds D1 of tile i - 1).
            if (lane == 0 && upd) {
                TC5_T0(tm);
                Counters c = cn;
                const unsigned id1 = instr_desc(TR, CW), id3 = instr_desc(TR, PB);
                const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
                auto load_up = [&](int tile) {
                    mbar_expect_tx(&sh->up_full[0], kOp3);
                    bulk_load(up, tile_piece(sp.upb, T0 + tile), kOp3, &sh->up_full[0]);
                };
                load_up(0);
                for (int it = 0; ok && it < ntl; ++it) {
                    if (!waitx(&sh->up_full[0], c.g1 & 1, 6, it, sh, a) ||
                        (c.g1 >= 2 && !waitx(&sh->d1_empty[c.g1 & 1], ((c.g1 >> 1) - 1) & 1, 13, it, sh, a))) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const unsigned d1 = tbase + kD1 + (c.g1 & 1) * CW;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                        for (int q = 0; q < 6; ++q)
                            mma_bf16(d1, smem_desc(up + pa[q] * kPiece + ks * (TR * 32)),
                                     smem_desc(kp + pb[q] * kPiece + ks * (CW * 32)), id1, (ks | q) != 0);
                    mma_commit(&sh->d1_full[c.g1 & 1]);
                    if (mat) {
                        // D3 is free once the epilogue has written tile i - 1's final columns
                        if (c.g3 >= 1 && !waitx(&sh->d3_empty, (c.g3 - 1) & 1, 7, it, sh, a)) {
                            ok = false;
                            break;
                        }
                        fence_after();
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                            for (int q = 0; q < 6; ++q)
                                mma_bf16(tbase + kD3, smem_desc(up + pa[q] * kPiece + ks * (TR * 32)),
                                         smem_desc(bpc + pb[q] * (PB * PB * 2) + ks * (PB * 32)), id3,
                                         (ks | q) != 0);
                        mma_commit(&sh->d3_full);
                    }
                    mma_commit(&sh->up_empty[0]);
                    // U_P(it + 1) once MMA1 and MMA3 of tile it have read the buffer (every tile's
                    // release is waited for, so the parity waits stay in step)
                    if (!waitx(&sh->up_empty[0], c.g1 & 1, 8, it, sh, a)) {
                        ok = false;
                        break;
                    }
                    if (it + 1 < ntl) load_up(it + 1);
                    c.g1++;
                    if (mat) c.g3++;
                }
                // the commit arrives once every MMA issued above has completed
                mma_commit(&sh->drained_a);
                mbar_drain(&sh->drained_a, sh->flag[0] & 1, a.timeout_ns);
                sh->flag[0]++;
                TC5_ADD(sm, kTmMma, tm);
            }
            __syncwarp();
        } else {
            // ---------------- MMA2, one thread (warp kAllocWarp): the dots of tile i as soon as the
            // epilogue has filled its four A slices; the V pieces are single-buffered (V(i + 1) is
            // loaded once MMA2(i) has read V(i), a tile before MMA2(i + 1) needs it).
            if (lane == 0 && dots) {
                Counters c = cn;
                // piece i of the A slice against V's pieces 0 .. 2 - i side by side (N = 32 (3 - i)):
                // block j of D2 collects the products with V's piece j
                const unsigned id2[3] = {instr_desc(TR, 3 * PB), instr_desc(TR, 2 * PB), instr_desc(TR, PB)};
                auto load_vp = [&](int tile) {
                    mbar_expect_tx(&sh->vp_full, kOp3);
                    bulk_load(vp, tile_piece(a.vpc, (int64_t)pv * a.ntiles + T0 + tile), kOp3, &sh->vp_full);
                };
                load_vp(0);
                for (int jt = 0; ok && jt < ntl; ++jt) {
                    const unsigned b = c.g2 & 1;
                    if (!waitx(&sh->vp_full, c.g2 & 1, 9, jt, sh, a) ||
                        (c.g2 >= 2 && !waitx(&sh->d2_empty[b], ((c.g2 >> 1) - 1) & 1, 14, jt, sh, a))) {
                        ok = false;
                        break;
                    }
                    const unsigned d2 = tbase + kD2 + b * kD2W;
                    for (int q = 0; q < NQ; ++q) {
                        const unsigned sig = 4u * c.g2 + (unsigned)q;
                        if (!waitx(&sh->as_full[q], c.g2 & 1, 10, jt, sh, a)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const unsigned char* asb = as + (sig % kNAs) * kOp3;
                        const unsigned char* vb = vp + q * (3 * PB * 32 * 2);
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                            for (int i = 0; i < 3; ++i)
                                mma_bf16(d2, smem_desc(asb + i * kPiece + ks * (CW * 32)),
                                         smem_desc(vb + ks * (3 * PB * 32)), id2[i], (q | ks | i) != 0);
                        mma_commit(&sh->as_empty[(q + kNAs) % NQ]);   // the next user of this buffer
                    }
                    if (!ok) break;
                    mma_commit(&sh->d2_full[b]);
                    mma_commit(&sh->vp_empty);
                    // V(jt + 1) once MMA2(jt) has read the buffer (every tile's release is waited for,
                    // the last one after the loop)
                    if (!waitx(&sh->vp_empty, c.g2 & 1, 11, jt, sh, a)) {
                        ok = false;
                        break;
                    }
                    if (jt + 1 < ntl) load_vp(jt + 1);
                    c.g2++;
                }
                mma_commit(&sh->drained_b);
                mbar_drain(&sh->drained_b, sh->flag[1] & 1, a.timeout_ns);
                sh->flag[1]++;
            }
            __syncwarp();
        }
#ifdef ENKF_TC5_TIMERS
        if (tid == 0) TC5_ADD(sm, kTmEpi, te);
#endif
        TC5_T0(tn);
        // the generic-proxy stores of this chunk (X, the next U_P pieces, the final panel
        // columns) are read by TMA and bulk copies (async proxy) in later sweeps
        asm volatile("fence.proxy.async;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) check_guards(sm, a.ctl);
#ifdef ENKF_TC5_TIMERS
        if (tid == 0) TC5_ADD(sm, kTmEnd, tn);
#endif
        if (sh->err) return false;
        // every role advanced the counters by the same tiles
        cn.gt += ntl;
        if (upd) cn.g1 += ntl;
        if (dots) cn.g2 += ntl;
        if (mat) cn.g3 += ntl;
    }
    return true;
}

// Fixed-order cross-CTA sum of the partial dots (nvals entries) into coefg: every CTA
// owns a slice of the entries, one warp per entry; lane l sums CTAs l, l + 32, ... in
// order, then a fixed butterfly.
__device__ bool reduce_tc5(const Tc5Args& a, Tc5Shared* sh, int nvals, unsigned& epoch) {
    const unsigned nblk = gridDim.x;
    TC5_T0(tr);
    if (!grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, &sh->flag[2])) return false;
    const int per = (nvals + (int)nblk - 1) / (int)nblk;
    const int e0 = blockIdx.x * per, e1 = min(e0 + per, nvals);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = e0 + warp; e < e1; e += kThreads / 32) {
        double v = 0.0;
        for (int b = lane; b < (int)nblk; b += 32) v += __ldcg(&a.part[(int64_t)b * a.part_stride + e]);
        v = warp_sum(v);
        if (lane == 0) __stcg(&a.coefg[e], v);
    }
    const bool okb = grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, &sh->flag[2]);
#ifdef ENKF_TC5_TIMERS
    if (threadIdx.x == 0) TC5_ADD(sh, kTmRed, tr);
#endif
    return okb;
}

// W_fin = diag(1/gamma) (I + L)^-1 of a factored panel, by one warp (lane l forms column l by
// forward substitution, (I + L) t = e_l): with h_m = u_m / gamma_m the final columns, the
// panel's b levels applied to any x are x <- x - U_fin W_fin (V_P^T x).
__device__ void store_wfin(const FactorView& fv, int bp, float* out) {
    const int l = threadIdx.x & 31;
    float t[PB];
#pragma unroll
    for (int m = 0; m < PB; ++m) {
        float v = (m == l) ? 1.f : 0.f;
        if (m > l && m < bp) {
#pragma unroll
            for (int j = 0; j < m; ++j)
                if (j >= l) v = fmaf(-fv.Lt[j * PB + m], t[j], v);
        }
        t[m] = (l < bp && m < bp) ? v : 0.f;
    }
#pragma unroll
    for (int m = 0; m < PB; ++m)
        out[m * PB + l] = (m < bp) ? t[m] * (float)(1.0 / fv.gam[m]) : 0.f;
}

__global__ void __launch_bounds__(kThreads, 1) ism_panel_tc05_kernel(const __grid_constant__ CUtensorMap tmU,
                                                                     const __grid_constant__ CUtensorMap tmZ,
                                                                     Tc5Args a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    Tc5Shared* sh = reinterpret_cast<Tc5Shared*>(sm + kOffMisc);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int q = 0; q < NQ * NS; ++q) mbar_init(&sh->slot_full[q], 1);
        mbar_init(&sh->vp_full, 1);
        mbar_init(&sh->vp_empty, 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init(&sh->up_full[q], 1), mbar_init(&sh->up_empty[q], 1);
            mbar_init(&sh->d1_full[q], 1), mbar_init(&sh->d1_empty[q], NEPI * 32);
            mbar_init(&sh->d2_full[q], 1), mbar_init(&sh->d2_empty[q], NEPI * 32);
        }
        for (int q = 0; q < NQ; ++q) mbar_init(&sh->as_full[q], NH * 32), mbar_init(&sh->as_empty[q], 1);
        mbar_init(&sh->d3_full, 1);
        mbar_init(&sh->d3_empty, NEPI * 32);
        mbar_init(&sh->drained_a, 1);
        mbar_init(&sh->drained_b, 1);
        sh->err = 0;
        for (int q = 0; q < 4; ++q) sh->flag[q] = 0;
        mbar_init_fence();
    }
#ifdef ENKF_TC5_TIMERS
    TC5_T0(tall);
    for (int i = tid; i < kNTimers; i += kThreads) tc5_tacc(sm)[i] = 0ull;
#endif
    for (int g = 0; g < kNGuard; ++g)
        for (int i = tid; i < kGuard / 4; i += kThreads) reinterpret_cast<unsigned*>(sm + guard_off(g))[i] = kGuardWord;
    if (warp == kAllocWarp) tmem_alloc(&sh->taddr, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tbase = sh->taddr;

    FactorView fv;
    fv.Gh = reinterpret_cast<float*>(sm + kOffSlots);
    fv.Gl = fv.Gh + PB * PB;
    fv.Bt = fv.Gh + 2 * PB * PB;
    fv.Lt = fv.Gh + 3 * PB * PB;
    fv.Bf = fv.Gh + 4 * PB * PB;
    fv.cb = fv.Gh + 5 * PB * PB;
    fv.W = reinterpret_cast<float*>(sm + kOffW);
    fv.gam = sh->gam;

    const int N = a.nens, b = PB;
    Counters cn = {0u, 0u, 0u, 0u};
    unsigned epoch = 0;
    // ---- the dots of panel 0: in the solve with every column of U^(0) = R^-1 V and Z^(0) =
    // R^-1 D (Step 1, eq. SM-step-1, was applied by the pass before this launch); in the
    // correction sweep with the columns of Z only (already scaled by R^-1)
    const int kz = a.refine ? N : 0;                 // first trailing U column of the first sweep
    int nb = b < N ? b : N;
    SweepSpec sp = {0, 0, kz, 0, nb, 0, 0, 0, 0, nullptr};
    bool ok = sweep_tc5(a, &tmU, &tmZ, sm, sh, tbase, sp, cn) && reduce_tc5(a, sh, nb * ((N - kz) + N), epoch);
    for (int k0 = 0; ok && k0 < N; k0 += b) {
        const int bp = (N - k0) < b ? (N - k0) : b;
        const int k1 = k0 + bp;
        const int pidx = k0 / b;
        TC5_T0(tf);
        if (a.refine) {
            // the panel's stored factor: K = -diag(1/gamma) (I + L)^-1 A applied to the final columns
            for (int e = tid; e < PB * PB; e += kThreads) fv.W[e] = __ldcg(&a.wfin[(int64_t)pidx * PB * PB + e]);
            if (a.C) {
                // the per-level coefficients c = (I + L)^-1 a of the corrected columns (one warp per
                // column, CTAs round-robin), so that V^T of the result follows from the identity
                // V^T x = (I - triu(Q,1)) diag(1/gamma) C without another pass over the rows
                __syncthreads();
                const int lane = tid & 31;
                for (int i = blockIdx.x * (kThreads / 32) + warp; i < N; i += gridDim.x * (kThreads / 32))
                    if (lane < bp) {
                        double v = 0.0;
                        for (int u = 0; u < bp; ++u)
                            v = fma((double)fv.W[lane * PB + u], __ldcg(&a.coefg[(int64_t)u * N + i]), v);
                        a.C[(int64_t)(k0 + lane) * N + i] = v * __ldcg(&a.gamma[k0 + lane]);
                    }
            }
            nb = (N - k1) < b ? (N - k1) : b;
            SweepSpec s2 = {k0, bp, N, k1, nb, 0, N, 0, 0, tile_piece(a.ufc, (int64_t)pidx * a.ntiles)};
            ok = sweep_tc5(a, &tmU, &tmZ, sm, sh, tbase, s2, cn);
            if (ok && nb > 0) ok = reduce_tc5(a, sh, nb * N, epoch);
            if (nb == 0) break;
            continue;
        }
        const int ncols_prev = (N - k0) + N;
        // factor of the panel (every CTA): the FP64 Gram split into float hi + lo
        for (int e = tid; e < PB * PB; e += kThreads) {
            const int t = e / PB, u = e % PB;
            const double g = (t < bp && u < bp) ? __ldcg(&a.coefg[t * ncols_prev + u]) : 0.0;
            const float h = (float)g;
            fv.Gh[e] = h;
            fv.Gl[e] = (float)(g - (double)h);
        }
        __syncthreads();
        if (warp == 0) factor_warp(fv, bp);
        __syncthreads();
        if (blockIdx.x == 0 && tid < bp) {
            const double g = fv.gam[tid];
            a.gamma[k0 + tid] = g;
            if (a.check && (!(g >= 1.0 - 64.0 * 1.1920928955078125e-07 * (1.0 + fabs(g - 1.0))) || !isfinite(g))) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = k0 + tid + 1;
            }
        }
        // per-level Z coefficients c = (I + L)^{-1} a of z_i (one warp per column, CTAs
        // round-robin over the columns): lane m holds a_m, level l broadcasts c_l
        for (int i = blockIdx.x * (kThreads / 32) + warp; i < N; i += gridDim.x * (kThreads / 32)) {
            const int lane = tid & 31;
            const int ai = (N - k0) + i;
            float v = lane < bp ? (float)__ldcg(&a.coefg[lane * ncols_prev + ai]) : 0.f;
            for (int l = 0; l < bp; ++l) {
                const float cl = __shfl_sync(0xffffffffu, v, l);
                if (lane > l) v = fmaf(-fv.Lt[l * PB + lane], cl, v);
            }
            if (lane < bp) a.C[(int64_t)(k0 + lane) * N + i] = (double)v;
        }
        // the stored factor for a correction sweep (the factor view is read before the sweep's
        // second CTA barrier, after which the X slots it aliases are refilled)
        if (a.wfin && blockIdx.x == 0 && warp == 0) store_wfin(fv, bp, a.wfin + (int64_t)pidx * PB * PB);
#ifdef ENKF_TC5_TIMERS
        if (tid == 0) TC5_ADD(sm, kTmFac, tf);
#endif
        nb = (N - k1) < b ? (N - k1) : b;
        const int par = pidx & 1;
        SweepSpec s2 = {k0, bp, k1, k1, nb, bp, ncols_prev, 1, par, tile_piece(a.upc, (int64_t)par * a.ntiles)};
        ok = sweep_tc5(a, &tmU, &tmZ, sm, sh, tbase, s2, cn);
        if (ok && nb > 0) ok = reduce_tc5(a, sh, nb * ((N - k1) + N), epoch);
        if (nb == 0) break;
    }
    fence_before();
    __syncthreads();
#ifdef ENKF_TC5_TIMERS
    if (tid == 0) TC5_ADD(sm, kTmAll, tall);
    __syncthreads();
    for (int i = tid; i < kNTimers; i += kThreads) atomicAdd(&g_tc5_timers[i], tc5_tacc(sm)[i]);
#endif
    if (warp == kAllocWarp) {
        fence_after();
        tmem_dealloc(tbase, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Step 1 (eq. SM-step-1) for the tensor-core panel path: U = R^-1 V and Z = R^-1 D (one
// reciprocal per row), the BF16 pieces of V for every panel in the B-operand order of
// MMA2 ([panel][tile][piece][slice][k-step][t / 8][k-group][t % 8][8 rows]) and the pieces
// of panel 0's U_P in the A-operand order of MMA1 ([tile][piece][k-step][row / 8]
// [k-group][row % 8][8 t]).  Rows past nobs are zero in the pieces.
// ---------------------------------------------------------------------------
struct Step1Args {
    int64_t nobs;
    int32_t nens, ntiles;
    const float* r;
    const float* V;
    int64_t ldv;
    const float* D;
    int64_t ldd;
    float* U;
    int64_t ldu;
    float* Z;
    int64_t ldz;
    unsigned char* vpc;
    unsigned char* upc;
    Control* ctl;
    int32_t check;
};

__global__ void __launch_bounds__(256) tc5_step1_kernel(Step1Args a) {
    const int N = a.nens;
    const int npan = (N + PB - 1) / PB;
    const int64_t T = blockIdx.x;                        // one 128-row tile per CTA
    const int tid = threadIdx.x;
    const int rg = tid & 15, cl = tid >> 4;              // 8-row group, column lane (16 per pass)
    const int64_t row0 = T * TR + rg * 8;
    // 1 / r of this thread's 8 rows (rows past nobs: 0, so that every product below is 0)
    float rinv[8];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t row = row0 + j;
        rinv[j] = 0.f;
        if (row < a.nobs) {
            const float rj = a.r[row];
            if (!(rj > 0.f && isfinite(rj))) bad = true;
            rinv[j] = 1.0f / rj;
        }
    }
    const bool full = row0 + 8 <= a.nobs;
    // V columns: U = V / r, the V pieces of every panel; D columns: Z = D / r
    for (int c = cl; c < npan * PB + N; c += 16) {
        const bool isv = c < npan * PB;
        const int col = isv ? c : c - npan * PB;
        float x8[8];
        const float* src = isv ? a.V + (int64_t)col * a.ldv : a.D + (int64_t)col * a.ldd;
        const bool have = col < N;
        const bool vec = have && full && (((uintptr_t)(src + row0)) & 15) == 0;
        if (vec) {
            const float4 p0 = *reinterpret_cast<const float4*>(src + row0);
            const float4 p1 = *reinterpret_cast<const float4*>(src + row0 + 4);
            x8[0] = p0.x, x8[1] = p0.y, x8[2] = p0.z, x8[3] = p0.w, x8[4] = p1.x, x8[5] = p1.y, x8[6] = p1.z,
            x8[7] = p1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) x8[j] = (have && row0 + j < a.nobs) ? src[row0 + j] : 0.f;
        }
        float s8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!isfinite(x8[j])) bad = true;
            s8[j] = x8[j] * rinv[j];
        }
        if (have) {
            float* dst = isv ? a.U + (int64_t)col * a.ldu : a.Z + (int64_t)col * a.ldz;
            if (full && (((uintptr_t)(dst + row0)) & 15) == 0) {
                *reinterpret_cast<float4*>(dst + row0) = make_float4(s8[0], s8[1], s8[2], s8[3]);
                *reinterpret_cast<float4*>(dst + row0 + 4) = make_float4(s8[4], s8[5], s8[6], s8[7]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (row0 + j < a.nobs) dst[row0 + j] = s8[j];
            }
        }
        if (isv) {
            const int pv = col / PB, t = col % PB;
            unsigned char* dstp = a.vpc + ((int64_t)pv * a.ntiles + T) * (int64_t)kOp3 + (rg >> 2) * (3 * PB * 32 * 2) +
                                  ((rg & 3) >> 1) * (3 * PB * 32) + (t >> 3) * 256 + (rg & 1) * 128 + (t & 7) * 16;
            uint4 pc[3];
            pieces8(x8, pc);
#pragma unroll
            for (int pq = 0; pq < 3; ++pq) *reinterpret_cast<uint4*>(dstp + pq * (PB * 32)) = pc[pq];
        }
    }
    // panel 0's U_P pieces: thread (row m, 8-wide group t8), U = V / r of the first 32 columns
    for (int e = tid; e < TR * 4; e += 256) {
        const int t8 = e & 3, m = e >> 2;
        const int64_t row = T * TR + m;
        float v8[8];
        const float ri = row < a.nobs ? 1.0f / a.r[row] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int t = t8 * 8 + j;
            v8[j] = (row < a.nobs && t < N) ? a.V[(int64_t)t * a.ldv + row] * ri : 0.f;
        }
        uint4 pc[3];
        pieces8(v8, pc);
        unsigned char* dst = a.upc + T * (int64_t)kOp3 + kmaj_off(m, t8, TR * 32);
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) *reinterpret_cast<uint4*>(dst + pq * kPiece) = pc[pq];
    }
    if (a.check && bad) {
        set_status(a.ctl, kErrNumeric);
        a.ctl->fail_level = 0;
    }
}

}  // namespace

size_t tc5_vpc_bytes(int64_t nobs, int32_t nens) {
    const int64_t ntiles = (nobs + TR - 1) / TR;
    return (size_t)((nens + PB - 1) / PB) * (size_t)ntiles * kOp3;
}
size_t tc5_upc_bytes(int64_t nobs) { return 2 * (size_t)((nobs + TR - 1) / TR) * kOp3; }
int tc5_panel_b() { return PB; }

cudaError_t tc5_plan(int64_t nobs, int32_t nens, Tc5Launch* L) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(ism_panel_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)) !=
        cudaSuccess)
        return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ism_panel_tc05_kernel, kThreads, kSmem)) !=
        cudaSuccess)
        return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t ntiles = (nobs + TR - 1) / TR;
    int64_t grid = nsm < ntiles ? nsm : ntiles;
    const int64_t tpb = (ntiles + grid - 1) / grid;
    grid = (ntiles + tpb - 1) / tpb;
    L->grid = (int)grid;
    L->ntiles = (int)ntiles;
    L->tiles_per_blk = (int)tpb;
    L->smem = kSmem;
    L->part_stride = (int64_t)PB * 2 * nens;
    return cudaSuccess;
}

// Step 1 and the tensor-core panel solve.  cudaErrorNotSupported when U or Z is not
// TMA-aligned (16-byte base, stride a multiple of 4 floats): the caller then takes the
// mma.sync panel kernel.  ufc and wfin (both or neither): keep the final columns' pieces
// and the per-panel factors for tc5_correct.  ev0 / ev1 (optional): recorded around the
// panel kernel alone (phase timing).
cudaError_t tc5_solve(const Tc5Launch& L, const PanelArgs& p, void* vpc, void* upc, void* ufc, float* wfin,
                      cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    CUtensorMap tmU, tmZ;
    memset(&tmU, 0, sizeof(tmU));
    memset(&tmZ, 0, sizeof(tmZ));
    if (!encode_f32_2d(&tmU, static_cast<const float*>(p.U), p.nobs, p.nens, p.ldu, 32, SWC, true) ||
        !encode_f32_2d(&tmZ, static_cast<const float*>(p.Z), p.nobs, p.nens, p.ldz, 32, SWC, true))
        return cudaErrorNotSupported;
    Step1Args s1;
    s1.nobs = p.nobs;
    s1.nens = p.nens;
    s1.ntiles = L.ntiles;
    s1.r = static_cast<const float*>(p.r);
    s1.V = static_cast<const float*>(p.V);
    s1.ldv = p.ldv;
    s1.D = static_cast<const float*>(p.D);
    s1.ldd = p.ldd;
    s1.U = static_cast<float*>(p.U);
    s1.ldu = p.ldu;
    s1.Z = static_cast<float*>(p.Z);
    s1.ldz = p.ldz;
    s1.vpc = static_cast<unsigned char*>(vpc);
    s1.upc = static_cast<unsigned char*>(upc);
    s1.ctl = p.ctl;
    s1.check = p.check;
    tc5_step1_kernel<<<L.ntiles, 256, 0, s>>>(s1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Tc5Args a;
    a.nobs = p.nobs;
    a.nens = p.nens;
    a.ntiles = L.ntiles;
    a.tiles_per_blk = L.tiles_per_blk;
    a.r = static_cast<const float*>(p.r);
    a.U = static_cast<float*>(p.U);
    a.ldu = p.ldu;
    a.Z = static_cast<float*>(p.Z);
    a.ldz = p.ldz;
    a.vpc = static_cast<const unsigned char*>(vpc);
    a.upc = static_cast<unsigned char*>(upc);
    a.part = p.part;
    a.part_stride = L.part_stride;
    a.coefg = p.coefg;
    a.C = p.C;
    a.gamma = p.gamma;
    a.ctl = p.ctl;
    a.check = p.check;
    a.timeout_ns = p.timeout_ns;
    a.ufc = static_cast<unsigned char*>(ufc);
    a.wfin = wfin;
    a.refine = 0;
    if ((e = cudaFuncSetAttribute(ism_panel_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem)) !=
        cudaSuccess)
        return e;
    void* args[] = {&tmU, &tmZ, &a};
    if (ev0) cudaEventRecord(ev0, s);
    e = cudaLaunchCooperativeKernel((const void*)ism_panel_tc05_kernel, dim3(L.grid), dim3(kThreads), args, L.smem, s);
    if (ev1) cudaEventRecord(ev1, s);
    return e;
}

// The stored factors of a tc5_solve (its V pieces, final-column pieces ufc and per-panel
// wfin) applied to p.Z, which holds R^-1 times a right-hand side: p.Z <- W^-1 R p.Z, the
// levels of Step 2 in panel form with no U columns left to update.  p.U, p.coefg, p.part
// and p.ctl as for the solve (U is not written); the grid-barrier word must be zero.
// p.gamma: the solve's gamma; p.C (nullable, N x N doubles): receives the per-level
// coefficients c_k = v_k^T x^(k-1) of the corrected columns.
cudaError_t tc5_correct(const Tc5Launch& L, const PanelArgs& p, const void* vpc, const void* ufc,
                        const float* wfin, cudaStream_t s) {
    CUtensorMap tmU, tmZ;
    memset(&tmU, 0, sizeof(tmU));
    memset(&tmZ, 0, sizeof(tmZ));
    if (!encode_f32_2d(&tmU, static_cast<const float*>(p.U), p.nobs, p.nens, p.ldu, 32, SWC, true) ||
        !encode_f32_2d(&tmZ, static_cast<const float*>(p.Z), p.nobs, p.nens, p.ldz, 32, SWC, true))
        return cudaErrorNotSupported;
    Tc5Args a;
    memset(&a, 0, sizeof(a));
    a.nobs = p.nobs;
    a.nens = p.nens;
    a.ntiles = L.ntiles;
    a.tiles_per_blk = L.tiles_per_blk;
    a.r = static_cast<const float*>(p.r);
    a.U = static_cast<float*>(p.U);
    a.ldu = p.ldu;
    a.Z = static_cast<float*>(p.Z);
    a.ldz = p.ldz;
    a.vpc = static_cast<const unsigned char*>(vpc);
    a.part = p.part;
    a.part_stride = L.part_stride;
    a.coefg = p.coefg;
    a.ctl = p.ctl;
    a.check = 0;
    a.timeout_ns = p.timeout_ns;
    a.ufc = const_cast<unsigned char*>(static_cast<const unsigned char*>(ufc));
    a.wfin = const_cast<float*>(wfin);
    a.refine = 1;
    a.C = p.C;              // nullable: the per-level coefficients of the corrected columns
    a.gamma = p.gamma;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ism_panel_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem)) !=
        cudaSuccess)
        return e;
    void* args[] = {&tmU, &tmZ, &a};
    return cudaLaunchCooperativeKernel((const void*)ism_panel_tc05_kernel, dim3(L.grid), dim3(kThreads), args, L.smem,
                                       s);
}

size_t tc5_wfin_bytes(int32_t nens) { return (size_t)((nens + PB - 1) / PB) * PB * PB * sizeof(float); }

}  // namespace enkf

#ifdef ENKF_TC5_TIMERS
// Profiling build only: copies the summed phase timers (SM cycles over all CTAs) to host
// and optionally clears them.
extern "C" __attribute__((visibility("default"))) int enkf_tc5_timers_read(unsigned long long* out, int n,
                                                                          int reset) {
    if (n > enkf::kNTimers) n = enkf::kNTimers;
    if (cudaMemcpyFromSymbol(out, enkf::g_tc5_timers, sizeof(unsigned long long) * n) != cudaSuccess) return -1;
    if (reset) {
        static const unsigned long long zero[enkf::kNTimers] = {};
        if (cudaMemcpyToSymbol(enkf::g_tc5_timers, zero, sizeof(zero)) != cudaSuccess) return -1;
    }
    return n;
}
#endif
