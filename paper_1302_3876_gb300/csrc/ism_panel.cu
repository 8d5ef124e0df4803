// Panel form of the iterative Sherman-Morrison solve for one large problem, on
// FP32 CUDA cores: b levels of Step 2 (eqs. SM-step-2-h/Z/u) per pass over HBM.
//
// For a panel P = {k0..k0+b-1} and every trailing column x (u_i, i >= k0+b, and
// all z_i), with a = V_P^T x (dots accumulated in the previous pass) and the panel
// Gram G = V_P^T U_P:
//   gamma_m = 1 + (G beta_m)_m,  B[:,m] = beta_m / gamma_m,
//   beta_j <- beta_j - B[:,m] (G beta_j)_m   (j > m)          (so h_m = U_P B[:,m])
//   c = (I + L)^{-1} a,  L = strictly lower part of G B        (c_m = v_m^T x^(m-1))
//   x <- x - U_P W a,    W = B (I + L)^{-1}
// which is the level-by-level recurrence regrouped (equal in exact arithmetic).
// The panel's own columns end as u_m^(m-1) = gamma_m U_P B[:,m]; they are written
// back so that the Gram V^T U of the M assembly sees the same final U as the
// level-by-level path.  The per-level Z coefficients c_{k,i} (rows of C) and
// gamma_k are produced by the factor, in FP64.
//
// Layout: one persistent cooperative launch; each CTA owns a fixed block of rows.
// Per panel: every CTA factors the b x b Gram redundantly (FP64), then sweeps its
// rows in 64 x 64 tiles of X (column-major, coalesced 64-row segments): the
// update GEMM X -= U_P W' (K = b) and the next panel's dots A' += V_{P'}^T X_new
// (K = rows), both register-tiled from shared memory.  A' partials are reduced
// across CTAs in a fixed order between two bounded grid barriers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "internal.h"
#include "panel_factor.cuh"

namespace enkf {
namespace {

constexpr int kPT = 256;    // threads
constexpr int kPB = 32;     // largest panel width
constexpr int RT = 64;      // rows per tile
constexpr int CT = 64;      // columns per tile
constexpr int XLD = RT + 4; // padded tile stride (keeps 16-byte alignment)
constexpr int kScratch = 256 * 16;   // floats: A tile of W' (kPB*CT) or the GEMM2 row-half combine (256*16)

struct PanelSmem {
    // factor temporaries (alias the X tiles, dead between sweeps)
    float* Gh;      // [kPB][kPB]  panel Gram, hi part (float)
    float* Gl;      // [kPB][kPB]  panel Gram, lo part: G = Gh + Gl to ~2^-48
    float* Bt;      // [kPB][kPB]  Bt[m][u] = B[u][m]
    float* cb;      // [kPB]       one column of beta
    // persistent through the sweep
    float* Lt;      // [kPB][kPB]  Lt[l][m] = L[m][l] (strictly lower part of G B)
    double* gam;    // [kPB]
    double* red;    // [32]
    float* W;       // [kPB][kPB]
    float* Bf;      // [kPB][kPB]  beta[u][m] = gamma_m B[u][m] (for the final panel columns)
    float* Wt;      // [kPB][CT]   W' = W A[:, tile]
    float* Xs;      // [CT][XLD]
    float* UPs;     // [kPB][RT]
    float* VNs;     // [kPB][RT]
    int* flag;      // [4]
    // column base pointers of the current column tile (staging source, write-back
    // destination) and of the panel's U and V columns
    const float** psrc;   // [CT]
    float** pdst;         // [CT]
    float** pu;           // [kPB]
    const float** pv;     // [kPB]
    // tensor-core variants: 16-bit operand tiles (hi, and lo for the split form)
    // (pieces: [0] = hi, [1] = the next 8 bits, [2] = the last 8 bits)
    unsigned short* U3[3];     // [kPB][HP]   -U_P, [t][row]
    unsigned short* W3[3];     // [CT][WPT]   W',   [col][t]
    unsigned short* X3[3];     // [CT][HP]    X,    [col][row]
    unsigned short* V3[3];     // [kPB][HP]   V',   [t][row]
};
constexpr int HP = RT + 8;     // 16-bit tile pitch along rows
constexpr int WPT = kPB + 8;   // 16-bit tile pitch along t
// 16-bit elements of one operand piece (U3 and V3 two stages, W3, X3): piece q of an array
// is piece 0 plus q * kPiece
constexpr int kPiece = 4 * kPB * HP + CT * WPT + CT * HP;

__device__ __forceinline__ float* col_ptr(const PanelArgs& a, int c) {
    return c < a.nens ? static_cast<float*>(a.U) + (int64_t)c * a.ldu
                      : static_cast<float*>(a.Z) + (int64_t)(c - a.nens) * a.ldz;
}

// trailing column a of the panel ending at k1 -> full column index (U: [0,N), Z: [N,2N))
__device__ __forceinline__ int trail_col(int a, int N, int k1) {
    const int nu = N - k1;
    return a < nu ? k1 + a : N + (a - nu);
}

// Cross-CTA sum of the partial dots in a fixed order: each CTA owns a slice of the
// entries; a team of threads per entry sums a fixed residue class of CTAs, then
// the team's subtotals are added in team order.
__device__ bool reduce_panel(const PanelArgs& a, const PanelSmem& s, int nvals, unsigned& epoch) {
    const unsigned nblk = gridDim.x;
    if (!grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, s.flag)) return false;
    const int per = (nvals + nblk - 1) / nblk;
    const int e0 = blockIdx.x * per;
    double* sub = reinterpret_cast<double*>(s.Xs);          // scratch: [kPT] doubles
    for (int eb = 0; eb < per; eb += kPT) {
        const int ne = min(kPT, per - eb);
        const int teams = kPT / ne;
        const int t = threadIdx.x, e = t % ne, g = t / ne;
        double v = 0.0;
        if (g < teams && e0 + eb + e < nvals) {
            const double* src = a.part + e0 + eb + e;
            unsigned b = g;
            for (; b + 3 * teams < nblk; b += 4 * teams) {   // four loads in flight, summed in order
                const double x0 = __ldcg(src + (int64_t)b * a.part_stride);
                const double x1 = __ldcg(src + (int64_t)(b + teams) * a.part_stride);
                const double x2 = __ldcg(src + (int64_t)(b + 2 * teams) * a.part_stride);
                const double x3 = __ldcg(src + (int64_t)(b + 3 * teams) * a.part_stride);
                v += x0;
                v += x1;
                v += x2;
                v += x3;
            }
            for (; b < nblk; b += teams) v += __ldcg(src + (int64_t)b * a.part_stride);
        }
        __syncthreads();
        sub[t] = v;
        __syncthreads();
        if (t < ne && e0 + eb + t < nvals) {
            double tot = 0.0;
            for (int gg = 0; gg < teams; ++gg) tot += sub[gg * ne + t];
            __stcg(&a.coefg[e0 + eb + t], tot);
        }
    }
    return grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, s.flag);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Stages rows [row0, row0 + nr) of ncl columns into a [col][XLD] tile (zero fill past nr / ncl).
// VEC: 16-byte copies (column bases 16-byte aligned and row0 % 4 == 0), else 4-byte copies.
template <bool VEC, typename ColFn>
__device__ __forceinline__ void stage_cols(float* dst, int ld, int ncols_tile, int ncl, int64_t row0, int nr, ColFn col) {
    const int tid = threadIdx.x;
    if (VEC) {
        for (int e = tid; e < ncols_tile * (RT / 4); e += kPT) {
            const int c = e >> 4, j4 = (e & 15) * 4;
            const int rem = nr - j4;
            const int bytes = (c < ncl && rem > 0) ? (rem >= 4 ? 16 : 4 * rem) : 0;
            const float* src = bytes ? col(c) + row0 + j4 : col(0) + row0;   // valid address even when 0 bytes
            cp_async16(dst + c * ld + j4, src, bytes);
        }
    } else {
        for (int e = tid; e < ncols_tile * RT; e += kPT) {
            const int c = e >> 6, j = e & 63;
            const int bytes = (c < ncl && j < nr) ? 4 : 0;
            cp_async4(dst + c * ld + j, bytes ? col(c) + row0 + j : col(0) + row0, bytes);
        }
    }
}

// Sweep options.
constexpr int kMaterialize = 1;   // write the panel's final U columns (last column tile)
constexpr int kStep1 = 2;         // first sweep: stage V and D, apply Step 1, write U and Z

// Step 1 (eq. SM-step-1) on a staged tile: x[c][j] = x[c][j] * (1 / r_j) -- one reciprocal per
// row and a product per element (at most one rounding more than a division).
__device__ __forceinline__ void scale_tile(float* xs, const float* r, int64_t row0, int nr) {
    const int j = threadIdx.x & 63;
    if (j < nr) {
        const float inv = 1.0f / r[row0 + j];
#pragma unroll 4
        for (int c = threadIdx.x >> 6; c < CT; c += kPT / 64) xs[c * XLD + j] = xs[c * XLD + j] * inv;
    }
}

// Writes the ncl columns of a staged tile back to rows [row0, row0 + nr): 16-byte stores along rows.
template <bool VEC, typename ColFn>
__device__ __forceinline__ void writeback_tile(const float* xs, int ncl, int64_t row0, int nr, ColFn col) {
    for (int e = threadIdx.x; e < CT * (RT / 4); e += kPT) {
        const int c = e >> 4, j4 = (e & 15) * 4;
        if (c >= ncl) continue;
        float* dst = col(c) + row0 + j4;
        const float4 v = *reinterpret_cast<const float4*>(&xs[c * XLD + j4]);
        if (VEC && j4 + 4 <= nr) {
            *reinterpret_cast<float4*>(dst) = v;
        } else {
            const float vv[4] = {v.x, v.y, v.z, v.w};
            for (int q = 0; q < 4; ++q)
                if (j4 + q < nr) dst[q] = vv[q];
        }
    }
}

// Final values of the panel's own columns on one row tile: u_{k0+m}^(k0+m-1) =
// gamma_m U_P B[:,m] = U_P beta_m, from the U_P rows staged in shared memory
// (ups: [t][row]).  Called in the sweep's last column tile, when no later stage
// reads these rows of U_P.
__device__ __forceinline__ void materialize_tile(const PanelArgs& a, const PanelSmem& s, const float* ups, int k0,
                                                 int bp, int64_t row0, int nr) {
    // thread: rows r4..r4+3, levels m and m + 16; beta[u][m] = 0 for u > m, so the sum runs
    // over every u < bp in the same order as the triangular one
    static_assert(RT == 64 && kPT == 256 && kPB == 32, "thread mapping");
    const int r4 = (threadIdx.x & 15) * 4, mg = threadIdx.x >> 4;
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
    for (int u = 0; u < bp; ++u) {
        const float4 x = *reinterpret_cast<const float4*>(&ups[u * RT + r4]);
        const float b0 = s.Bf[u * kPB + mg], b1 = s.Bf[u * kPB + mg + 16];
        acc0[0] = fmaf(x.x, b0, acc0[0]), acc0[1] = fmaf(x.y, b0, acc0[1]);
        acc0[2] = fmaf(x.z, b0, acc0[2]), acc0[3] = fmaf(x.w, b0, acc0[3]);
        acc1[0] = fmaf(x.x, b1, acc1[0]), acc1[1] = fmaf(x.y, b1, acc1[1]);
        acc1[2] = fmaf(x.z, b1, acc1[2]), acc1[3] = fmaf(x.w, b1, acc1[3]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = mg + 16 * h;
        if (m >= bp) continue;
        const float* v = h ? acc1 : acc0;
        float* dst = s.pu[m] + row0 + r4;
        if (r4 + 4 <= nr && ((uintptr_t)dst & 15) == 0) {
            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            for (int q = 0; q < 4; ++q)
                if (r4 + q < nr) dst[q] = v[q];
        }
    }
}

// One sweep over this CTA's rows for the panel [k0, k0+bp) (bp = 0: no update) and
// the next panel [k1, k1+nb) (nb = 0: no dots).  A (reduced dots of the previous
// sweep) is read from coefg with row stride ncols_prev = ncols + bp.
// Thread tiles use interleaved columns (c = x + 16 q) so that the 16-byte shared
// loads of 16 lanes fall in distinct banks.
template <bool VEC>
__device__ void sweep_t(const PanelArgs& a, const PanelSmem& s, int64_t r0, int64_t nrows, int k0, int bp, int ku,
                        int kv, int nb, int aoff, int opts) {
    const int N = a.nens;
    const int k1 = ku;   // trailing U columns start here (N: none)
    const int ncols = (N - k1) + N;
    const int ncols_prev = ncols + aoff;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float* V = static_cast<const float*>(a.V);
    const float* D = static_cast<const float*>(a.D);
    const float* r = static_cast<const float*>(a.r);
    const bool step1 = (opts & kStep1) != 0;
    const int ntiles = (int)((nrows + RT - 1) / RT);
    // GEMM2 mapping: columns cq + 16 q, dot rows tq*4 + s, row half
    const int cq = tid & 15, tq = (tid >> 4) & 7, half = tid >> 7;
    for (int c0 = 0; c0 < ncols; c0 += CT) {
        const int ncl = min(CT, ncols - c0);
        __syncthreads();
        if (bp > 0) {
            // A tile (float) then W'[t][c] = sum_u W[t][u] A[u][c], stored permuted: Wt[t][x*4+q] = W'[t][x+16q]
            float* As = s.VNs + 2 * kPB * RT;    // [kPB][CT] scratch after the double-buffered tiles
            for (int e = tid; e < bp * CT; e += kPT) {
                const int u = e >> 6, c = e & 63;
                As[u * CT + c] = c < ncl ? (float)__ldcg(&a.coefg[u * ncols_prev + c0 + c + aoff]) : 0.f;
            }
            __syncthreads();
            for (int e = tid; e < bp * CT; e += kPT) {
                const int t = e >> 6, c = e & 63;
                float v = 0.f;
                for (int u = 0; u < bp; ++u) v = fmaf(s.W[t * kPB + u], As[u * CT + c], v);
                s.Wt[t * CT + (c & 15) * 4 + (c >> 4)] = v;
            }
        }
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
        auto xcol = [&](int c) { return col_ptr(a, trail_col(c0 + c, N, k1)); };
        auto scol = [&](int c) -> const float* {       // staging source: V / D for the Step-1 sweep
            const int cc = trail_col(c0 + c, N, k1);
            if (!step1) return col_ptr(a, cc);
            return cc < N ? V + (int64_t)cc * a.ldv : D + (int64_t)(cc - N) * a.ldd;
        };
        auto ucol = [&](int t) { return col_ptr(a, k0 + t); };
        auto vcol = [&](int t) { return V + (int64_t)(kv + t) * a.ldv; };
        if (tid < CT) {
            const int c = tid < ncl ? tid : 0;   // a valid address for zero-byte copies
            s.psrc[tid] = scol(c);
            s.pdst[tid] = xcol(c);
        } else if (tid < CT + kPB) {
            const int t = tid - CT;
            s.pu[t] = ucol(t < bp ? t : 0);
            s.pv[t] = vcol(t < nb ? t : 0);
        }
        auto psrc = [&](int c) { return s.psrc[c]; };
        auto pdst = [&](int c) { return s.pdst[c]; };
        auto pu = [&](int t) { return s.pu[t]; };
        auto pv = [&](int t) { return s.pv[t]; };
        auto stage = [&](int tile, int buf) {
            const int64_t rr = (int64_t)tile * RT;
            const int nr = (int)min((int64_t)RT, nrows - rr);
            const int64_t row0 = r0 + rr;
            float* xs = s.Xs + buf * CT * XLD;
            stage_cols<VEC>(xs, XLD, CT, ncl, row0, nr, psrc);
            if (bp > 0) stage_cols<VEC>(s.UPs + buf * kPB * RT, RT, bp, bp, row0, nr, pu);
            if (nb > 0) stage_cols<VEC>(s.VNs + buf * kPB * RT, RT, nb, nb, row0, nr, pv);
            cp_async_commit();
        };
        __syncthreads();
        stage(0, 0);
        for (int tile = 0; tile < ntiles; ++tile) {
            const int buf = tile & 1;
            // this tile's copies (the only ones in flight) have landed; after the barrier every
            // thread is also done with the other buffer, so the next tile is staged into it
            cp_async_wait<0>();
            __syncthreads();
            if (tile + 1 < ntiles) stage(tile + 1, buf ^ 1);
            float* xs = s.Xs + buf * CT * XLD;
            const float* ups = s.UPs + buf * kPB * RT;
            const float* vns = s.VNs + buf * kPB * RT;
            const int64_t rr = (int64_t)tile * RT;
            const int nr = (int)min((int64_t)RT, nrows - rr);
            if (step1) {
                scale_tile(xs, r, r0 + rr, nr);
                __syncthreads();
                writeback_tile<VEC>(xs, ncl, r0 + rr, nr, pdst);
            }
            if (bp > 0) {
                // GEMM1: rows 4 ty.., columns tx + 16 q
                float x[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(&xs[(tx + 16 * q) * XLD + ty * 4]);
                    x[0][q] = v.x, x[1][q] = v.y, x[2][q] = v.z, x[3][q] = v.w;
                }
#pragma unroll 4
                for (int t = 0; t < bp; ++t) {
                    const float4 u = *reinterpret_cast<const float4*>(&ups[t * RT + ty * 4]);
                    const float4 w = *reinterpret_cast<const float4*>(&s.Wt[t * CT + tx * 4]);
                    const float uu[4] = {u.x, u.y, u.z, u.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int q = 0; q < 4; ++q) x[i][q] = fmaf(-uu[i], ww[q], x[i][q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<float4*>(&xs[(tx + 16 * q) * XLD + ty * 4]) =
                        make_float4(x[0][q], x[1][q], x[2][q], x[3][q]);
                __syncthreads();
                writeback_tile<VEC>(xs, ncl, r0 + rr, nr, pdst);
                if ((opts & kMaterialize) && c0 + CT >= ncols) materialize_tile(a, s, ups, k0, bp, r0 + rr, nr);
            }
            if (nb > 0 && tq * 4 < nb) {
                // GEMM2: acc[s][q] += sum_j VN[tq*4+s][j] X[cq+16q][j] over this thread's row half
                const int jb = half * (RT / 2);
#pragma unroll 2
                for (int j = jb; j < jb + RT / 2; j += 4) {
                    float4 xv[4], vv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) xv[q] = *reinterpret_cast<const float4*>(&xs[(cq + 16 * q) * XLD + j]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) vv[q] = *reinterpret_cast<const float4*>(&vns[(tq * 4 + q) * RT + j]);
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[s4][q] = fmaf(vv[s4].x, xv[q].x, fmaf(vv[s4].y, xv[q].y,
                                         fmaf(vv[s4].z, xv[q].z, fmaf(vv[s4].w, xv[q].w, acc[s4][q]))));
                }
            }
        }
        if (nb > 0) {
            // combine the two row halves in a fixed order, then write this CTA's partial
            float* red = s.VNs + 2 * kPB * RT;   // [256][16] scratch
            __syncthreads();
            if (half == 1)
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                    for (int q = 0; q < 4; ++q) red[(tid - 128) * 16 + s4 * 4 + q] = acc[s4][q];
            __syncthreads();
            if (half == 0 && tq * 4 < nb) {
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    const int t = tq * 4 + s4;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = cq + 16 * q;
                        if (t < nb && c < ncl)
                            __stcg(&a.part[(int64_t)blockIdx.x * a.part_stride + t * ncols + c0 + c],
                                   (double)(acc[s4][q] + red[tid * 16 + s4 * 4 + q]));
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core sweep (mma.sync m16n8k16, FP32 accumulation).  Operands are split into
// P 16-bit pieces x = x_0 + x_1 + ... and the products x_i y_j with i + j < P are
// summed, smallest first:
//   PREC 1  BF16, P = 2 (hi + lo, three products; operands kept to ~2^-17)
//   PREC 2  FP16, P = 1 (one product)
//   PREC 3  BF16, P = 3 (hi + mid + lo, six products; operands kept to ~2^-25, FP32-class)
// Same data flow as the FP32 sweep; the two GEMMs of a 64 x 64 tile:
//   GEMM1  X <- X + (-U_P) W'      (M = rows, N = columns, K = t), accumulators start at X
//   GEMM2  A' += V'^T X_new        (M = t, N = columns, K = rows), accumulators persist
// ---------------------------------------------------------------------------
template <int PREC>
struct Tc;
template <>
struct Tc<1> {
    static constexpr int pieces = 2;
    static __device__ __forceinline__ unsigned short hi(float x) { return __bfloat16_as_ushort(__float2bfloat16(x)); }
    static __device__ __forceinline__ float back(unsigned short h) { return __bfloat162float(__ushort_as_bfloat16(h)); }
    static __device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
template <>
struct Tc<2> {
    static constexpr int pieces = 1;
    static __device__ __forceinline__ unsigned short hi(float x) { return __half_as_ushort(__float2half_rn(x)); }
    static __device__ __forceinline__ float back(unsigned short h) { return __half2float(__ushort_as_half(h)); }
    static __device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

template <>
struct Tc<3> : Tc<1> {
    static constexpr int pieces = 3;
};

__device__ __forceinline__ void ldsm4(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm2(uint32_t* r, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// The P pieces of x: each is the 16-bit rounding of what the previous ones leave
// (the subtractions are exact in FP32).
template <int PREC>
__device__ __forceinline__ void split_pieces(float x, unsigned short* out) {
    float rest = x;
#pragma unroll
    for (int p = 0; p < Tc<PREC>::pieces; ++p) {
        out[p] = Tc<PREC>::hi(rest);
        if (p + 1 < Tc<PREC>::pieces) rest = rest - Tc<PREC>::back(out[p]);
    }
}

// The pieces of 4 floats stored as 4 consecutive 16-bit values in each piece array.
template <int PREC>
__device__ __forceinline__ void put4(unsigned short* d0, unsigned short* d1, unsigned short* d2, int off, float4 v) {
    unsigned short x[3], y[3], z[3], w[3];
    split_pieces<PREC>(v.x, x);
    split_pieces<PREC>(v.y, y);
    split_pieces<PREC>(v.z, z);
    split_pieces<PREC>(v.w, w);
    *reinterpret_cast<uint2*>(d0 + off) =
        make_uint2((uint32_t)x[0] | ((uint32_t)y[0] << 16), (uint32_t)z[0] | ((uint32_t)w[0] << 16));
    if (Tc<PREC>::pieces > 1)
        *reinterpret_cast<uint2*>(d1 + off) =
            make_uint2((uint32_t)x[1] | ((uint32_t)y[1] << 16), (uint32_t)z[1] | ((uint32_t)w[1] << 16));
    if (Tc<PREC>::pieces > 2)
        *reinterpret_cast<uint2*>(d2 + off) =
            make_uint2((uint32_t)x[2] | ((uint32_t)y[2] << 16), (uint32_t)z[2] | ((uint32_t)w[2] << 16));
}

// d += sum over piece pairs (i, j), i + j < P, of a_i b_j, smallest terms first
// (P = 2: a1 b0, a0 b1, a0 b0; P = 3: a2 b0, a1 b1, a0 b2, a1 b0, a0 b1, a0 b0).
template <int PREC>
__device__ __forceinline__ void mma_pieces(float* d, const uint32_t (&a)[Tc<PREC>::pieces][4],
                                           const uint32_t (&b0)[Tc<PREC>::pieces],
                                           const uint32_t (&b1)[Tc<PREC>::pieces]) {
    constexpr int P = Tc<PREC>::pieces;
#pragma unroll
    for (int sum = P - 1; sum >= 0; --sum)
#pragma unroll
        for (int i = sum; i >= 0; --i) Tc<PREC>::mma(d, a[i], b0[sum - i], b1[sum - i]);
}

template <bool VEC, int PREC>
__device__ void sweep_tc(const PanelArgs& a, const PanelSmem& s, int64_t r0, int64_t nrows, int k0, int bp, int ku,
                         int kv, int nb, int aoff, int opts) {
    constexpr int P = Tc<PREC>::pieces;
    const int N = a.nens;
    const int k1 = ku;
    const int ncols = (N - k1) + N;
    const int ncols_prev = ncols + aoff;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* V = static_cast<const float*>(a.V);
    const float* D = static_cast<const float*>(a.D);
    const float* r = static_cast<const float*>(a.r);
    const bool step1 = (opts & kStep1) != 0;
    const int ntiles = (int)((nrows + RT - 1) / RT);
    const int j8 = lane >> 3;
    for (int c0 = 0; c0 < ncols; c0 += CT) {
        const int ncl = min(CT, ncols - c0);
        __syncthreads();
        if (bp > 0) {
            float* As = s.VNs + 2 * kPB * RT;    // [kPB][CT]
            for (int e = tid; e < bp * CT; e += kPT) {
                const int u = e >> 6, c = e & 63;
                As[u * CT + c] = c < ncl ? (float)__ldcg(&a.coefg[u * ncols_prev + c0 + c + aoff]) : 0.f;
            }
            __syncthreads();
            // W'[t][c] into [col][t] 16-bit tiles; t >= bp is zero padding of K
            for (int e = tid; e < kPB * CT; e += kPT) {
                const int t = e >> 6, c = e & 63;
                float v = 0.f;
                if (t < bp)
                    for (int u = 0; u < bp; ++u) v = fmaf(s.W[t * kPB + u], As[u * CT + c], v);
                unsigned short pc[3];
                split_pieces<PREC>(-v, pc);   // -W': GEMM1 multiplies the pieces of +U_P
#pragma unroll
                for (int q = 0; q < P; ++q) s.W3[q][c * WPT + t] = pc[q];
            }
        }
        float acc2[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 4; ++h) acc2[mt][h] = 0.f;
        auto xcol = [&](int c) { return col_ptr(a, trail_col(c0 + c, N, k1)); };
        auto scol = [&](int c) -> const float* {       // staging source: V / D for the Step-1 sweep
            const int cc = trail_col(c0 + c, N, k1);
            if (!step1) return col_ptr(a, cc);
            return cc < N ? V + (int64_t)cc * a.ldv : D + (int64_t)(cc - N) * a.ldd;
        };
        auto ucol = [&](int t) { return col_ptr(a, k0 + t); };
        auto vcol = [&](int t) { return V + (int64_t)(kv + t) * a.ldv; };
        if (tid < CT) {
            const int c = tid < ncl ? tid : 0;   // a valid address for zero-byte copies
            s.psrc[tid] = scol(c);
            s.pdst[tid] = xcol(c);
        } else if (tid < CT + kPB) {
            const int t = tid - CT;
            s.pu[t] = ucol(t < bp ? t : 0);
            s.pv[t] = vcol(t < nb ? t : 0);
        }
        auto psrc = [&](int c) { return s.psrc[c]; };
        auto pdst = [&](int c) { return s.pdst[c]; };
        auto pu = [&](int t) { return s.pu[t]; };
        auto pv = [&](int t) { return s.pv[t]; };
        const bool mat_here = (opts & kMaterialize) && c0 + CT >= ncols;
        const int pidx = bp > 0 ? k0 / a.panel_b : 0;
        const int64_t uplane = (int64_t)kPB * a.ldp, ubuf = P * uplane, vplane = (int64_t)N * a.ldp;
        auto stage = [&](int tile, int buf) {
            const int64_t rr = (int64_t)tile * RT;
            const int nr = (int)min((int64_t)RT, nrows - rr);
            const int64_t row0 = r0 + rr;
            stage_cols<VEC>(s.Xs + buf * CT * XLD, XLD, CT, ncl, row0, nr, psrc);
            if (bp > 0) {
                if (mat_here) stage_cols<VEC>(s.UPs + buf * kPB * RT, RT, bp, bp, row0, nr, pu);
                // pieces of U_P and V_{P'}: [t][row] tiles, 16-byte copies of 8 rows, zero past nr / bp / nb
                for (int e = tid; e < 2 * P * kPB * (RT / 8); e += kPT) {
                    const int j8r = (e & 7) * 8, t = (e >> 3) % kPB, q = (e >> 3) / kPB % P, isv = e / (P * kPB * 8);
                    const int lim = isv ? nb : bp;
                    const int rem = nr - j8r;
                    const int bytes = (t < lim && rem > 0) ? (rem >= 8 ? 16 : 2 * rem) : 0;
                    const unsigned short* src =
                        isv ? a.vp + q * vplane + (int64_t)(kv + (t < lim ? t : 0)) * a.ldp + row0 + j8r
                            : a.up + (pidx & 1) * ubuf + q * uplane + (int64_t)(t < lim ? t : 0) * a.ldp + row0 + j8r;
                    unsigned short* dst = (isv ? s.V3[0] : s.U3[0]) + q * kPiece + buf * kPB * HP + t * HP + j8r;
                    cp_async16(dst, bytes ? src : a.vp, bytes);
                }
            } else if (nb > 0) {
                stage_cols<VEC>(s.VNs + buf * kPB * RT, RT, nb, nb, row0, nr, pv);
            }
            cp_async_commit();
        };
        __syncthreads();
        stage(0, 0);
        for (int tile = 0; tile < ntiles; ++tile) {
            const int buf = tile & 1;
            // this tile's copies (the only ones in flight) have landed; after the barrier every
            // thread is also done with the other buffer, so the next tile is staged into it
            cp_async_wait<0>();
            __syncthreads();
            if (tile + 1 < ntiles) stage(tile + 1, buf ^ 1);
            float* xs = s.Xs + buf * CT * XLD;
            const float* ups = s.UPs + buf * kPB * RT;
            const float* vns = s.VNs + buf * kPB * RT;
            const int64_t rr = (int64_t)tile * RT;
            const int nr = (int)min((int64_t)RT, nrows - rr);
            const int64_t row0 = r0 + rr;
            if (step1) {
                // pieces of the staged V columns (the source of U), kept for the later sweeps
                for (int e = tid; e < CT * (RT / 4); e += kPT) {
                    const int c = e >> 4, r4 = (e & 15) * 4;
                    const int cc = trail_col(c0 + c, N, k1);
                    if (c < ncl && cc < N && r4 < nr)
                        put4<PREC>(a.vp + cc * a.ldp, a.vp + vplane + cc * a.ldp, a.vp + 2 * vplane + cc * a.ldp,
                                   (int)(row0 + r4), *reinterpret_cast<const float4*>(&xs[c * XLD + r4]));
                }
                __syncthreads();
                scale_tile(xs, r, r0 + rr, nr);
                __syncthreads();
                // pieces of panel 0's U_P = the first columns of U after Step 1
                if (c0 == 0)
                    for (int e = tid; e < kPB * (RT / 4); e += kPT) {
                        const int c = e >> 4, r4 = (e & 15) * 4;
                        if (c < ncl && c < N && c < a.panel_b && r4 < nr)
                            put4<PREC>(a.up + c * a.ldp, a.up + uplane + c * a.ldp, a.up + 2 * uplane + c * a.ldp,
                                       (int)(row0 + r4), *reinterpret_cast<const float4*>(&xs[c * XLD + r4]));
                    }
            }
            if (bp == 0) {
                // first sweep: V' tile pieces from the staged FP32 columns (zero rows t >= nb)
                for (int e = tid; e < kPB * (RT / 4); e += kPT) {
                    const int t = e >> 4, r4 = (e & 15) * 4;
                    if (nb > 0) {
                        const float4 v =
                            t < nb ? *reinterpret_cast<const float4*>(&vns[t * RT + r4]) : make_float4(0, 0, 0, 0);
                        put4<PREC>(s.V3[0] + buf * kPB * HP, s.V3[1] + buf * kPB * HP, s.V3[2] + buf * kPB * HP,
                                   t * HP + r4, v);
                    }
                }
                for (int e = tid; e < CT * (RT / 4); e += kPT) {
                    const int c = e >> 4, r4 = (e & 15) * 4;
                    put4<PREC>(s.X3[0], s.X3[1], s.X3[2], c * HP + r4,
                               *reinterpret_cast<const float4*>(&xs[c * XLD + r4]));
                }
            }
            __syncthreads();
            if (bp > 0) {
                // GEMM1: warp -> rows mt*16.., columns nb0.. (4 n-tiles)
                const int mt = warp & 3, nb0 = (warp >> 2) * 32;
                // the update (-U_P W') accumulates from zero in the tensor core; X is added
                // afterwards with an IEEE FP32 add (tensor-core accumulation is truncating, and
                // its error would otherwise scale with |X| rather than with the update)
                float acc1[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int h = 0; h < 4; ++h) acc1[nt][h] = 0.f;
                for (int kk = 0; kk < bp; kk += 16) {
                    uint32_t af[P][4];
                    const int kr = kk + (j8 >> 1) * 8 + (lane & 7);
                    const int mr = mt * 16 + (j8 & 1) * 8;
#pragma unroll
                    for (int q = 0; q < P; ++q) ldsm4t(af[q], s.U3[q] + buf * kPB * HP + kr * HP + mr);
#pragma unroll
                    for (int np = 0; np < 2; ++np) {
                        const int nr2 = nb0 + np * 16 + (j8 >> 1) * 8 + (lane & 7);
                        const int kc = kk + (j8 & 1) * 8;
                        uint32_t bf[P][4];
#pragma unroll
                        for (int q = 0; q < P; ++q) ldsm4(bf[q], s.W3[q] + nr2 * WPT + kc);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            uint32_t b0[P], b1[P];
#pragma unroll
                            for (int q = 0; q < P; ++q) b0[q] = bf[q][2 * hh], b1[q] = bf[q][2 * hh + 1];
                            mma_pieces<PREC>(acc1[np * 2 + hh], af, b0, b1);
                        }
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int row = mt * 16 + (lane >> 2) + (h >> 1) * 8;
                        const int col = nb0 + nt * 8 + (lane & 3) * 2 + (h & 1);
                        const float v = xs[col * XLD + row] + acc1[nt][h];
                        xs[col * XLD + row] = v;
                        unsigned short pc[3];
                        split_pieces<PREC>(v, pc);
#pragma unroll
                        for (int q = 0; q < P; ++q) s.X3[q][col * HP + row] = pc[q];
                    }
                __syncthreads();
                writeback_tile<VEC>(xs, ncl, r0 + rr, nr, pdst);
                if (c0 == 0) {
                    // pieces of the next panel's U_P: trailing columns 0.. = u_{k1..} after this panel
                    const int nbn = min(a.panel_b, N - k1);
                    unsigned short* ub = a.up + ((pidx + 1) & 1) * ubuf;
                    for (int e = tid; e < kPB * (RT / 4); e += kPT) {
                        const int c = e >> 4, r4 = (e & 15) * 4;
                        if (c < nbn && c < ncl && r4 < nr)
                            put4<PREC>(ub + c * a.ldp, ub + uplane + c * a.ldp, ub + 2 * uplane + c * a.ldp,
                                       (int)(row0 + r4), *reinterpret_cast<const float4*>(&xs[c * XLD + r4]));
                    }
                }
                if (mat_here) materialize_tile(a, s, ups, k0, bp, r0 + rr, nr);
            }
            if (step1) writeback_tile<VEC>(xs, ncl, r0 + rr, nr, pdst);
            if (nb > 0) {
                // GEMM2: warp -> columns warp*8.. (one n-tile), t = 0..31 (two m-tiles), K = 64 rows;
                // the tile's sum starts at zero and is folded into acc2 with IEEE FP32 adds
                float tile2[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int h = 0; h < 4; ++h) tile2[mt][h] = 0.f;
#pragma unroll
                for (int kk = 0; kk < RT; kk += 16) {
                    uint32_t bf[P][2];
                    const int nrow = warp * 8 + (lane & 7);
                    const int kc = kk + ((lane >> 3) & 1) * 8;
#pragma unroll
                    for (int q = 0; q < P; ++q) ldsm2(bf[q], s.X3[q] + nrow * HP + kc);
                    uint32_t b0[P], b1[P];
#pragma unroll
                    for (int q = 0; q < P; ++q) b0[q] = bf[q][0], b1[q] = bf[q][1];
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        if (mt * 16 >= nb) continue;
                        uint32_t af[P][4];
                        const int mrow = mt * 16 + (j8 & 1) * 8 + (lane & 7);
                        const int kcol = kk + (j8 >> 1) * 8;
#pragma unroll
                        for (int q = 0; q < P; ++q) ldsm4(af[q], s.V3[q] + buf * kPB * HP + mrow * HP + kcol);
                        mma_pieces<PREC>(tile2[mt], af, b0, b1);
                    }
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int h = 0; h < 4; ++h) acc2[mt][h] += tile2[mt][h];
            }
        }
        if (nb > 0) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int t = mt * 16 + (lane >> 2) + (h >> 1) * 8;
                    const int c = warp * 8 + (lane & 3) * 2 + (h & 1);
                    if (t < nb && c < ncl)
                        __stcg(&a.part[(int64_t)blockIdx.x * a.part_stride + t * ncols + c0 + c], (double)acc2[mt][h]);
                }
        }
    }
}

// Sweep over this CTA's rows: update the trailing columns (u_ku.., all z) with the
// panel [k0, k0+bp) and accumulate the dots with v_kv.. (nb of them).  aoff: offset
// of the trailing columns in the previous sweep's column list; materialize: write
// the panel's final U columns.
template <int PREC>
__device__ void sweep(const PanelArgs& a, const PanelSmem& s, int64_t r0, int64_t nrows, int k0, int bp, int ku,
                      int kv, int nb, int aoff, int opts) {
    if (PREC == 0) {
        if (a.vec_ok)
            sweep_t<true>(a, s, r0, nrows, k0, bp, ku, kv, nb, aoff, opts);
        else
            sweep_t<false>(a, s, r0, nrows, k0, bp, ku, kv, nb, aoff, opts);
    } else {
        if (a.vec_ok)
            sweep_tc<true, PREC == 0 ? 1 : PREC>(a, s, r0, nrows, k0, bp, ku, kv, nb, aoff, opts);
        else
            sweep_tc<false, PREC == 0 ? 1 : PREC>(a, s, r0, nrows, k0, bp, ku, kv, nb, aoff, opts);
    }
}

// Stored-factor recurrence for the refinement (FP32 CUDA-core sweeps): applies
//   x <- x - h_m (v_m^T x),  h_m = u_m / gamma'_m,  gamma'_m = 1 + v_m^T u_m,   m = 0..N-1
// to the N columns held in Z (R^-1 times a residual), where u_m are the final U columns
// left by the solve and every inner product v_k^T u_m comes from one Gram Q = V^T U
// (row-major), so the b x b factors need no reduction.  Per panel: c = (I + L)^{-1}
// V_P^T x with L[m][l] = Q[m][l] / gamma'_l (l < m), then x <- x - U_P diag(1/gamma') c.
__device__ void refine_body(const PanelArgs& a, const PanelSmem& s, int64_t r0, int64_t nrows, unsigned& epoch) {
    const int N = a.nens, b = a.panel_b;
    const int tid = threadIdx.x;
    int nb = b < N ? b : N;
    sweep<0>(a, s, r0, nrows, 0, 0, N, 0, nb, 0, 0);
    if (!reduce_panel(a, s, nb * N, epoch)) return;
    for (int k0 = 0; k0 < N; k0 += b) {
        const int bp = (N - k0) < b ? (N - k0) : b;
        const int k1 = k0 + bp;
        if (tid < 32) {
            // gamma'_l = 1 + Q[l][l] and L[m][l] = Q[m][l] / gamma'_l (lane l), B = diag(1/gamma'),
            // then W = B (I + L)^{-1}
            const int l = tid;
            if (l < bp) {
                const double ginv = 1.0 / (1.0 + a.Qg[(int64_t)(k0 + l) * N + (k0 + l)]);
                for (int m = 0; m < bp; ++m) {
                    s.Lt[l * kPB + m] = m > l ? (float)(a.Qg[(int64_t)(k0 + m) * N + (k0 + l)] * ginv) : 0.f;
                    s.Bt[m * kPB + l] = m == l ? (float)ginv : 0.f;
                }
            }
            __syncwarp();
            panel_w(s, bp);
        }
        __syncthreads();
        nb = (N - k1) < b ? (N - k1) : b;
        sweep<0>(a, s, r0, nrows, k0, bp, N, k1, nb, 0, 0);
        if (nb > 0) {
            if (!reduce_panel(a, s, nb * N, epoch)) return;
        } else {
            break;
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kPT, PREC == 0 ? 2 : 1) ism_panel_kernel(PanelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // persistent: L, gamma, W, Bf, W'; tile buffers; the factor's temporaries G, beta, B
    // alias the X tile buffers (they are dead between sweeps)
    PanelSmem s;
    s.Lt = reinterpret_cast<float*>(smem_raw);
    s.gam = reinterpret_cast<double*>(s.Lt + kPB * kPB);
    s.red = s.gam + kPB;
    s.W = reinterpret_cast<float*>(s.red + 32);
    s.Bf = s.W + kPB * kPB;
    s.Wt = s.Bf + kPB * kPB;
    s.Xs = s.Wt + kPB * CT;
    s.UPs = s.Xs + 2 * CT * XLD;
    s.VNs = s.UPs + 2 * kPB * RT;
    s.flag = reinterpret_cast<int*>(s.VNs + 2 * kPB * RT + kScratch);
    {
        void** tab = reinterpret_cast<void**>(s.flag + 4);
        s.psrc = static_cast<const float**>(static_cast<void*>(tab));
        s.pdst = reinterpret_cast<float**>(tab + CT);
        s.pu = reinterpret_cast<float**>(tab + 2 * CT);
        s.pv = static_cast<const float**>(static_cast<void*>(tab + 2 * CT + kPB));
    }
    s.Gh = s.Xs;
    s.Gl = s.Gh + kPB * kPB;
    s.Bt = s.Gl + kPB * kPB;
    s.cb = s.Bt + kPB * kPB;
    {
        unsigned short* h = reinterpret_cast<unsigned short*>(reinterpret_cast<void**>(s.flag + 4) + 2 * CT + 2 * kPB);
        constexpr int NP = PREC == 0 ? 0 : Tc<PREC == 0 ? 1 : PREC>::pieces;
        // U3 and V3 hold two stages ([stage][t][row]); W3 and X3 one
        s.U3[0] = h; h += NP > 0 ? 2 * kPB * HP : 0;
        s.W3[0] = h; h += NP > 0 ? CT * WPT : 0;
        s.X3[0] = h; h += NP > 0 ? CT * HP : 0;
        s.V3[0] = h; h += NP > 0 ? 2 * kPB * HP : 0;
        s.U3[1] = h; h += NP > 1 ? 2 * kPB * HP : 0;
        s.W3[1] = h; h += NP > 1 ? CT * WPT : 0;
        s.X3[1] = h; h += NP > 1 ? CT * HP : 0;
        s.V3[1] = h; h += NP > 1 ? 2 * kPB * HP : 0;
        s.U3[2] = h; h += NP > 2 ? 2 * kPB * HP : 0;
        s.W3[2] = h; h += NP > 2 ? CT * WPT : 0;
        s.X3[2] = h; h += NP > 2 ? CT * HP : 0;
        s.V3[2] = h;
    }
    static_assert(3 * kPB * kPB + kPB <= 2 * CT * XLD, "factor temporaries fit the tiles");

    const int N = a.nens, b = a.panel_b;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_blk;
    const int64_t r1 = min(r0 + (int64_t)a.rows_per_blk, a.nobs);
    const int64_t nrows = r1 > r0 ? r1 - r0 : 0;
    unsigned epoch = 0;
    const float* r = static_cast<const float*>(a.r);

    if (a.refine) {   // correction sweep: U holds the final columns, Z the scaled residual
        refine_body(a, s, r0, nrows, epoch);
        return;
    }
    // ---- Step 1 (eq. SM-step-1), U = R^-1 V and Z = R^-1 D, is applied by the first sweep
    if (a.check)
        for (int64_t j = tid; j < nrows; j += kPT) {
            const float rj = r[r0 + j];
            if (!(rj > 0.f && isfinite(rj))) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = 0;
            }
        }
    __syncthreads();
    // ---- Step 1 and the dots of panel 0 with every column
    int nb = b < N ? b : N;
    sweep<PREC>(a, s, r0, nrows, 0, 0, 0, 0, nb, 0, kStep1);
    if (!reduce_panel(a, s, nb * 2 * N, epoch)) return;

    for (int k0 = 0; k0 < N; k0 += b) {
        const int bp = (N - k0) < b ? (N - k0) : b;
        const int k1 = k0 + bp;
        const int ncols_prev = (N - k0) + N;
        // factor of the panel (every CTA): the FP64 Gram split into float hi + lo
        for (int e = tid; e < kPB * kPB; e += kPT) {
            const int t = e / kPB, u = e % kPB;
            const double g = (t < bp && u < bp) ? __ldcg(&a.coefg[t * ncols_prev + u]) : 0.0;
            const float h = (float)g;
            s.Gh[e] = h;
            s.Gl[e] = (float)(g - (double)h);
        }
        __syncthreads();
        if (tid < 32) factor_warp(s, bp);
        __syncthreads();
        if (blockIdx.x == 0 && tid < bp) {
            const double g = s.gam[tid];
            a.gamma[k0 + tid] = g;
            if (a.check && (!(g >= 1.0 - 64.0 * 1.1920928955078125e-07 * (1.0 + fabs(g - 1.0))) || !isfinite(g))) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = k0 + tid + 1;
            }
        }
        // per-level Z coefficients c = (I + L)^{-1} a of z_i (one warp per column, CTAs
        // round-robin over the columns): lane m holds a_m, level l broadcasts c_l
        for (int i = blockIdx.x * (kPT / 32) + (tid >> 5); i < N; i += gridDim.x * (kPT / 32)) {
            const int lane = tid & 31;
            const int ai = (N - k0) + i;   // index of z_i among the previous sweep's columns
            float v = lane < bp ? (float)__ldcg(&a.coefg[lane * ncols_prev + ai]) : 0.f;
            for (int l = 0; l < bp; ++l) {
                const float cl = __shfl_sync(0xffffffffu, v, l);
                if (lane > l) v = fmaf(-s.Lt[l * kPB + lane], cl, v);
            }
            if (lane < bp) a.C[(int64_t)(k0 + lane) * N + i] = (double)v;
        }
        nb = (N - k1) < b ? (N - k1) : b;
        // every CTA has read coefg; it is rewritten only after the next barrier
        sweep<PREC>(a, s, r0, nrows, k0, bp, k1, k1, nb, bp, kMaterialize);
        if (nb > 0) {
            if (!reduce_panel(a, s, nb * ((N - k1) + N), epoch)) return;
        } else {
            break;
        }
    }
}

size_t panel_smem(int prec) {
    const size_t base = sizeof(double) * (kPB + 32) +
                        sizeof(float) * (3 * kPB * kPB + kPB * CT + 2 * CT * XLD + 4 * kPB * RT + kScratch) + 16 +
                        sizeof(void*) * (2 * CT + 2 * kPB);
    const int pieces = prec == 1 ? 2 : prec == 2 ? 1 : prec == 3 ? 3 : 0;
    const size_t tc = sizeof(unsigned short) * pieces * (4 * kPB * HP + CT * WPT + CT * HP);
    return base + tc;
}

const void* panel_kernel_ptr(int prec) {
    return prec == 1   ? (const void*)ism_panel_kernel<1>
           : prec == 2 ? (const void*)ism_panel_kernel<2>
           : prec == 3 ? (const void*)ism_panel_kernel<3>
                       : (const void*)ism_panel_kernel<0>;
}

}  // namespace

int panel_max_b() { return kPB; }

int panel_pieces(int prec) { return prec == 1 ? 2 : prec == 2 ? 1 : prec == 3 ? 3 : 0; }

cudaError_t panel_plan(int64_t nobs, int32_t nens, int32_t b, int32_t prec, PanelLaunch* L) {
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const size_t smem = panel_smem(prec);
    const void* fn = panel_kernel_ptr(prec);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPT, smem)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    occ = occ > 2 ? 2 : occ;
    int64_t grid = (int64_t)nsm * occ;
    const int64_t by_rows = (nobs + RT - 1) / RT;
    if (grid > by_rows) grid = by_rows;
    int64_t rpb = (nobs + grid - 1) / grid;
    rpb = (rpb + 7) / 8 * 8;   // 16-byte aligned rows of the 16-bit piece arrays
    grid = (nobs + rpb - 1) / rpb;
    L->grid = (int)grid;
    L->threads = kPT;
    L->smem = smem;
    L->rows_per_blk = (int)rpb;
    L->b = b;
    L->prec = prec;
    L->part_stride = (int64_t)b * 2 * nens;   // largest nb * ncols
    return cudaSuccess;
}

cudaError_t panel_launch(const PanelLaunch& L, PanelArgs a, cudaStream_t s) {
    a.rows_per_blk = L.rows_per_blk;
    a.panel_b = L.b;
    a.part_stride = L.part_stride;
    void* args[] = {&a};
    const void* fn = panel_kernel_ptr(L.prec);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(L.grid), dim3(L.threads), args, L.smem, s);
}

}  // namespace enkf
