// Batched iterative Sherman-Morrison analyses (many independent, uneven problems
// in one persistent launch), FP32 storage with FP64 level denominators.
//
// One CTA solves one problem at a time; problems are taken from an atomic queue in
// longest-processing-time order.  Inside a CTA the problem's iterates X = [U | Z]
// live in a row-major copy (n x 2N) in the workspace, and the levels are applied
// in panels of b levels (b = 1 is the plain level-by-level recurrence):
//
//   panel P = {k0, .., k0+b-1}, trailing columns x = u_i (i >= k0+b) and all z_i:
//     a = V_P^T x                     (b dots per column, accumulated in the previous sweep)
//     G = V_P^T U_P                   (the same dots for the panel's own columns)
//     b x b recurrence (eqs. SM-step-2-h/u restricted to the panel; FP32 coefficient
//     vectors, gamma in double-FP32 -- the factor shared with the single-problem kernel):
//       gamma_m = 1 + (G beta_m)_m,   B[:,m] = beta_m / gamma_m,
//       beta_j <- beta_j - B[:,m] (G beta_j)_m   (j > m),      so h_m = U_P B[:,m];
//     c_m = v_m^T x^(m-1) = a_m - sum_{l<m} (G B)[m,l] c_l,  i.e. c = (I + L)^{-1} a;
//     x <- x - sum_m h_m c_m = x - U_P (B (I + L)^{-1} a) = x - U_P W a,  W = B (I+L)^{-1}.
//
// Each sweep reads and writes every trailing column once, applies the whole
// panel, and accumulates the next panel's a = V_{P'}^T x_new.  One thread owns one
// trailing column (several row groups when there are fewer than 256 columns), so
// the row-major layout makes every column access coalesced across a warp and the
// panel rows of U_P and V_{P'} are warp broadcasts.  The panel width b is chosen
// per size class by the autotuner (batch_tune in abi.cu).
//
// M = V^T Z / sqrt(N-1) is assembled without the cancellation of a direct product:
// with chat_{k,i} = c_{k,i} / gamma_k (the per-level Z coefficients, from the panel
// factor) and Q_km = v_k^T u_m^(m-1) (final, frozen U columns, materialised after
// each panel), V^T Z = (I - triu(Q, 1)) chat -- the identity used by the single-
// problem path.  Z is written back in the caller's column-major layout.
#include <math.h>

#include "internal.h"
#include "panel_factor.cuh"

namespace enkf {
namespace {

constexpr int kBT = 256;      // threads per CTA
constexpr int kBmax = 32;     // largest panel width

struct SmemB {
    float* apart;      // [kBT][kBmax]   per-thread partial dots
    float* A;          // [kBmax][256]   reduced dots a_t of each active column
    float* Gh;         // [kBmax][kBmax] panel Gram G = V_P^T U_P (Gl = 0: FP32 dots)
    float* Gl;         // [kBmax][kBmax]
    float* Bt;         // [kBmax][kBmax] Bt[m][u] = B[u][m]
    float* cb;         // [kBmax]
    float* Lt;         // [kBmax][kBmax] Lt[l][m] = L[m][l]
    float* W;          // [kBmax][kBmax] W = B (I + L)^{-1}
    float* Bf;         // [kBmax][kBmax] beta[u][m] = gamma_m B[u][m] (final panel columns)
    float* tile;       // [2][32][33] transpose tiles
    double* gam;       // [kBmax]
    int* flag;         // [4]
};
static_assert(kBmax == kFB, "panel factor width");

__device__ __forceinline__ int col_of(int a, int N, int k1) {
    // trailing columns after panel ending at k1: u_{k1..N-1}, then z_{0..N-1}
    const int nu = N - k1;
    return a < nu ? k1 + a : N + (a - nu);
}

// Step 1 into the row-major iterate: X[j][c] = V[j,c]/r_j, X[j][N+c] = D[j,c]/r_j, Vr[j][c] = V[j,c].
// 32 x 32 tiles, one per warp at a time in the warp's own shared-memory tiles (XOR-
// swizzled, 2 x 4 KB per warp): read coalesced over rows, written coalesced over
// columns, no CTA barrier in the loop.
__device__ void load_problem(const BatchDesc& d, const float* __restrict__ in, float* X, float* Vr, float* wtiles,
                             Control* ctl) {
    const int n = d.nobs, N = d.nens, ldX = d.ldX, ldVr = d.ldVr;
    const float* r = in + d.r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* t1 = wtiles + warp * (2 * 32 * 32);
    float* t2 = t1 + 32 * 32;
    const int ncb = (2 * N + 31) / 32, njb = (n + 31) / 32;
    __syncthreads();
    for (int tt = warp; tt < njb * ncb; tt += kBT / 32) {
        const int j0 = (tt / ncb) * 32, cb = tt % ncb;
        const int j = j0 + lane;
        const float rj = j < n ? r[j] : 1.f;
        if (j < n && (!(rj > 0.f) || !isfinite(rj))) set_status(ctl, kErrNumeric);
#pragma unroll
        for (int h = 0; h < 32; h += 16) {     // 16 columns in flight per lane
            float src[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int c = cb * 32 + h + q;
                src[q] = (c < 2 * N && j < n)
                             ? (c < N ? in[d.V + (int64_t)c * d.ldv + j] : in[d.D + (int64_t)(c - N) * d.ldd + j])
                             : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int cc = h + q;
                t1[cc * 32 + (lane ^ cc)] = src[q] / rj;
                t2[cc * 32 + (lane ^ cc)] = src[q];
            }
        }
        __syncwarp();
        const int c = cb * 32 + lane;
        for (int jj = 0; jj < 32; ++jj) {
            const int jr = j0 + jj;
            if (jr >= n) break;
            if (c < 2 * N) X[(int64_t)jr * ldX + c] = t1[lane * 32 + (jj ^ lane)];
            if (c < N) Vr[(int64_t)jr * ldVr + c] = t2[lane * 32 + (jj ^ lane)];
        }
        __syncwarp();
    }
    __syncthreads();
}

// One sweep over the trailing columns of the panel ending at k1 (columns k1.. of U
// and all of Z): if UPDATE, x -= U_P w with U_P = X[:, k0..k0+bp); if nb > 0,
// accumulate a_t = V[:, k1+t]^T x_new for t < nb.  Leaves the reduced dots in s.A.
template <int B>
__device__ void sweep(const BatchDesc& d, float* X, const float* Vr, const SmemB& s, int k0, int bp, int k1, int nb,
                      bool update) {
    const int n = d.nobs, N = d.nens, ldX = d.ldX, ldVr = d.ldVr;
    const int ncols = (N - k1) + N;
    const int G = kBT / ncols;           // row groups
    const int t = threadIdx.x;
    const bool active = t < G * ncols;
    const int a = active ? t % ncols : 0;
    const int g = active ? t / ncols : 0;
    float w[B];
    float acc[B];      // running dots; folded every 64 rows into this thread's row of s.apart
#pragma unroll
    for (int q = 0; q < B; ++q) acc[q] = 0.f, w[q] = 0.f;
    if (update && active) {
        // w = W a_col for this column (a_col = dots of the panel's V with this column, index a + bp)
#pragma unroll
        for (int q = 0; q < B; ++q) {
            float sum = 0.f;
            if (q < bp)
                for (int u = 0; u < bp; ++u) sum = fmaf(s.W[q * kBmax + u], s.A[u * 256 + a + bp], sum);
            w[q] = sum;
        }
    }
    __syncthreads();   // s.A is rewritten below
    if (active)
        for (int q = 0; q < B; ++q) s.apart[t * kBmax + q] = 0.f;
    // rows in blocks of 32: the panel rows of U_P and V_{P'} are staged in shared memory
    // (zero beyond bp / nb) and read as broadcasts, four per 16-byte load
    float* Us = s.tile;                 // [32][B]
    float* Vs = s.tile + 32 * kBmax;    // [32][B]
    const int col = active ? col_of(a, N, k1) : 0;
    int cnt = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
        __syncthreads();
        for (int e = t; e < 32 * B; e += kBT) {
            const int jj = e / B, q = e % B, j = j0 + jj;
            Us[e] = (update && q < bp && j < n) ? X[(int64_t)j * ldX + k0 + q] : 0.f;
            Vs[e] = (nb > 0 && q < nb && j < n) ? Vr[(int64_t)j * ldVr + k1 + q] : 0.f;
        }
        __syncthreads();
        if (!active) continue;
        const int jend = min(32, n - j0);
        for (int jq = g; jq < jend; jq += 4 * G) {
          float xq[4];   // the next four rows of this column, loaded ahead of their use
#pragma unroll
          for (int u = 0; u < 4; ++u) {
              const int jj = jq + u * G;
              xq[u] = jj < jend ? X[(int64_t)(j0 + jj) * ldX + col] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jj = jq + u * G;
            if (jj >= jend) break;
            const int64_t j = j0 + jj;
            float x = xq[u];
            if (update) {
#pragma unroll
                for (int q = 0; q < B; q += (B >= 4 ? 4 : 1)) {
                    if (B >= 4) {
                        const float4 u4 = *reinterpret_cast<const float4*>(Us + jj * B + q);
                        x = fmaf(-u4.x, w[q], x);
                        x = fmaf(-u4.y, w[q + 1], x);
                        x = fmaf(-u4.z, w[q + 2], x);
                        x = fmaf(-u4.w, w[q + 3], x);
                    } else {
                        x = fmaf(-Us[jj * B + q], w[q], x);
                    }
                }
                X[j * ldX + col] = x;
            }
            if (nb > 0) {
#pragma unroll
                for (int q = 0; q < B; q += (B >= 4 ? 4 : 1)) {
                    if (B >= 4) {
                        const float4 v4 = *reinterpret_cast<const float4*>(Vs + jj * B + q);
                        acc[q] = fmaf(v4.x, x, acc[q]);
                        acc[q + 1] = fmaf(v4.y, x, acc[q + 1]);
                        acc[q + 2] = fmaf(v4.z, x, acc[q + 2]);
                        acc[q + 3] = fmaf(v4.w, x, acc[q + 3]);
                    } else {
                        acc[q] = fmaf(Vs[jj * B + q], x, acc[q]);
                    }
                }
                if (++cnt == 64) {
                    cnt = 0;
#pragma unroll
                    for (int q = 0; q < B; ++q) s.apart[t * kBmax + q] += acc[q], acc[q] = 0.f;
                }
            }
          }
        }
    }
    if (active) {
#pragma unroll
        for (int q = 0; q < B; ++q) s.apart[t * kBmax + q] += acc[q];
    }
    __syncthreads();
    if (nb > 0) {
        // reduce the row groups in a fixed order: A[q][a] = sum_g apart[(g*ncols + a)][q]
        for (int e = threadIdx.x; e < nb * ncols; e += kBT) {
            const int q = e / ncols, aa = e % ncols;
            float sum = 0.f;
            for (int gg = 0; gg < G; ++gg) sum += s.apart[(gg * ncols + aa) * kBmax + q];
            s.A[q * 256 + aa] = sum;
        }
    }
    __syncthreads();
}

// Panel factor from the Gram G = A[:, 0..bp): gamma, B, L = (G B) strictly lower,
// W = B (I + L)^{-1} (factor_warp); latches kErrNumeric on a bad gamma.
__device__ bool factor(const SmemB& s, int bp, Control* ctl, bool check) {
    const int t = threadIdx.x;
    for (int e = t; e < kBmax * kBmax; e += kBT) {
        const int q = e / kBmax, u = e % kBmax;
        s.Gh[e] = (q < bp && u < bp) ? s.A[q * 256 + u] : 0.f;      // G[t][s] = v_t^T u_s
        s.Gl[e] = 0.f;
    }
    __syncthreads();
    if (t < 32) {
        factor_warp(s, bp);
        if (t < bp && check) {
            const double g = s.gam[t];
            if (!(g >= 1.0 - 64.0 * 1.1920928955078125e-07 * (1.0 + fabs(g - 1.0))) || !isfinite(g))
                set_status(ctl, kErrNumeric);
        }
    }
    __syncthreads();
    return true;
}

// Per-level Z coefficients of the panel [k0, k0+bp): c = (I + L)^{-1} a_z for every z
// column (a_z = previous sweep's dots, index (N - k0) + i), stored as chat = c / gamma.
__device__ void panel_z_coefficients(const BatchDesc& d, const SmemB& s, float* Ch, int k0, int bp) {
    const int N = d.nens;
    for (int i = threadIdx.x; i < N; i += kBT) {
        float c[kBmax];
        for (int m = 0; m < bp; ++m) {
            float v = s.A[m * 256 + (N - k0) + i];
            for (int l = 0; l < m; ++l) v = fmaf(-s.Lt[l * kBmax + m], c[l], v);
            c[m] = v;
            Ch[(int64_t)(k0 + m) * N + i] = v / (float)s.gam[m];
        }
    }
    __syncthreads();
}

// Final values of the panel's own columns, u_m^(m-1) = gamma_m U_P B[:,m] = U_P beta_m, in
// place.  beta[u][m] = 0 for u > m, so each output sums over every u < bp in the order of
// the triangular sum; the rows of beta are read four at a time.
template <int B>
__device__ void panel_final_columns(const BatchDesc& d, float* X, const SmemB& s, int k0, int bp) {
    for (int j = threadIdx.x; j < d.nobs; j += kBT) {
        float* row = X + (int64_t)j * d.ldX + k0;
        float acc[B];
#pragma unroll
        for (int m = 0; m < B; ++m) acc[m] = 0.f;
        for (int u = 0; u < bp; ++u) {
            const float x = row[u];
            const float* bu = s.Bf + u * kBmax;
#pragma unroll
            for (int m = 0; m < B; m += (B >= 4 ? 4 : 1)) {
                if (B >= 4) {
                    const float4 b4 = *reinterpret_cast<const float4*>(bu + m);
                    acc[m] = fmaf(x, b4.x, acc[m]);
                    acc[m + 1] = fmaf(x, b4.y, acc[m + 1]);
                    acc[m + 2] = fmaf(x, b4.z, acc[m + 2]);
                    acc[m + 3] = fmaf(x, b4.w, acc[m + 3]);
                } else {
                    acc[m] = fmaf(x, bu[m], acc[m]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < B; ++m)
            if (m < bp) row[m] = acc[m];
    }
    __syncthreads();
}

// M = V^T Z / sqrt(N-1) and Z out (column-major).  256 threads, thread -> (k, i) blocks.
__device__ void finish_problem(const BatchDesc& d, float* __restrict__ out, const float* X, const float* Vr,
                               float* tile, float* stage, const float* Ch, float* ws_q) {
    const int n = d.nobs, N = d.nens, ldX = d.ldX, ldVr = d.ldVr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Z out: transpose X[:, N..2N) -> Z (column-major)
    if (d.Z >= 0) {
        // one 32 x 32 tile per warp at a time in the warp's own shared-memory tile
        float* wt = stage + warp * (32 * 32);   // XOR-swizzled 32 x 32 tile
        const int ncb = (N + 31) / 32, njb = (n + 31) / 32;
        __syncthreads();
        for (int tt = warp; tt < njb * ncb; tt += kBT / 32) {
            const int j0 = (tt / ncb) * 32, cb = tt % ncb;
            const int c = cb * 32 + lane;
#pragma unroll
            for (int h = 0; h < 32; h += 16) {
                float row[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = j0 + h + q;
                    row[q] = (j < n && c < N) ? X[(int64_t)j * ldX + N + c] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) wt[(h + q) * 32 + (lane ^ (h + q))] = row[q];
            }
            __syncwarp();
            const int j = j0 + lane;
            for (int cc = 0; cc < 32; ++cc) {
                const int cz = cb * 32 + cc;
                if (cz >= N) break;
                if (j < n) out[d.Z + (int64_t)cz * d.ldz + j] = wt[lane * 32 + (cc ^ lane)];
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (d.M >= 0 && N >= 2) {
        // Q_km = v_k^T u_m (k < m) in 4 x 4 blocks (N % 4 == 0), FP32 products folded into FP64
        // every 32 rows; then M = (I - triu(Q,1)) chat / sqrt(N-1).
        float* Qw = ws_q;
        const int nb4 = N / 4;
        const int nblk = nb4 * (nb4 + 1) / 2;            // upper blocks kb <= mb
        float* Vt = stage;                               // [32][N] rows of V
        float* Ut = stage + 32 * N;                      // [32][N] rows of the final U
        for (int b0 = 0; b0 < nblk; b0 += kBT) {
            int kb = 0, mb = 0;
            const int blk = b0 + threadIdx.x;
            if (blk < nblk) {                            // blk -> (kb, mb), kb <= mb, row by row
                int t = blk;
                while (t >= nb4 - kb) t -= nb4 - kb, ++kb;
                mb = kb + t;
            }
            float acc[16];
            double accd[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.f, accd[q] = 0.0;
            for (int j0 = 0; j0 < n; j0 += 32) {
                __syncthreads();
                for (int e = threadIdx.x; e < 32 * (N / 4); e += kBT) {
                    const int jj = e / (N / 4), c4 = (e % (N / 4)) * 4, j = j0 + jj;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f), u = v;
                    if (j < n) {
                        v = *reinterpret_cast<const float4*>(Vr + (int64_t)j * ldVr + c4);
                        u = *reinterpret_cast<const float4*>(X + (int64_t)j * ldX + c4);
                    }
                    *reinterpret_cast<float4*>(Vt + jj * N + c4) = v;
                    *reinterpret_cast<float4*>(Ut + jj * N + c4) = u;
                }
                __syncthreads();
                if (blk < nblk) {
                    for (int jj = 0; jj < 32; ++jj) {
                        const float4 v = *reinterpret_cast<const float4*>(Vt + jj * N + 4 * kb);
                        const float4 u = *reinterpret_cast<const float4*>(Ut + jj * N + 4 * mb);
                        const float vv[4] = {v.x, v.y, v.z, v.w};
                        const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int p = 0; p < 4; ++p) acc[q * 4 + p] = fmaf(vv[q], uu[p], acc[q * 4 + p]);
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) accd[q] += (double)acc[q], acc[q] = 0.f;   // every 32 rows
                }
            }
            if (blk < nblk) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        Qw[(int64_t)(4 * kb + q) * N + 4 * mb + p] = (float)accd[q * 4 + p];
            }
        }
        __syncthreads();
        const float scale = (float)(1.0 / sqrt((double)(N - 1)));
        for (int e = threadIdx.x; e < N * N; e += kBT) {
            const int k = e / N, i = e % N;   // a warp shares k (Q row broadcast), chat rows coalesced
            float v = Ch[(int64_t)k * N + i];
            for (int m = k + 1; m < N; ++m) v = fmaf(-Qw[(int64_t)k * N + m], Ch[(int64_t)m * N + i], v);
            out[d.M + k + (int64_t)i * N] = v * scale;
        }
    }
    __syncthreads();
}

template <int B>
__device__ void solve_problem(const BatchDesc& d, const float* in, float* out, float* ws, const SmemB& s,
                              Control* ctl, bool check) {
    float* X = ws + d.X;
    float* Vr = ws + d.Vr;
    float* Ch = ws + d.Ch;
    const int N = d.nens;
    load_problem(d, in, X, Vr, s.apart, ctl);
    // initial dots of panel 0 with every column
    int bp = B < N ? B : N;
    sweep<B>(d, X, Vr, s, 0, 0, 0, bp, false);
    for (int k0 = 0; k0 < N; k0 += B) {
        bp = (N - k0) < B ? (N - k0) : B;
        factor(s, bp, ctl, check);
        panel_z_coefficients(d, s, Ch, k0, bp);
        const int k1 = k0 + bp;
        const int nb = (N - k1) < B ? (N - k1) : B;
        sweep<B>(d, X, Vr, s, k0, bp, k1, nb, true);
        panel_final_columns<B>(d, X, s, k0, bp);
    }
    finish_problem(d, out, X, Vr, s.tile, s.apart, Ch, ws + d.Qw);
}

__global__ void __launch_bounds__(kBT, 2) ism_batch_kernel(const BatchDesc* __restrict__ desc,
                                                        const int* __restrict__ order, int nprob,
                                                        const float* in, float* out, float* ws, Control* ctl,
                                                        int check, int force_b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemB s;
    s.apart = reinterpret_cast<float*>(smem_raw);
    s.A = s.apart + kBT * kBmax;
    s.gam = reinterpret_cast<double*>(s.A + kBmax * 256);
    s.Gh = reinterpret_cast<float*>(s.gam + kBmax);
    s.Gl = s.Gh + kBmax * kBmax;
    s.Bt = s.Gl + kBmax * kBmax;
    s.Lt = s.Bt + kBmax * kBmax;
    s.cb = s.Lt + kBmax * kBmax;
    s.W = s.cb + kBmax;
    s.Bf = s.W + kBmax * kBmax;
    s.tile = s.Bf + kBmax * kBmax;
    s.flag = reinterpret_cast<int*>(s.tile + 2 * 32 * 33);
    for (;;) {
        if (threadIdx.x == 0) s.flag[0] = atomicAdd(&ctl->barrier, 1u);
        __syncthreads();
        const int idx = s.flag[0];
        __syncthreads();
        if (idx >= nprob) break;
        const BatchDesc d = desc[order[idx]];
        const int b = force_b > 0 ? force_b : d.b;
        switch (b) {
            case 1: solve_problem<1>(d, in, out, ws, s, ctl, check); break;
            case 8: solve_problem<8>(d, in, out, ws, s, ctl, check); break;
            case 16: solve_problem<16>(d, in, out, ws, s, ctl, check); break;
            default: solve_problem<32>(d, in, out, ws, s, ctl, check); break;
        }
    }
}

}  // namespace

size_t batch_smem_bytes() {
    return sizeof(float) * (size_t)kBT * kBmax + sizeof(float) * kBmax * 256 + sizeof(double) * kBmax +
           sizeof(float) * (6 * kBmax * kBmax + kBmax) + sizeof(float) * 2 * 32 * 33 + 16;
}

cudaError_t batch_configure(int* grid) {
    const size_t smem = batch_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(ism_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ism_batch_kernel, kBT, smem)) != cudaSuccess) return e;
    *grid = nsm * (occ > 0 ? occ : 1);
    return cudaSuccess;
}

cudaError_t batch_launch(int grid, const BatchDesc* desc, const int* order, int nprob, const float* in, float* out,
                         float* ws, Control* ctl, int check, int force_b, cudaStream_t s) {
    ism_batch_kernel<<<grid, kBT, batch_smem_bytes(), s>>>(desc, order, nprob, in, out, ws, ctl, check, force_b);
    return cudaGetLastError();
}

}  // namespace enkf
