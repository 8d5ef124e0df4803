// Inflation and partial localization around the SMEnKF analysis (Sec. 3.1.1 and
// Sec. 3.1.2), with the C-ABI entry points enkf_inflate_prep and
// enkf_localized_update (declared in include/enkf_ism.h).
//
// enkf_inflate_prep: multiplicative inflation x_i <- xbar + alpha (x_i - xbar)
// fused into the centering observation prep: the row's members are read once for the
// mean and once more to write the inflated ensemble, its deviations,
// V = H dX_B / sqrt(Nens - 1) and D = Y - H X_B (FP64 storage: one thread per row, FP64
// arithmetic; FP32 storage: 32-row tiles, compensated FP32 arithmetic).
//
// enkf_localized_update: X_A = X_B + (Delta o (S V^T)) Z, S = dX_B / sqrt(Nens - 1),
// Delta = (delta_ij) the impact factors of observation j on state component i:
// exp(-d / length) inside the radius of influence, 0 outside, d the periodic
// distance between state index i and the observed index j * stride.  One CTA owns
// 32 state rows and every member: it stages its rows of S once, then for each
// block of 32 observations in the tile's band stages V and Z, forms the 32 x 32
// block T = Delta o (S V^T) (K = Nens) in shared memory and accumulates T Z into
// registers (K = 32).  Two contractions per observation block, FP32 or FP64
// CUDA-core arithmetic; the band is a superset of the radius, the exact weight
// decides.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace enkf {
namespace {

enkf_status lfail(enkf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

enkf_status lcuda(cudaError_t e, const char* what) {
    return lfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------------------------
// inflation fused into the centering prep
// ---------------------------------------------------------------------------------------------

template <typename T>
__global__ void inflate_center_observe_kernel(int64_t nstate, int64_t nobs, int n, int stride, double alpha,
                                              T* __restrict__ XB, int64_t ldb, T* __restrict__ dXB, int64_t ldx,
                                              const T* __restrict__ Y, int64_t ldy, T* __restrict__ V, int64_t ldv,
                                              T* __restrict__ D, int64_t ldd, double scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nstate;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int e = 0; e < n; ++e) s += (double)XB[(int64_t)e * ldb + i];
        const double mean = s / (double)n;
        const bool observed = (i % stride == 0) && (i / stride < nobs);
        const int64_t j = i / stride;
        for (int e = 0; e < n; ++e) {
            const double x = (double)XB[(int64_t)e * ldb + i];
            const T xi = (T)(mean + alpha * (x - mean));
            XB[(int64_t)e * ldb + i] = xi;
            const T d = (T)((double)xi - mean);
            if (dXB) dXB[(int64_t)e * ldx + i] = d;
            if (observed) {
                V[(int64_t)e * ldv + j] = (T)((double)d * scale);
                if (Y) D[(int64_t)e * ldd + j] = Y[(int64_t)e * ldy + j] - xi;
            }
        }
    }
}

// FP32 storage: FP32 arithmetic only (per-element FP64 arithmetic and conversions would run on
// GB300's narrow FP64 pipe).  A CTA takes tiles of 32 rows; lane = row, warp w sums members
// w, w + 8, ... with a compensated (Neumaier) FP32 sum, the eight partials are combined in a
// fixed order, and the mean is kept as an unevaluated pair mh + ml (ml = the rounding residual
// of mh), so deviations are formed as (x - mh) - ml.  The second pass re-reads the tile (16 KB at
// 128 members, an L2 hit) and writes the outputs.  alpha == 1 leaves X_B untouched.
constexpr int kInfWarps = 8;

__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

__global__ void __launch_bounds__(kInfWarps * 32) inflate_prep_f32_kernel(
    int64_t nstate, int64_t nobs, int n, int stride, float alpha, int inflate, float* __restrict__ XB, int64_t ldb,
    float* __restrict__ dXB, int64_t ldx, const float* __restrict__ Y, int64_t ldy, float* __restrict__ V,
    int64_t ldv, float* __restrict__ D, int64_t ldd, float scale) {
    __shared__ float ps[kInfWarps][32], pc[kInfWarps][32], mhs[32], mls[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i0 = (int64_t)blockIdx.x * 32; i0 < nstate; i0 += (int64_t)gridDim.x * 32) {
        const int64_t i = i0 + lane;
        const bool in = i < nstate;
        float s = 0.f, c = 0.f;
        if (in) {
#pragma unroll 4
            for (int e = warp; e < n; e += kInfWarps) neumaier_add(s, c, XB[(int64_t)e * ldb + i]);
        }
        ps[warp][lane] = s;
        pc[warp][lane] = c;
        __syncthreads();
        if (warp == 0) {
            float S = 0.f, C = 0.f;
            for (int w = 0; w < kInfWarps; ++w) {
                neumaier_add(S, C, ps[w][lane]);
                C += pc[w][lane];
            }
            const float tot = S + C;
            const float lo = C - (tot - S);                       // S + C = tot + lo
            const float mh = tot / (float)n;
            const float ml = (fmaf(-mh, (float)n, tot) + lo) / (float)n;
            mhs[lane] = mh;
            mls[lane] = ml;
        }
        __syncthreads();
        const float mh = mhs[lane], ml = mls[lane];
        const bool observed = in && (i % stride == 0) && (i / stride < nobs);
        const int64_t j = i / stride;
        if (in) {
            for (int e = warp; e < n; e += kInfWarps) {
                const float x = XB[(int64_t)e * ldb + i];
                float xi = x;
                if (inflate) {
                    xi = mh + fmaf(alpha, (x - mh) - ml, ml);
                    XB[(int64_t)e * ldb + i] = xi;
                }
                const float d = (xi - mh) - ml;
                if (dXB) dXB[(int64_t)e * ldx + i] = d;
                if (observed) {
                    V[(int64_t)e * ldv + j] = d * scale;
                    if (Y) D[(int64_t)e * ldd + j] = Y[(int64_t)e * ldy + j] - xi;
                }
            }
        }
        __syncthreads();                                         // ps / mhs reused by the next tile
    }
}

// ---------------------------------------------------------------------------------------------
// partial localization
// ---------------------------------------------------------------------------------------------

constexpr int kTI = 32;        // state rows per CTA
constexpr int kTJ = 32;        // observations per staged block
constexpr int kLocThreads = 256;
constexpr int kLocMaxN = 256;  // members (register tile: 4 rows x 8 column groups of 32 per thread)

template <typename T>
struct LocArgs {
    int64_t nstate, nobs;
    int32_t n, stride;
    double inv_length;         // 1 / correlation length (0: delta = 1 inside the radius)
    double radius;             // < 0: no cut-off
    int64_t band;              // ceil(radius) when the tile's band is narrower than the ring, else -1
    double scale;              // 1 / sqrt(n - 1)
    const T* dXB; int64_t ldx;
    const T* V; int64_t ldv;
    const T* Z; int64_t ldz;
    const T* XB; int64_t ldb;
    T* XA; int64_t lda;
};

__host__ __device__ inline int loc_pitch(int n) { return n | 1; }   // odd row pitch: conflict-free columns

template <typename T>
size_t loc_smem_bytes(int n) {
    const int sp = loc_pitch(n);
    return sizeof(T) * ((size_t)kTI * sp + 2 * (size_t)kTJ * sp + (size_t)kTI * (kTJ + 1));
}

// Observation index ranges [lo, hi] (at most two) whose locations can fall within the band of
// state rows [i0, i0 + kTI) on the ring.  A superset: the weight is decided per pair.
template <typename T>
__device__ int loc_ranges(const LocArgs<T>& a, int64_t i0, int64_t* lo, int64_t* hi) {
    if (a.band < 0) {
        lo[0] = 0;
        hi[0] = a.nobs - 1;
        return 1;
    }
    const int64_t p = i0 - a.band, q = i0 + kTI - 1 + a.band;   // q - p + 1 < nstate
    int64_t sp[2], sq[2];
    int ns = 0;
    if (p < 0) {
        sp[ns] = p + a.nstate; sq[ns++] = a.nstate - 1;
        sp[ns] = 0; sq[ns++] = q;
    } else if (q >= a.nstate) {
        sp[ns] = p; sq[ns++] = a.nstate - 1;
        sp[ns] = 0; sq[ns++] = q - a.nstate;
    } else {
        sp[ns] = p; sq[ns++] = q;
    }
    int nr = 0;
    for (int r = 0; r < ns; ++r) {
        const int64_t jl = (sp[r] + a.stride - 1) / a.stride;
        int64_t jh = sq[r] / a.stride;
        if (jh > a.nobs - 1) jh = a.nobs - 1;
        if (jl <= jh) {
            lo[nr] = jl;
            hi[nr++] = jh;
        }
    }
    return nr;
}

template <typename T>
__device__ __forceinline__ T loc_weight(const LocArgs<T>& a, int64_t i, int64_t j) {
    int64_t d = i - j * (int64_t)a.stride;
    if (d < 0) d = -d;
    if (a.nstate - d < d) d = a.nstate - d;
    if (a.radius >= 0.0 && (double)d > a.radius) return T(0);
    if (sizeof(T) == 8) return (T)exp(-(double)d * a.inv_length);
    return (T)expf(-(float)d * (float)a.inv_length);
}

template <typename T>
__global__ void __launch_bounds__(kLocThreads) localized_update_kernel(LocArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ss = reinterpret_cast<T*>(smem_raw);          // [kTI][sp]  rows of dX_B (later: the accumulators)
    const int n = a.n, sp = loc_pitch(n);
    T* Vs = Ss + (size_t)kTI * sp;                  // [kTJ][sp]
    T* Zs = Vs + (size_t)kTJ * sp;                  // [kTJ][sp]
    T* Ts = Zs + (size_t)kTJ * sp;                  // [kTI][kTJ + 1]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kTI;

    for (int idx = t; idx < kTI * n; idx += kLocThreads) {
        const int i = idx % kTI, k = idx / kTI;
        const int64_t gi = i0 + i;
        Ss[i * sp + k] = gi < a.nstate ? a.dXB[(int64_t)k * a.ldx + gi] : T(0);
    }

    T acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = T(0);

    int64_t lo[2], hi[2];
    const int nr = loc_ranges(a, i0, lo, hi);
    const int ti = t >> 4, tj = t & 15;             // T tile: rows ti, ti + 16; columns tj, tj + 16
    for (int r = 0; r < nr; ++r) {
        for (int64_t jb = lo[r]; jb <= hi[r]; jb += kTJ) {
            __syncthreads();                        // previous block's Vs / Zs / Ts no longer read
            for (int idx = t; idx < kTJ * n; idx += kLocThreads) {
                const int jj = idx % kTJ, k = idx / kTJ;
                const int64_t gj = jb + jj;
                const bool ok = gj <= hi[r];
                Vs[jj * sp + k] = ok ? a.V[(int64_t)k * a.ldv + gj] : T(0);
                Zs[jj * sp + k] = ok ? a.Z[(int64_t)k * a.ldz + gj] : T(0);
            }
            __syncthreads();
            T s00 = 0, s01 = 0, s10 = 0, s11 = 0;
            const T* S0 = Ss + ti * sp;
            const T* S1 = Ss + (ti + 16) * sp;
            const T* V0 = Vs + tj * sp;
            const T* V1 = Vs + (tj + 16) * sp;
            for (int k = 0; k < n; ++k) {
                const T x0 = S0[k], x1 = S1[k], y0 = V0[k], y1 = V1[k];
                s00 = fma(x0, y0, s00);
                s01 = fma(x0, y1, s01);
                s10 = fma(x1, y0, s10);
                s11 = fma(x1, y1, s11);
            }
            const T sc = (T)a.scale;
            const int64_t gj0 = jb + tj, gj1 = jb + tj + 16;
            Ts[ti * (kTJ + 1) + tj] = s00 * sc * loc_weight(a, i0 + ti, gj0);
            Ts[ti * (kTJ + 1) + tj + 16] = s01 * sc * loc_weight(a, i0 + ti, gj1);
            Ts[(ti + 16) * (kTJ + 1) + tj] = s10 * sc * loc_weight(a, i0 + ti + 16, gj0);
            Ts[(ti + 16) * (kTJ + 1) + tj + 16] = s11 * sc * loc_weight(a, i0 + ti + 16, gj1);
            __syncthreads();
            const T* Tw = Ts + (warp * 4) * (kTJ + 1);
#pragma unroll 4
            for (int j = 0; j < kTJ; ++j) {
                const T w0 = Tw[j], w1 = Tw[(kTJ + 1) + j], w2 = Tw[2 * (kTJ + 1) + j], w3 = Tw[3 * (kTJ + 1) + j];
                const T* zr = Zs + j * sp;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int l = lane + 32 * c;
                    if (l < n) {
                        const T z = zr[l];
                        acc[0][c] = fma(w0, z, acc[0][c]);
                        acc[1][c] = fma(w1, z, acc[1][c]);
                        acc[2][c] = fma(w2, z, acc[2][c]);
                        acc[3][c] = fma(w3, z, acc[3][c]);
                    }
                }
            }
        }
    }
    // epilogue: accumulators through shared memory so that every store runs down a column
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int l = lane + 32 * c;
            if (l < n) Ss[(warp * 4 + r) * sp + l] = acc[r][c];
        }
    __syncthreads();
    for (int idx = t; idx < kTI * n; idx += kLocThreads) {
        const int i = idx % kTI, l = idx / kTI;
        const int64_t gi = i0 + i;
        if (gi < a.nstate) {
            const T xb = a.XB[(int64_t)l * a.ldb + gi];
            a.XA[(int64_t)l * a.lda + gi] = xb + Ss[i * sp + l];
        }
    }
}

template <typename T>
cudaError_t localized_launch(const LocArgs<T>& a, cudaStream_t s) {
    const size_t smem = loc_smem_bytes<T>(a.n);
    cudaError_t e = cudaFuncSetAttribute(localized_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.nstate + kTI - 1) / kTI;
    localized_update_kernel<T><<<(unsigned)grid, kLocThreads, smem, s>>>(a);
    return cudaGetLastError();
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace
}  // namespace enkf

using namespace enkf;

extern "C" enkf_status enkf_inflate_prep(int64_t nstate, int64_t nobs, int32_t nens, int32_t precision,
                                         int32_t obs_stride, double alpha, void* XB, int64_t ldb, void* dXB,
                                         int64_t ldx, const void* Y, int64_t ldy, void* V, int64_t ldv, void* D,
                                         int64_t ldd, void* stream) {
    if (!XB || !V) return lfail(ENKF_ERR_ARG, "enkf_inflate_prep: NULL XB or V");
    if (Y && !D) return lfail(ENKF_ERR_ARG, "enkf_inflate_prep: Y given without D");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return lfail(ENKF_ERR_ARG, "enkf_inflate_prep: precision must be ENKF_FP64 or ENKF_FP32");
    if (!(alpha >= 0.0) || !isfinite(alpha)) return lfail(ENKF_ERR_ARG, "enkf_inflate_prep: alpha must be >= 0");
    if (nstate < 1 || nobs < 1 || nens < 2 || obs_stride < 1)
        return lfail(ENKF_ERR_SHAPE, "enkf_inflate_prep: need nstate, nobs, obs_stride >= 1 and nens >= 2");
    if ((nobs - 1) * (int64_t)obs_stride >= nstate)
        return lfail(ENKF_ERR_SHAPE, "enkf_inflate_prep: observed rows (nobs - 1) * obs_stride exceed the state");
    if (ldb < nstate || (dXB && ldx < nstate) || ldv < nobs || (Y && (ldy < nobs || ldd < nobs)))
        return lfail(ENKF_ERR_SHAPE, "enkf_inflate_prep: leading dimension smaller than the rows");
    const double scale = 1.0 / sqrt((double)(nens - 1));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((nstate + 255) / 256);
    if (precision == ENKF_FP64)
        inflate_center_observe_kernel<double><<<blocks, 256, 0, s>>>(
            nstate, nobs, nens, obs_stride, alpha, (double*)XB, ldb, (double*)dXB, ldx, (const double*)Y, ldy,
            (double*)V, ldv, (double*)D, ldd, scale);
    else {
        int64_t tiles = (nstate + 31) / 32;
        if (tiles > 152 * 64) tiles = 152 * 64;
        inflate_prep_f32_kernel<<<(unsigned)tiles, kInfWarps * 32, 0, s>>>(
            nstate, nobs, nens, obs_stride, (float)alpha, alpha != 1.0, (float*)XB, ldb, (float*)dXB, ldx,
            (const float*)Y, ldy, (float*)V, ldv, (float*)D, ldd, (float)scale);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lcuda(e, "enkf_inflate_prep: launch");
    return ENKF_OK;
}

extern "C" enkf_status enkf_localized_update(int64_t nstate, int64_t nobs, int32_t nens, int32_t precision,
                                             int32_t obs_stride, double length, double radius, const void* dXB,
                                             int64_t ldx, const void* V, int64_t ldv, const void* Z, int64_t ldz,
                                             const void* XB, int64_t ldb, void* XA, int64_t lda, void* stream) {
    if (!dXB || !V || !Z || !XB || !XA) return lfail(ENKF_ERR_ARG, "enkf_localized_update: NULL array");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return lfail(ENKF_ERR_ARG, "enkf_localized_update: precision must be ENKF_FP64 or ENKF_FP32");
    if (!(length > 0.0)) return lfail(ENKF_ERR_ARG, "enkf_localized_update: length must be > 0 (may be +inf)");
    if (isnan(radius)) return lfail(ENKF_ERR_ARG, "enkf_localized_update: radius is NaN");
    if (nstate < 1 || nobs < 1 || obs_stride < 1 || nens < 2 || nens > kLocMaxN)
        return lfail(ENKF_ERR_SHAPE, "enkf_localized_update: need nstate, nobs, obs_stride >= 1 and 2 <= nens <= %d",
                     kLocMaxN);
    if ((nobs - 1) * (int64_t)obs_stride >= nstate)
        return lfail(ENKF_ERR_SHAPE, "enkf_localized_update: observed rows (nobs - 1) * obs_stride exceed the state");
    if (ldx < nstate || ldb < nstate || lda < nstate || ldv < nobs || ldz < nobs)
        return lfail(ENKF_ERR_SHAPE, "enkf_localized_update: leading dimension smaller than the rows");
    const bool fp64 = precision == ENKF_FP64;
    const size_t w = fp64 ? 8 : 4;
    if (((uintptr_t)dXB | (uintptr_t)V | (uintptr_t)Z | (uintptr_t)XB | (uintptr_t)XA) & (w - 1))
        return lfail(ENKF_ERR_ARG, "enkf_localized_update: pointer not aligned to the element size");
    // X_A may be X_B itself (same pointer and ld: each element is read by the thread that writes it);
    // any other overlap of X_A with an input is rejected
    const size_t xa_bytes = w * ((size_t)lda * (nens - 1) + nstate);
    const bool alias_xb = (XA == XB && lda == ldb);
    if ((!alias_xb && overlaps(XA, xa_bytes, XB, w * ((size_t)ldb * (nens - 1) + nstate))) ||
        overlaps(XA, xa_bytes, dXB, w * ((size_t)ldx * (nens - 1) + nstate)) ||
        overlaps(XA, xa_bytes, V, w * ((size_t)ldv * (nens - 1) + nobs)) ||
        overlaps(XA, xa_bytes, Z, w * ((size_t)ldz * (nens - 1) + nobs)))
        return lfail(ENKF_ERR_ARG, "enkf_localized_update: XA overlaps an input (only XA == XB is allowed)");

    int64_t band = -1;
    if (radius >= 0.0 && radius < (double)nstate) {
        const int64_t rc = (int64_t)ceil(radius);
        if (kTI + 2 * rc < nstate) band = rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (fp64) {
        LocArgs<double> a{nstate, nobs, nens, obs_stride, 1.0 / length, radius, band, 1.0 / sqrt((double)(nens - 1)),
                          (const double*)dXB, ldx, (const double*)V, ldv, (const double*)Z, ldz,
                          (const double*)XB, ldb, (double*)XA, lda};
        e = localized_launch(a, s);
    } else {
        LocArgs<float> a{nstate, nobs, nens, obs_stride, 1.0 / length, radius, band, 1.0 / sqrt((double)(nens - 1)),
                         (const float*)dXB, ldx, (const float*)V, ldv, (const float*)Z, ldz,
                         (const float*)XB, ldb, (float*)XA, lda};
        e = localized_launch(a, s);
    }
    if (e != cudaSuccess) return lcuda(e, "enkf_localized_update: launch");
    return ENKF_OK;
}
