// Plain level-streaming iterative Sherman-Morrison solve (Sec. 3.1 of Nino-Ruiz,
// Sandu and Anderson): Step 1 (eq. SM-step-1) and every level of Step 2
// (eqs. SM-step-2-h, SM-step-2-Z, SM-step-2-u) in ONE persistent cooperative
// launch.
//
// Layout: each CTA owns a fixed block of observation rows of U and Z for the
// whole solve, so a CTA only ever reads and writes its own rows.  Level k is one
// fused pass over the active columns (all of Z, and u_i for i > k):
//     x <- x - h_k c_x                       (update with the level-k dots)
//     partial += v_{k+1}[rows] . x_new        (this CTA's share of the level-(k+1) dots)
// The level-(k+1) dots (including gamma_{k+1} - 1 = v_{k+1}^T u_{k+1}^(k)) are then
// reduced across CTAs in a fixed order (deterministic): barrier, each CTA sums a
// slice of the columns over all CTAs, barrier, every CTA reads the reduced vector.
// h_k = u_k / gamma_k and v_{k+1} are staged in shared memory per row chunk.
// Loads and stores are 16-byte vectors, one warp per column, 32 lanes over rows.
//
// The Z coefficients c_{k,i} = v_k^T Z^(k-1)[:, i] and gamma_k are kept (FP64)
// so that V^T Z can be assembled without the cancellation of a direct product.
#include <math.h>

#include "internal.h"

namespace enkf {
namespace {

constexpr int kThreads = 512;

template <typename T, int N>
struct alignas(sizeof(T) * N) Pack {
    T v[N];
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__device__ __forceinline__ double gamma_tol();
template <>
__device__ __forceinline__ double gamma_tol<float>() { return 64.0 * 1.1920928955078125e-07; }
template <>
__device__ __forceinline__ double gamma_tol<double>() { return 64.0 * 2.220446049250313e-16; }

// Step 1 for one column slice: dst = src / r, and returns this lane's share of w . dst.
template <typename T, int VEC>
__device__ __forceinline__ T stream_step1(const T* __restrict__ src, T* __restrict__ dst,
                                          const T* __restrict__ r, const T* __restrict__ w, int n, int lane) {
    using P = Pack<T, VEC>;
    T acc = T(0);
    const int nv = n / VEC;
    const P* sp = reinterpret_cast<const P*>(src);
    P* dp = reinterpret_cast<P*>(dst);
    const P* rp = reinterpret_cast<const P*>(r);
    const P* wp = reinterpret_cast<const P*>(w);
    int v = lane;
    constexpr int UN = 4;
    for (; v + 32 * (UN - 1) < nv; v += 32 * UN) {
        P x[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) x[u] = sp[v + 32 * u];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const P rv = rp[v + 32 * u], wv = wp[v + 32 * u];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                x[u].v[e] = x[u].v[e] / rv.v[e];
                acc = fma_t(wv.v[e], x[u].v[e], acc);
            }
            dp[v + 32 * u] = x[u];
        }
    }
    for (; v < nv; v += 32) {
        P x = sp[v];
        const P rv = rp[v], wv = wp[v];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            x.v[e] = x.v[e] / rv.v[e];
            acc = fma_t(wv.v[e], x.v[e], acc);
        }
        dp[v] = x;
    }
    for (int j = nv * VEC + lane; j < n; j += 32) {
        T x = src[j] / r[j];
        acc = fma_t(w[j], x, acc);
        dst[j] = x;
    }
    return acc;
}

// One level for one column slice: x <- x - h * cf, returns this lane's share of
// w . x_new (w = v_{k+1}) when DOT.
template <typename T, int VEC, bool DOT>
__device__ __forceinline__ T stream_level(T* __restrict__ x, const T* __restrict__ h, const T* __restrict__ w,
                                          T cf, int n, int lane) {
    using P = Pack<T, VEC>;
    T acc = T(0);
    const int nv = n / VEC;
    P* xp = reinterpret_cast<P*>(x);
    const P* hp = reinterpret_cast<const P*>(h);
    const P* wp = reinterpret_cast<const P*>(w);
    const T ncf = -cf;
    int v = lane;
    constexpr int UN = 4;
    for (; v + 32 * (UN - 1) < nv; v += 32 * UN) {
        P xv[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) xv[u] = xp[v + 32 * u];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const P hv = hp[v + 32 * u];
#pragma unroll
            for (int e = 0; e < VEC; ++e) xv[u].v[e] = fma_t(hv.v[e], ncf, xv[u].v[e]);
            if (DOT) {
                const P wv = wp[v + 32 * u];
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc = fma_t(wv.v[e], xv[u].v[e], acc);
            }
            xp[v + 32 * u] = xv[u];
        }
    }
    for (; v < nv; v += 32) {
        P xv = xp[v];
        const P hv = hp[v];
#pragma unroll
        for (int e = 0; e < VEC; ++e) xv.v[e] = fma_t(hv.v[e], ncf, xv.v[e]);
        if (DOT) {
            const P wv = wp[v];
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc = fma_t(wv.v[e], xv.v[e], acc);
        }
        xp[v] = xv;
    }
    for (int j = nv * VEC + lane; j < n; j += 32) {
        T xj = fma_t(h[j], ncf, x[j]);
        if (DOT) acc = fma_t(w[j], xj, acc);
        x[j] = xj;
    }
    return acc;
}

struct Smem {
    double* coef;   // [2N] reduced coefficients of the current level
    double* acc;    // [2N] this CTA's partial dots
    double* red;    // [32] block-reduction scratch
    int* flag;      // [4]
};

// Deterministic cross-CTA reduction of the partial dots into s.coef.  Indices
// [N, N + first_u) are not needed at the next level and are skipped.
__device__ bool reduce_coefs(const LevelArgs& a, const Smem& s, int first_u, unsigned& epoch) {
    const int N = a.nens, NN = 2 * N;
    const unsigned nblk = gridDim.x;
    const int tid = threadIdx.x;
    if (nblk == 1) {
        // one CTA: its own sums are the totals (a block barrier orders the global accesses)
        __syncthreads();
        for (int i = tid; i < NN; i += blockDim.x) s.coef[i] = s.acc[i];
        __syncthreads();
        return ld_volatile_s32(&a.ctl->status) == 0;
    }
    for (int i = tid; i < NN; i += blockDim.x) __stcg(&a.part[(int64_t)blockIdx.x * NN + i], s.acc[i]);
    if (!grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, s.flag)) return false;
    // one warp per entry: lane l sums CTAs l, l + 32, ... in order, then a fixed butterfly.
    // (A block-wide FP64 reduction per entry costs microseconds on GB300's narrow FP64 pipe.)
    {
        const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
        int j = 0;
        for (int idx = blockIdx.x; idx < NN; idx += nblk, ++j) {
            if (idx >= N && idx < N + first_u) continue;
            if (j % nw != warp) continue;
            double v = 0.0;
            for (int b = lane; b < (int)nblk; b += 32) v += __ldcg(&a.part[(int64_t)b * NN + idx]);
            v = warp_sum(v);
            if (lane == 0) __stcg(&a.coefg[idx], v);
        }
    }
    if (!grid_barrier(a.ctl, nblk, epoch, a.timeout_ns, s.flag)) return false;
    for (int i = tid; i < NN; i += blockDim.x) s.coef[i] = __ldcg(&a.coefg[i]);
    __syncthreads();
    return true;
}

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) ism_levels_kernel(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.nens, NN = 2 * N;
    const int RC = a.rows_chunk;
    Smem s;
    s.coef = reinterpret_cast<double*>(smem_raw);
    s.acc = s.coef + NN;
    s.red = s.acc + NN;
    s.flag = reinterpret_cast<int*>(s.red + 32);
    T* s_h = reinterpret_cast<T*>(s.flag + 4);
    T* s_w = s_h + RC;
    T* s_r = s_w + RC;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_blk;
    const int64_t r1 = min(r0 + (int64_t)a.rows_per_blk, a.nobs);
    const int64_t nrows = r1 > r0 ? r1 - r0 : 0;
    const T* __restrict__ V = static_cast<const T*>(a.V);
    const T* __restrict__ D = static_cast<const T*>(a.D);
    const T* __restrict__ rv = static_cast<const T*>(a.r);
    T* __restrict__ U = static_cast<T*>(a.U);
    T* __restrict__ Z = static_cast<T*>(a.Z);
    unsigned epoch = 0;

    if (a.test_skip_arrival && blockIdx.x == 0) return;   // exercises the bounded wait only

    // ---- Step 1: Z^(0) = R^-1 D, U^(0) = R^-1 V, and the CTA's share of the level-1 dots.
    for (int i = tid; i < NN; i += blockDim.x) s.acc[i] = 0.0;
    for (int64_t c0 = 0; c0 < nrows; c0 += RC) {
        const int n = (int)((nrows - c0) < (int64_t)RC ? (nrows - c0) : (int64_t)RC);
        __syncthreads();
        for (int j = tid; j < n; j += blockDim.x) {
            const T rj = rv[r0 + c0 + j];
            if (a.check && !(rj > T(0) && isfinite(rj))) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = 0;
            }
            s_r[j] = rj;
            s_w[j] = V[r0 + c0 + j];
        }
        __syncthreads();
        for (int idx = warp; idx < NN; idx += nwarps) {
            const T* src;
            T* dst;
            if (idx < N) {
                src = D + (int64_t)idx * a.ldd;
                dst = Z + (int64_t)idx * a.ldz;
            } else {
                src = V + (int64_t)(idx - N) * a.ldv;
                dst = U + (int64_t)(idx - N) * a.ldu;
            }
            T acc = stream_step1<T, VEC>(src + r0 + c0, dst + r0 + c0, s_r, s_w, n, lane);
            acc = warp_sum(acc);
            if (lane == 0) s.acc[idx] += (double)acc;
        }
    }
    __syncthreads();
    if (!reduce_coefs(a, s, 0, epoch)) return;

    // ---- Step 2: levels k = 0 .. N-1 (the paper's k = 1 .. Nens).
    for (int k = 0; k < N; ++k) {
        const double gam = 1.0 + s.coef[N + k];
        if (blockIdx.x == 0) {
            for (int i = tid; i < N; i += blockDim.x) a.C[(int64_t)k * N + i] = s.coef[i];
            if (tid == 0) a.gamma[k] = gam;
            if (a.check) {
                bool bad = false;
                for (int i = tid; i < NN; i += blockDim.x)
                    if ((i < N || i >= N + k) && !isfinite(s.coef[i])) bad = true;
                if (tid == 0 && !(gam >= 1.0 - gamma_tol<T>() * (1.0 + fabs(gam - 1.0)))) bad = true;
                if (bad) {
                    set_status(a.ctl, kErrNumeric);
                    a.ctl->fail_level = k + 1;
                }
            }
        }
        const bool last = (k + 1 == N);
        // one FP64 division per level, by one thread (GB300's FP64 pipe is narrow)
        if (tid == 0) s.red[0] = 1.0 / gam;
        for (int i = tid; i < NN; i += blockDim.x) s.acc[i] = 0.0;
        for (int64_t c0 = 0; c0 < nrows; c0 += RC) {
            const int n = (int)((nrows - c0) < (int64_t)RC ? (nrows - c0) : (int64_t)RC);
            __syncthreads();
            const T ginv = (T)s.red[0];
            const T* uk = U + (int64_t)k * a.ldu + r0 + c0;
            const T* vn = V + (int64_t)(k + 1) * a.ldv + r0 + c0;
            for (int j = tid; j < n; j += blockDim.x) {
                s_h[j] = uk[j] * ginv;
                if (!last) s_w[j] = vn[j];
            }
            __syncthreads();
            const int ncols = N + (N - 1 - k);
            for (int ai = warp; ai < ncols; ai += nwarps) {
                int idx;
                T* x;
                if (ai < N) {
                    idx = ai;
                    x = Z + (int64_t)ai * a.ldz;
                } else {
                    const int i = k + 1 + (ai - N);
                    idx = N + i;
                    x = U + (int64_t)i * a.ldu;
                }
                const T cf = (T)s.coef[idx];
                if (last) {
                    stream_level<T, VEC, false>(x + r0 + c0, s_h, s_w, cf, n, lane);
                } else {
                    T acc = stream_level<T, VEC, true>(x + r0 + c0, s_h, s_w, cf, n, lane);
                    acc = warp_sum(acc);
                    if (lane == 0) s.acc[idx] += (double)acc;
                }
            }
        }
        __syncthreads();
        if (last) break;
        if (!reduce_coefs(a, s, k + 1, epoch)) return;
    }
}

template <typename T, int VEC>
size_t level_smem(int nens, int rc) {
    return sizeof(double) * (4 * (size_t)nens + 32) + 16 + 3 * (size_t)rc * sizeof(T);
}

template <typename T, int VEC>
cudaError_t plan_t(int64_t nobs, int32_t nens, LevelLaunch* L) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int rc_cap = sizeof(T) == 4 ? 2048 : 1024;
    size_t smem = level_smem<T, VEC>(nens, rc_cap);
    // the launch may take the vector or the scalar variant: size the cooperative
    // grid for whichever fits fewer CTAs per SM
    int occ = 1 << 30;
    const void* variants[2] = {(const void*)ism_levels_kernel<T, VEC>, (const void*)ism_levels_kernel<T, 1>};
    for (const void* f : variants) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, kThreads, smem);
        if (e != cudaSuccess) return e;
        occ = o < occ ? o : occ;
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    occ = occ > 2 ? 2 : occ;
    int64_t grid = (int64_t)nsm * occ;
    const int64_t min_rows = 64;
    const int64_t by_rows = (nobs + min_rows - 1) / min_rows;
    if (grid > by_rows) grid = by_rows;
    if (grid < 1) grid = 1;
    int64_t rpb = (nobs + grid - 1) / grid;
    rpb = (rpb + VEC - 1) / VEC * VEC;
    grid = (nobs + rpb - 1) / rpb;
    int64_t rc = rpb < rc_cap ? rpb : rc_cap;
    if (rpb > rc_cap) {
        // balance the chunks of one CTA
        int64_t nch = (rpb + rc_cap - 1) / rc_cap;
        rc = (rpb + nch - 1) / nch;
        rc = (rc + VEC - 1) / VEC * VEC;
    }
    L->grid = (int)grid;
    L->threads = kThreads;
    L->rows_per_blk = (int)rpb;
    L->rows_chunk = (int)rc;
    L->smem = level_smem<T, VEC>(nens, (int)rc);
    L->vec = VEC;
    return cudaSuccess;
}

template <typename T, int VEC>
cudaError_t launch_t(const LevelLaunch& L, LevelArgs a, cudaStream_t s) {
    a.rows_per_blk = L.rows_per_blk;
    a.rows_chunk = L.rows_chunk;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)ism_levels_kernel<T, VEC>, dim3(L.grid), dim3(L.threads), args,
                                       L.smem, s);
}

}  // namespace

cudaError_t level_plan(bool fp64, int64_t nobs, int32_t nens, LevelLaunch* out) {
    return fp64 ? plan_t<double, 2>(nobs, nens, out) : plan_t<float, 4>(nobs, nens, out);
}

cudaError_t level_launch(bool fp64, const LevelLaunch& L, LevelArgs a, cudaStream_t s) {
    // The vector path needs 16-byte aligned columns; otherwise use scalar accesses.
    const size_t w = fp64 ? 8 : 4;
    const int vec = fp64 ? 2 : 4;
    auto al = [&](const void* p, int64_t ld) {
        return ((uintptr_t)p % 16 == 0) && (ld % vec == 0);
    };
    const bool vec_ok = al(a.V, a.ldv) && al(a.D, a.ldd) && al(a.U, a.ldu) && al(a.Z, a.ldz) &&
                        ((uintptr_t)a.r % 16 == 0);
    (void)w;
    if (fp64) {
        if (vec_ok) {
            cudaFuncSetAttribute(ism_levels_kernel<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
            return launch_t<double, 2>(L, a, s);
        }
        cudaFuncSetAttribute(ism_levels_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        return launch_t<double, 1>(L, a, s);
    }
    if (vec_ok) {
        cudaFuncSetAttribute(ism_levels_kernel<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        return launch_t<float, 4>(L, a, s);
    }
    cudaFuncSetAttribute(ism_levels_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    return launch_t<float, 1>(L, a, s);
}

}  // namespace enkf
