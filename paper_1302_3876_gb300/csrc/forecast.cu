// Forecast step of the EnKF cycle (Sec. 2, eq. forecast-step) for the Lorenz-96
// model of Sec. 4.2 (eq. eqn:Lorenz96):
//     dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F,   periodic indices,
// integrated with the classical fourth-order Runge-Kutta scheme.
//
// One CTA per ensemble member: the member's state lives in shared memory for all
// nsteps steps (one HBM read and one write per launch).  Stage inputs are double
// buffered so each stage needs one barrier.  Every operation is an explicitly
// rounded IEEE operation (no FMA contraction), in the order
//     k = ((x_{i+1} - x_{i-2}) x_{i-1} - x_i) + F
//     y = x + (dt/2) k            (stages 1, 2),   y = x + dt k  (stage 3)
//     x = x + (dt/6) (((k1 + 2 k2) + 2 k3) + k4)
// so the result is reproducible bit for bit by a plain sequential evaluation.
#include "internal.h"

namespace enkf {
namespace {

template <typename T>
struct RN;
template <>
struct RN<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct RN<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

template <typename T>
__device__ __forceinline__ T l96(const T* y, int i, int n, T F) {
    const int ip1 = (i + 1 == n) ? 0 : i + 1;
    const int im1 = (i == 0) ? n - 1 : i - 1;
    const int im2 = (i >= 2) ? i - 2 : i - 2 + n;
    using R = RN<T>;
    return R::add(R::sub(R::mul(R::sub(y[ip1], y[im2]), y[im1]), y[i]), F);
}

template <typename T>
__global__ void l96_rk4_kernel(T* X, int64_t ld, int n, T F, T half_dt, T dt, T sixth_dt, T two, int nsteps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* x = reinterpret_cast<T*>(smem_raw);
    T* ya = x + n;
    T* yb = ya + n;
    T* acc = yb + n;
    using R = RN<T>;
    T* col = X + (int64_t)blockIdx.x * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = col[i];
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {        // stage 1: x -> ya
            const T k = l96(x, i, n, F);
            acc[i] = k;
            ya[i] = R::add(x[i], R::mul(half_dt, k));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {        // stage 2: ya -> yb
            const T k = l96(ya, i, n, F);
            acc[i] = R::add(acc[i], R::mul(two, k));
            yb[i] = R::add(x[i], R::mul(half_dt, k));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {        // stage 3: yb -> ya
            const T k = l96(yb, i, n, F);
            acc[i] = R::add(acc[i], R::mul(two, k));
            ya[i] = R::add(x[i], R::mul(dt, k));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {        // stage 4: ya -> x
            const T k = l96(ya, i, n, F);
            x[i] = R::add(x[i], R::mul(sixth_dt, R::add(acc[i], k)));
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = x[i];
}

}  // namespace

size_t rk4_smem(bool fp64, int64_t nstate) { return (fp64 ? 8 : 4) * 4 * (size_t)nstate; }

cudaError_t l96_rk4(bool fp64, void* X, int64_t ld, int64_t nstate, int32_t nens, double F, double dt, int32_t nsteps,
                    cudaStream_t s) {
    const size_t smem = rk4_smem(fp64, nstate);
    int threads = (int)((nstate + 31) / 32 * 32);
    if (threads > 256) threads = 256;
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(l96_rk4_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        l96_rk4_kernel<double><<<nens, threads, smem, s>>>((double*)X, ld, (int)nstate, F, 0.5 * dt, dt, dt / 6.0, 2.0,
                                                           nsteps);
    } else {
        e = cudaFuncSetAttribute(l96_rk4_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        l96_rk4_kernel<float><<<nens, threads, smem, s>>>((float*)X, ld, (int)nstate, (float)F, (float)(0.5 * dt),
                                                          (float)dt, (float)(dt / 6.0), 2.0f, nsteps);
    }
    return cudaGetLastError();
}

}  // namespace enkf
