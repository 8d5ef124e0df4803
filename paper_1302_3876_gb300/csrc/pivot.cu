// Iterative Sherman-Morrison solve with pivoting (Sec. 3.4, eq. EnKSM:gamma-value),
// C-ABI entry points enkf_ism_solve_pivot and enkf_ism_pivot_workspace (declared in
// include/enkf_ism.h).
//
// Before level k the remaining column with the largest |1 + v_i^T u_i^(k-1)| becomes the
// level's pivot (ties to the lowest index); the interchange of columns in V and U is kept
// as a permutation (perm[k] = the member column used at level k), so the caller's V is
// never written.  Each level is four launches, with no grid-wide wait inside a kernel:
//   choose  (1 CTA)  the candidates' gamma from the per-CTA partial dots, fixed order; argmax;
//   dots    (G CTAs) partial dots of v_p with every Z column and every remaining U column;
//   reduce  (1 CTA)  the dots summed over the CTAs in a fixed order; gamma_k; checks;
//   update  (G CTAs) Z and the remaining U columns minus h_k times their dots, and the
//                    partial dots v_i^T u_i of the remaining columns for the next choice.
// Dots accumulate in FP64 (the products of FP32 operands are exact there).  M = V^T Z /
// sqrt(N - 1) comes from the coefficient identity in pivot order,
//   (V^T Z)[p_k, :] = c_k / gamma_k - sum_{m > k} (v_{p_k}^T u_{p_m}) c_m / gamma_m,
// with c_k the level-k dots of Z and u_{p_m} frozen from level m on; the Gram V^T U is
// formed in FP64 over row slices and reduced in a fixed order.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace enkf {
namespace {

constexpr int kPivMaxN = 256;
constexpr int kPivThreads = 256;
constexpr int kGramTile = 16;
constexpr int kGramRows = 64;
constexpr int kGramSplit = 64;

enkf_status pfail(enkf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

enkf_status pcuda(cudaError_t e, const char* what) {
    return pfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

struct PivLayout {
    int G;                       // CTAs of the row-parallel kernels
    int64_t rows;                // rows per CTA
    int gsplit;                  // row slices of the Gram
    int64_t ldu;
    size_t off_U, off_cpart, off_dpart, off_coef, off_C, off_gam, off_perm, off_done, off_Ppart, off_P, total;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

PivLayout piv_layout(int64_t nobs, int32_t n, size_t w) {
    PivLayout L;
    int64_t g = (nobs + 511) / 512;
    if (g > 304) g = 304;
    if (g < 1) g = 1;
    L.G = (int)g;
    L.rows = (nobs + g - 1) / g;
    int64_t gs = (nobs + 1023) / 1024;
    L.gsplit = (int)(gs < 1 ? 1 : gs > kGramSplit ? kGramSplit : gs);
    L.ldu = (nobs + 31) / 32 * 32;
    const size_t N = (size_t)n;
    size_t o = al256(sizeof(Control));
    L.off_U = o;      o = al256(o + w * (size_t)L.ldu * N);
    L.off_cpart = o;  o = al256(o + sizeof(double) * (size_t)L.G * 2 * N);
    L.off_dpart = o;  o = al256(o + sizeof(double) * (size_t)L.G * N);
    L.off_coef = o;   o = al256(o + sizeof(double) * 2 * N);
    L.off_C = o;      o = al256(o + sizeof(double) * N * N);
    L.off_gam = o;    o = al256(o + sizeof(double) * N);
    L.off_perm = o;   o = al256(o + sizeof(int) * N);
    L.off_done = o;   o = al256(o + sizeof(int) * N);
    L.off_Ppart = o;  o = al256(o + sizeof(double) * (size_t)L.gsplit * N * N);
    L.off_P = o;      o = al256(o + sizeof(double) * N * N);
    L.total = o;
    return L;
}

struct PivArgs {
    int64_t nobs;
    int32_t n;
    int64_t rows;                 // rows per CTA
    const void* r;
    const void* V; int64_t ldv;
    const void* D; int64_t ldd;
    void* U; int64_t ldu;
    void* Z; int64_t ldz;
    double *cpart, *dpart, *coef, *C, *gam, *Ppart, *P;
    int *perm, *done;
    Control* ctl;
};

// Step 1 (eq. SM-step-1): U = R^{-1} V, Z = R^{-1} D, and the partial dots v_i^T u_i.
template <typename T>
__global__ void __launch_bounds__(kPivThreads) piv_step1_kernel(PivArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPivThreads / 32;
    const int64_t j0 = (int64_t)blockIdx.x * a.rows;
    int64_t j1 = j0 + a.rows;
    if (j1 > a.nobs) j1 = a.nobs;
    const T* r = (const T*)a.r;
    const int n = a.n;
    for (int c = warp; c < 2 * n; c += nw) {
        double s = 0.0;
        for (int64_t j = j0 + lane; j < j1; j += 32) {
            const T rj = r[j];
            if (!(rj > T(0)) || !isfinite(rj)) set_status(a.ctl, kErrNumeric);
            if (c < n) {
                const T v = ((const T*)a.V)[(int64_t)c * a.ldv + j];
                const T u = v / rj;
                ((T*)a.U)[(int64_t)c * a.ldu + j] = u;
                s += (double)v * (double)u;
            } else {
                const int e = c - n;
                ((T*)a.Z)[(int64_t)e * a.ldz + j] = ((const T*)a.D)[(int64_t)e * a.ldd + j] / rj;
            }
        }
        s = warp_sum(s);
        if (c < n && lane == 0) a.dpart[(int64_t)blockIdx.x * n + c] = s;
    }
}

// Pivot of level k: argmax over the remaining columns of |1 + sum of the partial dots|.
__global__ void __launch_bounds__(kPivThreads) piv_choose_kernel(PivArgs a, int G, int k) {
    __shared__ double key[kPivThreads];
    __shared__ int idx[kPivThreads];
    const int t = threadIdx.x, n = a.n;
    double kv = -1.0;
    if (t < n && !a.done[t]) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) s += a.dpart[(int64_t)b * n + t];
        const double g = 1.0 + s;
        kv = isnan(g) ? INFINITY : fabs(g);
    }
    key[t] = kv;
    idx[t] = t;
    __syncthreads();
    for (int off = kPivThreads / 2; off > 0; off >>= 1) {
        if (t < off) {
            const double k2 = key[t + off];
            const int i2 = idx[t + off];
            if (k2 > key[t] || (k2 == key[t] && i2 < idx[t])) {
                key[t] = k2;
                idx[t] = i2;
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        const int p = idx[0];
        a.perm[k] = p;
        a.done[p] = 1;
    }
}

// Partial dots of v_p with every Z column (0..n-1) and every remaining U column and u_p (n..2n-1).
template <typename T>
__global__ void __launch_bounds__(kPivThreads) piv_dots_kernel(PivArgs a, int k) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPivThreads / 32;
    const int n = a.n, p = a.perm[k];
    const int64_t j0 = (int64_t)blockIdx.x * a.rows;
    int64_t j1 = j0 + a.rows;
    if (j1 > a.nobs) j1 = a.nobs;
    const T* vp = (const T*)a.V + (int64_t)p * a.ldv;
    for (int c = warp; c < 2 * n; c += nw) {
        const bool active = c < n || c - n == p || !a.done[c - n];
        double s = 0.0;
        if (active) {
            const T* x = c < n ? (const T*)a.Z + (int64_t)c * a.ldz : (const T*)a.U + (int64_t)(c - n) * a.ldu;
            for (int64_t j = j0 + lane; j < j1; j += 32) s += (double)vp[j] * (double)x[j];
        }
        s = warp_sum(s);
        if (lane == 0) a.cpart[(int64_t)blockIdx.x * 2 * n + c] = s;
    }
}

// Dots summed over the CTAs in CTA order; gamma_k = 1 + v_p^T u_p; the Z coefficients of the level.
__global__ void __launch_bounds__(kPivThreads) piv_reduce_kernel(PivArgs a, int G, int k, int check) {
    const int n = a.n, p = a.perm[k];
    for (int c = threadIdx.x; c < 2 * n; c += kPivThreads) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) s += a.cpart[(int64_t)b * 2 * n + c];
        a.coef[c] = s;
        if (c < n) a.C[(int64_t)k * n + c] = s;
        if (check && !isfinite(s)) set_status(a.ctl, kErrNumeric);
        if (c == n + p) {
            const double g = 1.0 + s;
            a.gam[k] = g;
            if (check && !(g >= 1.0 - 64.0 * 2.220446049250313e-16 * (1.0 + fabs(s)))) set_status(a.ctl, kErrNumeric);
        }
    }
}

// Level k update: h = u_p / gamma_k; Z -= h c_Z; remaining u_i -= h c_i; then partial v_i^T u_i.
template <typename T>
__global__ void __launch_bounds__(kPivThreads) piv_update_kernel(PivArgs a, int k) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPivThreads / 32;
    const int n = a.n, p = a.perm[k];
    const int64_t j0 = (int64_t)blockIdx.x * a.rows;
    int64_t j1 = j0 + a.rows;
    if (j1 > a.nobs) j1 = a.nobs;
    const T inv_g = (T)(1.0 / a.gam[k]);
    const T* up = (const T*)a.U + (int64_t)p * a.ldu;
    for (int c = warp; c < 2 * n; c += nw) {
        const bool zcol = c < n;
        const int i = c - n;
        if (!zcol && a.done[i]) {
            if (lane == 0) a.dpart[(int64_t)blockIdx.x * n + i] = 0.0;
            continue;
        }
        const T cf = (T)a.coef[c];
        T* x = zcol ? (T*)a.Z + (int64_t)c * a.ldz : (T*)a.U + (int64_t)i * a.ldu;
        const T* vi = zcol ? nullptr : (const T*)a.V + (int64_t)i * a.ldv;
        double s = 0.0;
        for (int64_t j = j0 + lane; j < j1; j += 32) {
            const T h = up[j] * inv_g;
            const T xn = x[j] - h * cf;
            x[j] = xn;
            if (!zcol) s += (double)vi[j] * (double)xn;
        }
        if (!zcol) {
            s = warp_sum(s);
            if (lane == 0) a.dpart[(int64_t)blockIdx.x * n + i] = s;
        }
    }
}

// Partial Grams Ppart[slice][a][b] = sum over the slice's rows of V[j,a] U[j,b] (FP64 sums).
template <typename T>
__global__ void __launch_bounds__(kGramTile * kGramTile) piv_gram_kernel(PivArgs a, int gsplit) {
    __shared__ double Vs[kGramRows][kGramTile + 1], Us[kGramRows][kGramTile + 1];
    const int n = a.n, t = threadIdx.x, ta = t / kGramTile, tb = t % kGramTile;
    const int a0 = blockIdx.x * kGramTile, b0 = blockIdx.y * kGramTile, sl = blockIdx.z;
    const int64_t per = (a.nobs + gsplit - 1) / gsplit;
    const int64_t j0 = (int64_t)sl * per;
    int64_t j1 = j0 + per;
    if (j1 > a.nobs) j1 = a.nobs;
    double s = 0.0;
    for (int64_t jb = j0; jb < j1; jb += kGramRows) {
        __syncthreads();
        for (int idx = t; idx < kGramRows * kGramTile; idx += kGramTile * kGramTile) {
            const int jj = idx % kGramRows, cc = idx / kGramRows;
            const int64_t j = jb + jj;
            const bool ok = j < j1;
            Vs[jj][cc] = (ok && a0 + cc < n) ? (double)((const T*)a.V)[(int64_t)(a0 + cc) * a.ldv + j] : 0.0;
            Us[jj][cc] = (ok && b0 + cc < n) ? (double)((const T*)a.U)[(int64_t)(b0 + cc) * a.ldu + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kGramRows; ++jj) s += Vs[jj][ta] * Us[jj][tb];
    }
    if (a0 + ta < n && b0 + tb < n) a.Ppart[((int64_t)sl * n + a0 + ta) * n + b0 + tb] = s;
}

__global__ void piv_gram_reduce_kernel(PivArgs a, int gsplit) {
    const int n = a.n;
    const int64_t nn = (int64_t)n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sl = 0; sl < gsplit; ++sl) s += a.Ppart[sl * nn + q];
        a.P[q] = s;
    }
}

// M[p_k + e n] = (c_{k,e} / gamma_k - sum_{m > k} P[p_k][p_m] c_{m,e} / gamma_m) / sqrt(n - 1); one CTA per e.
template <typename T>
__global__ void __launch_bounds__(kPivThreads) piv_assemble_M_kernel(PivArgs a, T* M, double scale) {
    __shared__ double y[kPivMaxN];
    const int n = a.n, e = blockIdx.x;
    for (int m = threadIdx.x; m < n; m += kPivThreads) y[m] = a.C[(int64_t)m * n + e] / a.gam[m];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += kPivThreads) {
        const int pk = a.perm[k];
        double s = y[k];
        for (int m = k + 1; m < n; ++m) s -= a.P[(int64_t)pk * n + a.perm[m]] * y[m];
        M[(int64_t)e * n + pk] = (T)(s * scale);
    }
}

template <typename T>
cudaError_t piv_run(const PivLayout& L, PivArgs a, T* M, int check, cudaStream_t s) {
    const int n = a.n;
    piv_step1_kernel<T><<<L.G, kPivThreads, 0, s>>>(a);
    for (int k = 0; k < n; ++k) {
        piv_choose_kernel<<<1, kPivThreads, 0, s>>>(a, L.G, k);
        piv_dots_kernel<T><<<L.G, kPivThreads, 0, s>>>(a, k);
        piv_reduce_kernel<<<1, kPivThreads, 0, s>>>(a, L.G, k, check);
        piv_update_kernel<T><<<L.G, kPivThreads, 0, s>>>(a, k);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !M) return e;
    dim3 gg((unsigned)((n + kGramTile - 1) / kGramTile), (unsigned)((n + kGramTile - 1) / kGramTile),
            (unsigned)L.gsplit);
    piv_gram_kernel<T><<<gg, kGramTile * kGramTile, 0, s>>>(a, L.gsplit);
    piv_gram_reduce_kernel<<<64, 256, 0, s>>>(a, L.gsplit);
    piv_assemble_M_kernel<T><<<n, kPivThreads, 0, s>>>(a, M, 1.0 / sqrt((double)(n - 1)));
    return cudaGetLastError();
}

bool spans_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace
}  // namespace enkf

using namespace enkf;

extern "C" enkf_status enkf_ism_pivot_workspace(int64_t nobs, int32_t nens, int32_t precision, size_t* bytes) {
    if (!bytes) return pfail(ENKF_ERR_ARG, "enkf_ism_pivot_workspace: NULL bytes");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return pfail(ENKF_ERR_ARG, "enkf_ism_pivot_workspace: precision must be ENKF_FP64 or ENKF_FP32");
    if (nobs < 1 || nens < 1 || nens > kPivMaxN || nobs > ((int64_t)1 << 40))
        return pfail(ENKF_ERR_SHAPE, "enkf_ism_pivot_workspace: need nobs >= 1 and 1 <= nens <= %d", kPivMaxN);
    *bytes = piv_layout(nobs, nens, precision == ENKF_FP64 ? 8 : 4).total;
    return ENKF_OK;
}

extern "C" enkf_status enkf_ism_solve_pivot(int64_t nobs, int32_t nens, int32_t precision, const void* r,
                                            const void* V, int64_t ldv, const void* D, int64_t ldd, void* Z,
                                            int64_t ldz, void* M, int32_t* perm, double* gamma, void* workspace,
                                            size_t workspace_bytes, void* stream, int32_t* status) {
    if (!r || !V || !D || !Z) return pfail(ENKF_ERR_ARG, "enkf_ism_solve_pivot: NULL r, V, D or Z");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return pfail(ENKF_ERR_ARG, "enkf_ism_solve_pivot: precision must be ENKF_FP64 or ENKF_FP32");
    if (nobs < 1 || nens < 1 || nens > kPivMaxN || nobs > ((int64_t)1 << 40))
        return pfail(ENKF_ERR_SHAPE, "enkf_ism_solve_pivot: need nobs >= 1 and 1 <= nens <= %d", kPivMaxN);
    if (M && nens < 2) return pfail(ENKF_ERR_SHAPE, "enkf_ism_solve_pivot: M needs nens >= 2");
    if (ldv < nobs || ldd < nobs || ldz < nobs)
        return pfail(ENKF_ERR_SHAPE, "enkf_ism_solve_pivot: ldv/ldd/ldz smaller than nobs");
    const bool fp64 = precision == ENKF_FP64;
    const size_t w = fp64 ? 8 : 4;
    if (((uintptr_t)r | (uintptr_t)V | (uintptr_t)D | (uintptr_t)Z | (uintptr_t)M) & (w - 1) ||
        ((uintptr_t)gamma & 7) || ((uintptr_t)perm & 3))
        return pfail(ENKF_ERR_ARG, "enkf_ism_solve_pivot: pointer not aligned to its element size");
    const size_t zbytes = w * ((size_t)ldz * (nens - 1) + nobs);
    if (spans_overlap(Z, zbytes, V, w * ((size_t)ldv * (nens - 1) + nobs)) ||
        spans_overlap(Z, zbytes, D, w * ((size_t)ldd * (nens - 1) + nobs)) ||
        spans_overlap(Z, zbytes, r, w * (size_t)nobs))
        return pfail(ENKF_ERR_ARG, "enkf_ism_solve_pivot: Z overlaps an input");
    const PivLayout L = piv_layout(nobs, nens, w);
    if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255))
        return pfail(ENKF_ERR_WORKSPACE, "enkf_ism_solve_pivot: workspace NULL, not 256-byte aligned or below %zu bytes",
                     L.total);
    char* ws = (char*)workspace;
    PivArgs a;
    a.nobs = nobs;
    a.n = nens;
    a.rows = L.rows;
    a.r = r;
    a.V = V;
    a.ldv = ldv;
    a.D = D;
    a.ldd = ldd;
    a.U = ws + L.off_U;
    a.ldu = L.ldu;
    a.Z = Z;
    a.ldz = ldz;
    a.cpart = (double*)(ws + L.off_cpart);
    a.dpart = (double*)(ws + L.off_dpart);
    a.coef = (double*)(ws + L.off_coef);
    a.C = (double*)(ws + L.off_C);
    a.gam = (double*)(ws + L.off_gam);
    a.Ppart = (double*)(ws + L.off_Ppart);
    a.P = (double*)(ws + L.off_P);
    a.perm = (int*)(ws + L.off_perm);
    a.done = (int*)(ws + L.off_done);
    a.ctl = (Control*)ws;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(Control), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.done, 0, sizeof(int) * (size_t)nens, s);
    if (e != cudaSuccess) return pcuda(e, "enkf_ism_solve_pivot: clearing the workspace");
    e = fp64 ? piv_run<double>(L, a, (double*)M, 1, s) : piv_run<float>(L, a, (float*)M, 1, s);
    if (e != cudaSuccess) return pcuda(e, "enkf_ism_solve_pivot: launch");
    if (perm) e = cudaMemcpyAsync(perm, a.perm, sizeof(int) * (size_t)nens, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && gamma) e = cudaMemcpyAsync(gamma, a.gam, sizeof(double) * (size_t)nens, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return pcuda(e, "enkf_ism_solve_pivot: copying perm / gamma");
    if (status) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return pcuda(e, "enkf_ism_solve_pivot: cudaStreamSynchronize");
        int dst = 0;
        e = cudaMemcpy(&dst, &a.ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return pcuda(e, "enkf_ism_solve_pivot: status read");
        *status = dst;
        if (dst != 0) return pfail((enkf_status)dst, "enkf_ism_solve_pivot: device status %d", dst);
    }
    return ENKF_OK;
}
