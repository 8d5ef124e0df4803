// Row-sharded iterative Sherman-Morrison analysis: the data path of one row block.
//
// The observations (rows of V, D, U, Z) are split into blocks, one per rank.  Step 1
// (eq. SM-step-1) is local to a block.  Level k of Step 2 (eqs. SM-step-2-h/Z/u) needs
// the 2N - k dots of v_k with the columns z_0..z_{N-1}, u_k..u_{N-1} over ALL rows; every
// block forms its partial dots, the caller sums them over the ranks (one all-reduce of
// 2N doubles per level), and every block then applies the level to its own rows with the
// same reduced dots.  The pass that applies level k also forms the block's partial dots
// of level k + 1 (v_{k+1} with the updated columns), so one level is one launch and one
// exchange.  M needs the Gram Q = V^T U of the final U columns (one more all-reduce of
// N x N) and the per-level coefficients, which every rank already holds; X_A is local to
// a block of state rows.
//
// Launch shape: CTAs own contiguous runs of kRows rows; warp w takes the active columns
// w, w + 8, ...; lanes run down a column (coalesced), the block's h_k = u_k / gamma_k and
// v_{k+1} rows staged in shared memory.  Per-CTA partial dots are kept in FP64 and summed
// over the CTAs in a fixed order by a second kernel, so a block's partial is
// deterministic; the cross-rank sum is the caller's collective.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace enkf {
namespace {

constexpr int kRT = 256;      // threads
constexpr int kRows = 1024;   // rows per CTA

template <typename T>
__device__ __forceinline__ T tol_gamma_rows();
template <>
__device__ __forceinline__ float tol_gamma_rows<float>() { return 64.f * 1.1920928955078125e-07f; }
template <>
__device__ __forceinline__ double tol_gamma_rows<double>() { return 64.0 * 2.220446049250313e-16; }

struct RowsArgs {
    int64_t nobs;
    int32_t nens, k;           // k = -1: Step 1 (and the dots of level 0)
    const void* r;
    const void* V;
    int64_t ldv;
    const void* D;
    int64_t ldd;
    void* U;
    int64_t ldu;
    void* Z;
    int64_t ldz;
    const double* coef;        // reduced dots of level k (2N: v_k^T z_i at i, v_k^T u_i at N + i)
    double* C;                 // [N][N] per-level Z coefficients (row k written)
    double* gamma;             // [N]
    double* part;              // [grid][2N] per-CTA partial dots of level k + 1
    Control* ctl;
};

template <typename T>
__global__ void __launch_bounds__(kRT) rows_pass_kernel(RowsArgs a) {
    __shared__ T sh_h[kRows];      // k >= 0: h_k = u_k / gamma_k; k = -1: 1 / r
    __shared__ T sh_v[kRows];      // v_{k+1}
    const int N = a.nens, k = a.k;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const int nr = (int)min((int64_t)kRows, a.nobs - row0);
    const T* V = static_cast<const T*>(a.V);
    T* U = static_cast<T*>(a.U);
    T* Z = static_cast<T*>(a.Z);
    const bool next = k + 1 < N;                // dots of level k + 1 wanted
    T ginv = T(1);
    if (k >= 0) {
        const double g = 1.0 + a.coef[N + k];
        ginv = (T)(1.0 / g);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.gamma[k] = g;
            if (!(g >= 1.0 - (double)tol_gamma_rows<T>() * (1.0 + fabs(g - 1.0))) || !isfinite(g)) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = k + 1;
            }
        }
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < N; i += kRT) a.C[(int64_t)k * N + i] = a.coef[i];
    }
    const T* r = static_cast<const T*>(a.r);
    for (int j = threadIdx.x; j < nr; j += kRT) {
        const int64_t jr = row0 + j;
        if (k < 0) {
            const T rj = r[jr];
            if (!(rj > T(0)) || !isfinite(rj)) {
                set_status(a.ctl, kErrNumeric);
                a.ctl->fail_level = 0;
            }
            sh_h[j] = T(1) / rj;
        } else {
            sh_h[j] = U[(int64_t)k * a.ldu + jr] * ginv;
        }
        sh_v[j] = next ? V[(int64_t)(k + 1) * a.ldv + jr] : T(0);
    }
    // the slots of the columns no longer active (u_0..u_k) hold zeros
    if (next)
        for (int i = threadIdx.x; i <= k; i += kRT) a.part[(int64_t)blockIdx.x * 2 * N + N + i] = 0.0;
    __syncthreads();
    // active columns: z_0..z_{N-1}, then u_{k+1}..u_{N-1}
    const int nu = N - (k + 1);
    const int ncol = N + nu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T* D = static_cast<const T*>(a.D);
    for (int c = warp; c < ncol; c += kRT / 32) {
        const bool zc = c < N;
        const int i = zc ? c : (k + 1) + (c - N);            // column index within Z or U
        T* x = zc ? Z + (int64_t)i * a.ldz + row0 : U + (int64_t)i * a.ldu + row0;
        T cf = T(0);
        const T* src = nullptr;
        if (k >= 0) {
            cf = (T)(zc ? a.coef[i] : a.coef[N + i]);
        } else {
            src = zc ? D + (int64_t)i * a.ldd + row0 : V + (int64_t)i * a.ldv + row0;
        }
        T acc = T(0);
        for (int j = lane; j < nr; j += 32) {
            T v;
            if (k >= 0) {
                v = fma(-sh_h[j], cf, x[j]);
            } else {
                v = src[j] * sh_h[j];
                if (!isfinite(v)) {
                    set_status(a.ctl, kErrNumeric);
                    a.ctl->fail_level = 0;
                }
            }
            x[j] = v;
            acc = fma(sh_v[j], v, acc);
        }
        acc = warp_sum(acc);
        if (next && lane == 0) {
            // slot: v_{k+1}^T z_i at i, v_{k+1}^T u_i at N + i
            const int slot = zc ? i : N + i;
            a.part[(int64_t)blockIdx.x * 2 * N + slot] = (double)acc;
        }
    }
}

// out[s] = sum over CTAs (in CTA order) of part[cta][s], for the slots of level k + 1.
__global__ void rows_reduce_kernel(const double* __restrict__ part, int nblk, int n2, int s0, double* out) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n2) return;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += part[(int64_t)b * n2 + s];
    out[s] = v;
}

}  // namespace

int rows_grid(int64_t nobs) { return (int)((nobs + kRows - 1) / kRows); }

cudaError_t rows_pass(bool fp64, int64_t nobs, int32_t nens, int32_t k, const void* r, const void* V, int64_t ldv,
                      const void* D, int64_t ldd, void* U, int64_t ldu, void* Z, int64_t ldz, const double* coef,
                      double* C, double* gamma, double* cta_part, double* out, Control* ctl, cudaStream_t s) {
    RowsArgs a;
    a.nobs = nobs;
    a.nens = nens;
    a.k = k;
    a.r = r;
    a.V = V;
    a.ldv = ldv;
    a.D = D;
    a.ldd = ldd;
    a.U = U;
    a.ldu = ldu;
    a.Z = Z;
    a.ldz = ldz;
    a.coef = coef;
    a.C = C;
    a.gamma = gamma;
    a.part = cta_part;
    a.ctl = ctl;
    const int grid = rows_grid(nobs);
    if (fp64)
        rows_pass_kernel<double><<<grid, kRT, 0, s>>>(a);
    else
        rows_pass_kernel<float><<<grid, kRT, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || k + 1 >= nens) return e;
    // the partial dots of level k + 1: z columns and u_{k+1..N-1}
    const int n2 = 2 * nens;
    rows_reduce_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(cta_part, grid, n2, 0, out);
    return cudaGetLastError();
}

namespace {

enkf_status wfail(enkf_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

enkf_status wcuda(cudaError_t e, const char* what) {
    return wfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// workspace: [Control][per-CTA partial dots: grid x 2N doubles][Gram partials: nsplit x N x N doubles]
size_t ws_part_off() { return 256; }
size_t ws_qpart_off(int64_t nobs, int32_t nens) {
    return (ws_part_off() + sizeof(double) * (size_t)rows_grid(nobs) * 2 * nens + 255) / 256 * 256;
}
size_t ws_bytes(int64_t nobs, int32_t nens) {
    return ws_qpart_off(nobs, nens) + sizeof(double) * (size_t)gram_upper_nsplit(nobs, nens) * nens * nens;
}

enkf_status check_common(const char* who, int32_t precision, int64_t nobs, int32_t nens) {
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return wfail(ENKF_ERR_ARG, "%s: precision must be ENKF_FP64 or ENKF_FP32", who);
    if (nobs < 1 || nens < 1 || nens > 1024) return wfail(ENKF_ERR_SHAPE, "%s: need nobs >= 1, 1 <= nens <= 1024", who);
    return ENKF_OK;
}

}  // namespace
}  // namespace enkf

using namespace enkf;

extern "C" ENKF_API enkf_status enkf_rows_workspace(int64_t nobs, int32_t nens, size_t* bytes) {
    if (!bytes) return wfail(ENKF_ERR_ARG, "enkf_rows_workspace: NULL bytes");
    if (nobs < 1 || nens < 1 || nens > 1024) return wfail(ENKF_ERR_SHAPE, "enkf_rows_workspace: bad sizes");
    *bytes = ws_bytes(nobs, nens);
    return ENKF_OK;
}

extern "C" ENKF_API enkf_status enkf_rows_level(int32_t precision, int64_t nobs, int32_t nens, int32_t k, const void* r,
                                       const void* V, int64_t ldv, const void* D, int64_t ldd, void* U, int64_t ldu,
                                       void* Z, int64_t ldz, const double* coef, double* C, double* gamma,
                                       double* part, void* workspace, size_t workspace_bytes, void* stream) {
    const char* who = "enkf_rows_level";
    enkf_status st = check_common(who, precision, nobs, nens);
    if (st != ENKF_OK) return st;
    if (k < -1 || k >= nens) return wfail(ENKF_ERR_ARG, "%s: k = %d out of [-1, %d)", who, k, nens);
    if (!V || !U || !Z || !workspace || (k + 1 < nens && !part))
        return wfail(ENKF_ERR_ARG, "%s: NULL V, U, Z, part or workspace", who);
    if (k < 0 && (!r || !D)) return wfail(ENKF_ERR_ARG, "%s: Step 1 (k = -1) needs r and D", who);
    if (k >= 0 && (!coef || !C || !gamma)) return wfail(ENKF_ERR_ARG, "%s: k >= 0 needs coef, C and gamma", who);
    if (ldv < nobs || ldu < nobs || ldz < nobs || (k < 0 && ldd < nobs))
        return wfail(ENKF_ERR_SHAPE, "%s: leading dimension smaller than nobs", who);
    if (workspace_bytes < ws_bytes(nobs, nens)) return wfail(ENKF_ERR_WORKSPACE, "%s: workspace too small", who);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    Control* ctl = reinterpret_cast<Control*>(ws);
    double* cta_part = reinterpret_cast<double*>(ws + ws_part_off());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k < 0) {
        cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Control), s);
        if (e != cudaSuccess) return wcuda(e, "enkf_rows_level: control reset");
    }
    cudaError_t e = rows_pass(precision == ENKF_FP64, nobs, nens, k, r, V, ldv, D, ldd, U, ldu, Z, ldz, coef, C,
                              gamma, cta_part, part, ctl, s);
    return e == cudaSuccess ? ENKF_OK : wcuda(e, "enkf_rows_level: launch");
}

extern "C" ENKF_API enkf_status enkf_rows_gram(int32_t precision, int64_t nobs, int32_t nens, const void* V, int64_t ldv,
                                      const void* U, int64_t ldu, double* Q, void* workspace, size_t workspace_bytes,
                                      void* stream) {
    const char* who = "enkf_rows_gram";
    enkf_status st = check_common(who, precision, nobs, nens);
    if (st != ENKF_OK) return st;
    if (!V || !U || !Q || !workspace) return wfail(ENKF_ERR_ARG, "%s: NULL argument", who);
    if (ldv < nobs || ldu < nobs) return wfail(ENKF_ERR_SHAPE, "%s: leading dimension smaller than nobs", who);
    if (workspace_bytes < ws_bytes(nobs, nens)) return wfail(ENKF_ERR_WORKSPACE, "%s: workspace too small", who);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    Control* ctl = reinterpret_cast<Control*>(ws);
    double* qpart = reinterpret_cast<double*>(ws + ws_qpart_off(nobs, nens));
    cudaError_t e = gram_upper(precision == ENKF_FP64, nobs, nens, V, ldv, U, ldu, qpart,
                               gram_upper_nsplit(nobs, nens), Q, ctl, 2000000000ull, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ENKF_OK : wcuda(e, "enkf_rows_gram: launch");
}

extern "C" ENKF_API enkf_status enkf_rows_assemble(int32_t precision, int32_t nens, const double* Q, const double* C,
                                          const double* gamma, void* M, void* stream) {
    const char* who = "enkf_rows_assemble";
    enkf_status st = check_common(who, precision, 1, nens);
    if (st != ENKF_OK) return st;
    if (nens < 2) return wfail(ENKF_ERR_SHAPE, "%s: M needs nens >= 2", who);
    if (!Q || !C || !gamma || !M) return wfail(ENKF_ERR_ARG, "%s: NULL argument", who);
    cudaError_t e = assemble_M(precision == ENKF_FP64, nens, Q, C, gamma, M, nullptr, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ENKF_OK : wcuda(e, "enkf_rows_assemble: launch");
}

extern "C" ENKF_API enkf_status enkf_rows_xa(int32_t precision, int64_t nstate, int32_t nens, const void* XB, int64_t ldb,
                                    const void* dXB, int64_t ldx, const void* M, void* XA, int64_t lda, void* stream) {
    const char* who = "enkf_rows_xa";
    enkf_status st = check_common(who, precision, 1, nens);
    if (st != ENKF_OK) return st;
    if (nstate < 1) return wfail(ENKF_ERR_SHAPE, "%s: nstate < 1", who);
    if (!XB || !dXB || !M || !XA) return wfail(ENKF_ERR_ARG, "%s: NULL argument", who);
    if (ldb < nstate || ldx < nstate || lda < nstate) return wfail(ENKF_ERR_SHAPE, "%s: leading dimension", who);
    cudaError_t e = xa_update(precision == ENKF_FP64, nstate, nens, XB, ldb, dXB, ldx, M, XA, lda,
                              static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ENKF_OK : wcuda(e, "enkf_rows_xa: launch");
}

extern "C" ENKF_API enkf_status enkf_rows_status(void* workspace, void* stream, int32_t* status) {
    if (!workspace || !status) return wfail(ENKF_ERR_ARG, "enkf_rows_status: NULL argument");
    Control h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return wcuda(e, "enkf_rows_status: copy");
    *status = h.status;
    return ENKF_OK;
}
