// Internal launcher interfaces between the translation units of libenkf_ism.
// Host code only; no torch types, no exceptions.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "common.cuh"

namespace enkf {

// Plain level-streaming solve (Step 1 + Step 2 of the iterative Sherman-Morrison
// formula) for one problem.
struct LevelArgs {
    int64_t nobs;
    int32_t nens;
    const void* r;
    const void* V; int64_t ldv;
    const void* D; int64_t ldd;
    void* U; int64_t ldu;          // workspace, nobs x nens
    void* Z; int64_t ldz;          // output, nobs x nens
    double* part;                  // [grid][2*nens] per-CTA partial dots
    double* coefg;                 // [2*nens] reduced coefficients of the current level
    double* C;                     // [nens][nens] Z coefficients c_{k,i} = v_k^T Z^(k-1)[:,i]
    double* gamma;                 // [nens]
    Control* ctl;
    int32_t rows_per_blk;          // rows owned by one CTA (multiple of the vector width)
    int32_t rows_chunk;            // rows staged in shared memory at a time
    int32_t check;                 // run the numeric checks
    int32_t test_skip_arrival;     // test-only: CTA 0 leaves before its first arrival
    uint64_t timeout_ns;
};

// Whole analysis of a small problem in one CTA (small.cu): V, U and Z resident in shared
// memory.  XB/dXB/XA, Z and M are optional (NULL).
struct SmallArgs {
    int32_t nobs, nens;
    int64_t nstate;
    const void* r;
    const void* V; int64_t ldv;
    const void* D; int64_t ldd;
    const void* dXB; int64_t ldx;
    const void* XB; int64_t ldb;
    void* XA; int64_t lda;
    void* Z; int64_t ldz;
    void* M;
    double* gamma;                 // [nens]
    Control* ctl;
    int32_t check;
};
bool small_fits(bool fp64, int64_t nobs, int32_t nens);
cudaError_t small_launch(bool fp64, const SmallArgs& a, cudaStream_t s);

struct LevelLaunch {
    int grid;
    int threads;
    size_t smem;
    int rows_per_blk;
    int rows_chunk;
    int vec;
};

// Chooses the launch shape for (nobs, nens) on the current device.
cudaError_t level_plan(bool fp64, int64_t nobs, int32_t nens, LevelLaunch* out);
cudaError_t level_launch(bool fp64, const LevelLaunch& L, LevelArgs a, cudaStream_t s);

// Panel form (FP32 CUDA cores) of the solve for one problem.
struct PanelArgs {
    int64_t nobs;
    int32_t nens;
    const void* r;
    const void* V; int64_t ldv;
    const void* D; int64_t ldd;
    void* U; int64_t ldu;
    void* Z; int64_t ldz;
    double* part;                  // [grid][part_stride] per-CTA partial dots of the next panel
    int64_t part_stride;
    double* coefg;                 // [b * 2N] reduced dots of the current panel
    double* C;                     // [nens][nens] per-level Z coefficients
    double* gamma;                 // [nens]
    Control* ctl;
    int32_t rows_per_blk;
    int32_t panel_b;
    int32_t check;
    int32_t vec_ok;                // 16-byte aligned columns (U, Z, V) and row blocks
    int32_t refine;                // 1: stored-factor recurrence on the columns in Z (R^-1 times a residual)
    const double* Qg;              // [nens][nens] Gram V^T U of the final U columns (refinement)
    uint64_t timeout_ns;
    // tensor-core modes: 16-bit operand pieces prepared once in the workspace
    unsigned short* vp;            // [pieces][nens][ldp]   pieces of V (written by the Step-1 sweep)
    unsigned short* up;            // [2][pieces][kPB][ldp] pieces of each panel's U_P (two buffers)
    int64_t ldp;                   // row pitch of vp / up (multiple of 8, >= nobs + 63)
};

struct PanelLaunch {
    int grid;
    int threads;
    size_t smem;
    int rows_per_blk;
    int b;
    int prec;                      // 0 FP32 CUDA cores; tensor cores: 1 BF16 x2 pieces, 2 FP16, 3 BF16 x3 pieces
    int64_t part_stride;
};

int panel_max_b();
int panel_pieces(int prec);   // 16-bit operand pieces of the tensor-core variants (0: FP32 cores)
cudaError_t panel_plan(int64_t nobs, int32_t nens, int32_t b, int32_t prec, PanelLaunch* out);
cudaError_t panel_launch(const PanelLaunch& L, PanelArgs a, cudaStream_t s);

// Panel solve with the trailing update and the dots on tcgen05 tensor cores (three BF16
// pieces per value, b = 32 levels per panel; ism_panel_tc05.cu), preceded by a Step-1
// pass.  Workspace: tc5_vpc_bytes (V pieces) and tc5_upc_bytes (two panels' U_P pieces).
struct Tc5Launch {
    int grid, ntiles, tiles_per_blk;
    size_t smem;
    int64_t part_stride;
};
size_t tc5_vpc_bytes(int64_t nobs, int32_t nens);
size_t tc5_upc_bytes(int64_t nobs);
int tc5_panel_b();
cudaError_t tc5_plan(int64_t nobs, int32_t nens, Tc5Launch* out);
// Uses p.r, V, D, U, Z (and lds), part, coefg, C, gamma, ctl, check, timeout_ns.
// cudaErrorNotSupported when U or Z is not TMA-aligned.
cudaError_t tc5_solve(const Tc5Launch& L, const PanelArgs& p, void* vpc, void* upc, void* ufc, float* wfin,
                      cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// The stored factors of a tc5_solve applied to p.Z (the refinement's correction sweep);
// workspace: ufc tc5_vpc_bytes, wfin tc5_wfin_bytes.
cudaError_t tc5_correct(const Tc5Launch& L, const PanelArgs& p, const void* vpc, const void* ufc,
                        const float* wfin, cudaStream_t s);
size_t tc5_wfin_bytes(int32_t nens);

// Q[k][m] = sum_j A[j,k] B[j,m] for k < m (strict upper triangle), split over rows,
// partials in double; then Q = sum of the partials in a fixed order.
// FP32 operands run on tcgen05 (gram_tc05) when both arrays are TMA-aligned, else on mma.sync
// (gram_tc); ctl and timeout_ns bound the waits of the tcgen05 kernel.
cudaError_t gram_upper(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B,
                       int64_t ldb, double* Qpart, int32_t nsplit, double* Q, Control* ctl, uint64_t timeout_ns,
                       cudaStream_t s);
int32_t gram_upper_nsplit(int64_t nrows, int32_t n);
// FP32 operands: the partial Grams on tensor cores (three BF16 pieces per operand, six products,
// 32-row stages folded into FP32 and every 512 rows into FP64); Qpart as for gram_upper.  At most
// nsplit row slices are used -- fewer where nsplit slices would not fit one wave of resident CTAs;
// *used receives the count, the number of partial Grams written.
cudaError_t gram_tc(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                    double* Qpart, int32_t nsplit, int full, cudaStream_t s, int32_t* used);
// The same partial Grams on tcgen05: 128 x 128 tiles, one CTA per SM, the same three-piece BF16
// products, each stage of 32 * stage_chunks rows added into a double-FP32 running sum in TMEM
// (the relative error grows with the stage: ~1.8e-7 for one chunk, ~8e-7 for four).  Returns
// cudaErrorNotSupported (nothing launched) when A or B cannot be described by a TMA tensor map
// (16-byte aligned base and stride).
cudaError_t gram_tc05(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                      double* Qpart, int32_t nsplit, int full, int stage_chunks, Control* ctl, uint64_t timeout_ns,
                      cudaStream_t s, int32_t* used);
// Full Gram P[k][m] = sum_j A[j,k] B[j,m] (every k, m), same splitting and fixed-order reduction.
cudaError_t gram_full(bool fp64, int64_t nrows, int32_t n, const void* A, int64_t lda, const void* B, int64_t ldb,
                      double* Qpart, int32_t nsplit, double* Q, Control* ctl, uint64_t timeout_ns, cudaStream_t s);

// Refinement helpers (FP32 storage):
//   gram_comp:       P[k][m] = sum_j A[j,k] B[j,m] (every k, m; row-major) with exact
//                    products and compensated sums folded into FP64 (same splitting and
//                    fixed-order reduction as gram_full; part holds nsplit * n * n doubles);
//   refine_residual: delta = (D - r o Z - V P) / r with P = V^T Z (row-major P[m][i]):
//                    T = D - r o Z by FP32 FMAs, then the tensor-core X_A update with
//                    -P (rounded to FP32 into Mneg, n * n floats; its split images in
//                    msplit, xa_split_bytes(n) bytes) and the divisor r per row;
//   refine_apply:    Z += delta and M = (P + Pd) / sqrt(n - 1) (column-major M[k + i n],
//                    written to M64 and/or M when not NULL).
cudaError_t gram_comp(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                      double* part, int32_t nsplit, double* P, cudaStream_t s);
// The same P on tcgen05 tensor cores from fixed-point BF16 digits (three per value, scaled per
// 32-row chunk and column, exact level sums folded into double FP32; ~2^-32 of sum |a||b|).
// cudaErrorNotSupported when A or B is not TMA-aligned (16-byte base and stride).
cudaError_t gram_exact(int64_t nrows, int32_t n, const float* A, int64_t lda, const float* B, int64_t ldb,
                       double* part, int32_t nsplit, double* P, Control* ctl, uint64_t timeout_ns, cudaStream_t s);
cudaError_t refine_residual(int64_t nobs, int32_t n, const float* r, const float* V, int64_t ldv, const float* D,
                            int64_t ldd, const float* Z, int64_t ldz, const double* P, float* Mneg, void* msplit,
                            float* delta, int64_t ldo, Control* ctl, uint64_t timeout_ns, cudaStream_t s);
// out[0] = ||delta||_F / ||D / r||_F (FP64, fixed-order; part: 1024 doubles of scratch).
cudaError_t refine_resid_norm(int64_t nobs, int32_t n, const float* delta, int64_t ldd, const float* r,
                              const float* D, int64_t ldD, double* part, double* out, cudaStream_t s);
cudaError_t refine_apply(int64_t nobs, int32_t n, float* Z, int64_t ldz, const float* delta, int64_t ldd,
                         const double* P, const double* Pd, double* M64, float* M, cudaStream_t s);

// M = (I - triu(Q,1)) diag(1/gamma) C / sqrt(nens - 1)  (nens x nens, column-major
// output in T: M[m + e*nens]).  C is [level][column].
cudaError_t assemble_M(bool fp64, int32_t nens, const double* Q, const double* C, const double* gamma,
                       void* M, double* M64, cudaStream_t s);

// P = (I - triu(Q,1)) diag(1/gamma) C = V^T Z unscaled, row-major P[k n + i].
cudaError_t assemble_P(int32_t nens, const double* Q, const double* C, const double* gamma, double* P,
                       cudaStream_t s);

// XA = XB + dXB * M  (nstate x nens, K = nens); XA may alias XB.
cudaError_t xa_update(bool fp64, int64_t nstate, int32_t nens, const void* XB, int64_t ldb,
                      const void* dXB, int64_t ldx, const void* M, void* XA, int64_t lda, cudaStream_t s);

// X_A = X_B + dX_B M on tcgen05 tensor cores (split BF16 operands, FP32 accumulators
// in TMEM); msplit: xa_split_bytes(nens) bytes of workspace (the split images of M);
// waits are bounded by timeout_ns and latch kErrTimeout in ctl.
size_t xa_split_bytes(int32_t nens);
// rdiv (nullable): row i of the result is divided by rdiv[i].  pieces: 2 (hi + lo, three
// products) or 3 (hi + mid + lo, six products).
cudaError_t xa_update_tc05(int64_t nstate, int32_t nens, const float* XB, int64_t ldb, const float* dXB, int64_t ldx,
                           const float* M, void* msplit, float* XA, int64_t lda, const float* rdiv, int pieces,
                           Control* ctl, uint64_t timeout_ns, cudaStream_t s);

// Observation-space preparation.
cudaError_t obs_prep(bool fp64, int64_t nstate, int64_t nobs, int32_t nens, int32_t stride, int32_t center,
                     const void* XB, int64_t ldb, void* dXB, int64_t ldx, const void* Y, int64_t ldy,
                     void* V, int64_t ldv, void* D, int64_t ldd, cudaStream_t s);

// Batched analyses: one device descriptor per problem (element offsets).
struct BatchDesc {
    int32_t nobs, nens, b, ldX, ldVr, pad;
    int64_t r, V, D, Z, M;     // offsets into the caller's input (r, V, D) and output (Z, M) base; -1 = none
    int64_t ldv, ldd, ldz;
    int64_t X, Vr;             // offsets of the row-major iterate [U | Z] and of V (row-major) in the workspace
    int64_t Ch, Qw;            // offsets of chat (N x N) and of the Gram Q (N x N) in the workspace
};
size_t batch_smem_bytes();
cudaError_t batch_configure(int* grid);
cudaError_t batch_launch(int grid, const BatchDesc* desc, const int* order, int nprob, const float* in, float* out,
                         float* ws, Control* ctl, int check, int force_b, cudaStream_t s);

// Learned forecast surrogate: views of the packed parameter buffer.
struct SurrogatePacked {
    __nv_bfloat16 *W2, *W3, *WT2, *WT3;   // [o][t][i] and [i][t][o] (tap-flipped)
    float *W1, *b1, *b2, *b3, *W4, *b4;
};
int64_t surrogate_n_params();
size_t surrogate_packed_bytes();
size_t surrogate_forecast_ws(int64_t nstate, int32_t nens);
size_t surrogate_train_ws(int64_t nstate, int32_t nbatch);
cudaError_t surrogate_pack(const float* flat, void* packed, cudaStream_t s);
cudaError_t surrogate_forecast(float* X, int64_t ld, int64_t nstate, int32_t nens, int32_t nsteps, const void* packed,
                               void* ws, cudaStream_t s);
cudaError_t surrogate_train_step(float* master, float* mom, float* vel, int32_t step, float lr, void* packed,
                                 const float* X, const float* target, int64_t nstate, int32_t nbatch, void* ws,
                                 float* loss, float* grad_out, cudaStream_t s);

// Sets the text returned by enkf_last_error() on the calling thread.
void set_last_error(const char* msg);

// Lorenz-96 RK4 forecast, one CTA per member, state in shared memory.
size_t rk4_smem(bool fp64, int64_t nstate);
cudaError_t l96_rk4(bool fp64, void* X, int64_t ld, int64_t nstate, int32_t nens, double F, double dt, int32_t nsteps,
                    cudaStream_t s);

}  // namespace enkf
