/*
 * enkf_ism.h -- C ABI of the GB300 (sm_103a) iterative Sherman-Morrison EnKF
 * analysis library (libenkf_ism.so).
 *
 * The method is the one of Nino-Ruiz, Sandu and Anderson, "An Efficient
 * Implementation of the Ensemble Kalman Filter Based on an Iterative
 * Sherman-Morrison Formula" (Statistics and Computing, 2014):
 *
 *   D   = Y - H X_B                                    (Sec. 3, eq. EnKSM:system-rhs)
 *   V   = H S,  S = (X_B - xbar 1^T) / sqrt(Nens - 1)  (eqs. EnSM:Matrix-member-deviations,
 *                                                        EnKSM:member-observations)
 *   Z   = S_*(R, V, D) = (R + V V^T)^{-1} D            (Sec. 3.1, Steps 1 and 2, eqs.
 *                                                        SM-step-1, SM-step-2-h/Z/u)
 *   X_A = X_B + S V^T Z = X_B + dX_B M,
 *   M   = V^T Z / sqrt(Nens - 1)                       (Sec. 3.1, SMEnKF analysis)
 *
 * with R = diag(r) (r holds observation-error VARIANCES, r_j > 0).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major, one ensemble member per column, with a leading
 *   dimension ld >= rows.  Only rows [0, rows) of each column are read or
 *   written; padding rows are never touched.
 * - Every array argument is a DEVICE pointer owned by the caller (for example
 *   a torch tensor's data_ptr()).  The library never allocates or frees device
 *   memory on the analysis path: scratch space is the caller's workspace, sized
 *   by enkf_ism_plan().  The one exception is enkf_ism_plan() itself, which
 *   allocates nothing on the device either (it only queries device properties).
 * - Element type follows the plan's mode: ENKF_FP64 means every floating-point
 *   buffer is double; every other mode uses float storage.  Entry points that take
 *   no plan take a precision argument (ENKF_FP64 or ENKF_FP32) instead.
 * - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 *   void*; NULL is the legacy default stream).  Device-side checks (r_j <= 0,
 *   non-finite values, gamma_k < 1 - tol, an expired bounded wait) latch a status
 *   word in the workspace; it is returned by the next call on the same plan, or
 *   immediately when a non-NULL info pointer is given (which synchronises the
 *   stream).
 * - Errors are return codes only: no exit(), no abort(), no device trap.  After
 *   ENKF_ERR_CUDA the detail text is in enkf_last_error().
 * - Pointers passed to one call must not overlap unless stated (X_A may alias
 *   X_B).
 */
#ifndef ENKF_ISM_H
#define ENKF_ISM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ENKF_API __attribute__((visibility("default")))
#else
#define ENKF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ENKF_OK = 0,
    ENKF_ERR_ARG = 1,         /* NULL where a pointer is required, bad enum or flag, bad alignment */
    ENKF_ERR_SHAPE = 2,       /* a size or leading dimension out of range */
    ENKF_ERR_CUDA = 3,        /* a CUDA runtime call failed (see enkf_last_error) */
    ENKF_ERR_NUMERIC = 4,     /* r_j <= 0, a non-finite value, or gamma_k < 1 - tol (Sec. 3.3) */
    ENKF_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    ENKF_ERR_UNSUPPORTED = 6, /* mode / size combination the library does not implement */
    ENKF_ERR_WORKSPACE = 7    /* workspace NULL, too small or not 256-byte aligned */
} enkf_status;

typedef enum {
    ENKF_FP64 = 0,        /* plain level-by-level path, double storage and arithmetic */
    ENKF_FP32 = 1,        /* plain level-by-level path, float storage, double gamma */
    ENKF_PANEL_BF16 = 2,  /* panel form, tensor-core trailing updates and dots with split BF16 operands
                             (x = hi + lo, three products), FP32 storage/accumulation, FP64 denominators */
    ENKF_PANEL_FP16 = 3,  /* panel form, tensor-core trailing updates and dots in one FP16 product,
                             FP32 storage/accumulation, FP64 denominators */
    ENKF_PANEL_FP32 = 4,  /* panel form on FP32 CUDA cores (b levels per pass), FP64 denominators */
    ENKF_PANEL_BF16X3 = 5 /* panel form, tensor-core trailing updates and dots with BF16 operands split
                             in three (x = hi + mid + lo, six products: operands kept to ~2^-25),
                             FP32 storage/accumulation, FP64 denominators */
} enkf_mode;

/* Plan flags. */
#define ENKF_FLAG_REFINE        0x1u  /* panel modes: one step of iterative refinement of Z and M:
                                         the residual R^{-1}(D - r o Z - V P), P = V^T Z taken from
                                         the solve's own per-level coefficients (summed exactly from
                                         the columns for PANEL_FP16), corrected by the solve's stored
                                         panel factors; M = (P + V^T delta) / sqrt(Nens - 1).  One step
                                         contracts the error by about u * gamma_max (u the operand
                                         precision): effective for PANEL_FP32, PANEL_BF16X3 and
                                         PANEL_BF16, not for PANEL_FP16 once gamma_max approaches
                                         1/u = 2^11 */
#define ENKF_FLAG_NO_CHECKS     0x2u  /* skip the device-side gamma / finiteness checks */
#define ENKF_FLAG_TEST_TIMEOUT  0x4u  /* test only: one CTA skips its first grid-barrier arrival,
                                         so the others' bounded wait expires (ENKF_ERR_TIMEOUT) */

typedef struct enkf_ism_plan_s* enkf_ism_plan_t;  /* opaque plan handle, host-owned */

/* Diagnostics filled by enkf_ism_analysis when info != NULL (forces a stream sync). */
typedef struct {
    double gamma_min;      /* min_k gamma_k = 1 + v_k^T u_k^(k-1)  (Theorem 2: > 1) */
    double gamma_max;      /* max_k gamma_k */
    int32_t panel_b;       /* panel width used (0 for the plain path) */
    int32_t grid_ctas;     /* CTAs of the level-streaming launch */
    int32_t status;        /* device status word of this call */
    int32_t reserved;
    double refine_resid;   /* with ENKF_FLAG_REFINE: ||R^-1 (D - (R + V V^T) Z1)||_F / ||R^-1 D||_F of the
                              solve's Z1 before the correction (the scaled residual the refinement
                              applies the stored factors to); 0 without refinement */
} enkf_ism_info;

/*
 * enkf_ism_plan -- validate sizes and choose launch shapes for one problem size.
 * Infrastructure around the method (no passage of the paper defines it): it fixes the
 * launch shapes of the analysis of Sec. 3.1 and the size of the caller's workspace.
 *
 *   out              receives the plan (host object; free with enkf_ism_plan_destroy).
 *   nstate           state dimension (rows of X_B, dX_B, X_A); >= 1.
 *   nobs             number of observations (rows of V, D, Z); >= 1.
 *   nens             ensemble size (columns); 1 <= nens <= 1024.  nens = 1 allows
 *                    the solve only (M and X_A need nens >= 2, since S divides
 *                    by sqrt(Nens - 1)).
 *   mode             an enkf_mode.
 *   panel_b          panel width for the panel modes (0 = default 32; 1 <= panel_b <= 32,
 *                    else ENKF_ERR_ARG); ignored otherwise.  ENKF_PANEL_BF16X3 with b = 32
 *                    runs the tcgen05 panel kernel when U and Z are TMA-aligned.
 *   flags            ENKF_FLAG_* bits.
 *   workspace_bytes  receives the device workspace size enkf_ism_analysis needs.
 *
 * Uses the CUDA device current on the calling thread.  Returns ENKF_ERR_SHAPE
 * for out-of-range sizes, ENKF_ERR_UNSUPPORTED for an unimplemented mode.
 */
ENKF_API enkf_status enkf_ism_plan(enkf_ism_plan_t* out, int64_t nstate, int64_t nobs, int32_t nens,
                          int32_t mode, int32_t panel_b, uint32_t flags, size_t* workspace_bytes);

ENKF_API void enkf_ism_plan_destroy(enkf_ism_plan_t plan);

/*
 * enkf_obs_prep -- observation-space preparation (Sec. 2 eq. ensemble-background-mean,
 * Sec. 3 eqs. EnSM:Matrix-member-deviations, EnKSM:member-observations,
 * EnKSM:system-rhs), with H selecting state rows 0, obs_stride, 2 obs_stride, ...
 *
 *   center = 1: dX_B = X_B - xbar 1^T is computed from X_B (written to dXB).
 *   center = 0: dXB is an input (deviations given); XB may be NULL when Y is NULL.
 *   Always:     V = H dX_B / sqrt(Nens - 1)           (nobs x nens, written to V).
 *   Y != NULL:  D = Y - H X_B                          (nobs x nens, written to D).
 *
 * Requires (nobs - 1) * obs_stride < nstate and nens >= 2.  Sizes come from the plan.
 */
ENKF_API enkf_status enkf_obs_prep(enkf_ism_plan_t plan, int32_t obs_stride, int32_t center,
                          const void* XB, int64_t ldb,
                          void* dXB, int64_t ldx,
                          const void* Y, int64_t ldy,
                          void* V, int64_t ldv,
                          void* D, int64_t ldd,
                          void* stream);

/*
 * enkf_ism_analysis -- one EnKF analysis by the iterative Sherman-Morrison formula.
 *
 *   r     [nobs]         observation-error variances (R = diag(r)), all > 0.
 *   V     nobs x nens    observation-space deviations, ld ldv.
 *   D     nobs x nens    innovations, ld ldd.
 *   dXB   nstate x nens  background deviations, ld ldx; NULL computes Z (and M) only.
 *   XB    nstate x nens  background ensemble, ld ldb (ignored when dXB is NULL).
 *   XA    nstate x nens  analysis ensemble (output), ld lda; may alias XB (then ldb == lda).
 *   Z     nobs x nens    solution of (R + V V^T) Z = D (output, nullable), ld ldz.
 *   M     nens x nens    V^T Z / sqrt(Nens - 1) (output, nullable), column-major, ld nens.
 *   workspace            device scratch of at least the plan's workspace_bytes,
 *                        256-byte aligned; owned by the caller, reused across calls,
 *                        not shared by calls in flight at the same time.
 *   stream               cudaStream_t to run on.
 *   info                 host pointer or NULL; when given, the call synchronises the
 *                        stream and fills it.
 *
 * Every array is read-only except XA, Z, M and the workspace.  Z and M are
 * written only when non-NULL.  Returns ENKF_ERR_NUMERIC / ENKF_ERR_TIMEOUT from
 * the device status word (immediately with info, else at the next call).
 */
ENKF_API enkf_status enkf_ism_analysis(enkf_ism_plan_t plan,
                              const void* r,
                              const void* V, int64_t ldv,
                              const void* D, int64_t ldd,
                              const void* dXB, int64_t ldx,
                              const void* XB, int64_t ldb,
                              void* XA, int64_t lda,
                              void* Z, int64_t ldz,
                              void* M,
                              void* workspace, size_t workspace_bytes,
                              void* stream, enkf_ism_info* info);

/*
 * Batched analyses: many independent problems of uneven size (for example the local
 * analyses of a domain decomposition) solved in ONE persistent launch, replayed from
 * a CUDA graph.  Each problem is the solve Z = (R + V V^T)^{-1} D of Sec. 3.1 plus
 * M = V^T Z / sqrt(Nens - 1) (the ensemble-space factor of the SMEnKF update).
 * FP32 storage with FP64 level denominators (ENKF_FP32 only).
 *
 * A problem is described by element offsets (in floats) into two caller buffers:
 * base_in holds r (nobs), V and D (column-major, ld ldv / ldd); base_out receives
 * Z (column-major, ld ldz; offset -1 to skip) and M (nens x nens column-major;
 * offset -1 to skip).  2 <= nens <= 128 with nens % 4 == 0; nobs >= 1.
 */
typedef struct {
    int64_t nobs;
    int32_t nens;
    int32_t reserved;         /* set to 0 */
    int64_t r, V, D;          /* offsets into base_in */
    int64_t ldv, ldd;
    int64_t Z, ldz;           /* offset into base_out (or -1), leading dimension */
    int64_t M;                /* offset into base_out (or -1) */
} enkf_ism_problem;

typedef struct enkf_ism_batch_plan_s* enkf_ism_batch_plan_t;

/*
 * enkf_ism_batch_plan -- host-side plan of a batch: validates the descriptors,
 * orders the problems by cost (longest first), lays out the workspace and assigns
 * each problem the panel width of its size class (nens x nobs bucket).  Widths come
 * from the autotune cache file named by the environment variable
 * ENKF_AUTOTUNE_CACHE when it holds this GPU's entries, else a default (16).
 */
ENKF_API enkf_status enkf_ism_batch_plan(enkf_ism_batch_plan_t* out, int32_t nprob, const enkf_ism_problem* problems,
                                         int32_t mode, uint32_t flags, size_t* workspace_bytes);
ENKF_API void enkf_ism_batch_plan_destroy(enkf_ism_batch_plan_t plan);

/*
 * enkf_ism_batch_autotune -- times every panel width b in {1, 8, 16, 32} on each size
 * class of this batch (using the caller's data and workspace; synchronises the
 * stream), keeps the fastest per class in the plan, and appends the choices to
 * cache_path (or ENKF_AUTOTUNE_CACHE when cache_path is NULL; no file when both are
 * absent).  widths (host, nullable) receives the 16 per-class choices.
 */
ENKF_API enkf_status enkf_ism_batch_autotune(enkf_ism_batch_plan_t plan, const void* base_in, void* base_out,
                                             void* workspace, size_t workspace_bytes, void* stream,
                                             const char* cache_path, int32_t* widths);

/*
 * enkf_ism_batch -- runs the batch.  The first call with a given (base_in, base_out,
 * workspace) uploads the descriptor table into the workspace and captures a CUDA
 * graph (on an internal stream); later calls with the same pointers replay it on
 * `stream` (new data in place is fine).  status (host, nullable): when given, the
 * call synchronises and stores the device status word.
 */
ENKF_API enkf_status enkf_ism_batch(enkf_ism_batch_plan_t plan, const void* base_in, void* base_out, void* workspace,
                                    size_t workspace_bytes, void* stream, int32_t* status);

/*
 * enkf_forecast -- forecast step X_B(t_next) = M(X_A(t_cur)) (Sec. 2, eq. forecast-step)
 * for the Lorenz-96 model of Sec. 4.2 (eq. eqn:Lorenz96, periodic, forcing F), in place.
 *
 *   X        nstate x nens ensemble (device, ld >= nstate), overwritten.
 *   precision ENKF_FP64 or ENKF_FP32 (element type of X).
 *   method   ENKF_FORECAST_RK4: nsteps classical Runge-Kutta steps of size dt, one CTA
 *            per member with the state in shared memory (nstate <= 6144 in FP64,
 *            12288 in FP32); every operation is an explicitly rounded IEEE operation
 *            in a fixed order, so the result is reproducible bit for bit.
 *            ENKF_FORECAST_SURROGATE: the learned surrogate (see enkf_surrogate_*),
 *            weights = its packed parameter buffer, nsteps surrogate applications.
 *   workspace / workspace_bytes: device scratch (size from enkf_forecast_workspace;
 *            0 bytes for RK4, NULL allowed then).
 * Returns ENKF_ERR_SHAPE for sizes out of range, ENKF_ERR_UNSUPPORTED otherwise.
 */
#define ENKF_FORECAST_RK4       0
#define ENKF_FORECAST_SURROGATE 1
ENKF_API enkf_status enkf_forecast(void* X, int64_t ld, int64_t nstate, int32_t nens, int32_t precision,
                                   double F, double dt, int32_t nsteps, int32_t method, const void* weights,
                                   void* workspace, size_t workspace_bytes, void* stream);
ENKF_API enkf_status enkf_forecast_workspace(int64_t nstate, int32_t nens, int32_t method, size_t* bytes);

/*
 * Learned forecast surrogate (a stand-in for the model propagation of eq. forecast-step):
 *   x_next = x + f(x), f = 4 periodic 1-D convolutions over the state index, channels
 *   1 -> 64 -> 64 -> 64 -> 1, kernel 5, circular padding 2, GELU-tanh between layers,
 *   input normalised as (x - 2.5) / 4.  BF16 weights and activations, FP32 accumulation.
 * The FP32 master parameters are a flat vector in the order W1 (64,1,5), b1 (64),
 * W2 (64,64,5), b2, W3 (64,64,5), b3, W4 (1,64,5), b4 (row-major (out, in, tap)).
 * The packed buffer holds the BF16 / FP32 copies the kernels read (it is the `weights`
 * argument of enkf_forecast with ENKF_FORECAST_SURROGATE).
 *
 * enkf_surrogate_sizes: parameter count, packed-buffer bytes, and the workspace bytes of
 *   one training step on nbatch states of length nstate (any output pointer may be NULL).
 * enkf_surrogate_pack: packed <- master (device pointers).
 * enkf_surrogate_train_step: forward, MSE loss, backward on X -> target (nbatch x nstate,
 *   contiguous FP32); writes the sum of squared errors to sq_err (device float) and the
 *   flat gradient of the mean squared error to grad (device, nullable).  step >= 1 then
 *   applies Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with t = step, learning
 *   rate lr) to master / adam_m / adam_v and repacks; step = 0 computes gradients only.
 */
ENKF_API enkf_status enkf_surrogate_sizes(int64_t nstate, int32_t nbatch, int64_t* n_params, size_t* packed_bytes,
                                          size_t* train_workspace_bytes);
ENKF_API enkf_status enkf_surrogate_pack(const float* master, void* packed, void* stream);
ENKF_API enkf_status enkf_surrogate_train_step(float* master, float* adam_m, float* adam_v, int32_t step, float lr,
                                               void* packed, const float* X, const float* target, int64_t nstate,
                                               int32_t nbatch, void* workspace, size_t workspace_bytes,
                                               float* sq_err, float* grad, void* stream);

/*
 * enkf_inflate_prep -- multiplicative inflation fused into the centering observation
 * prep (Sec. 3.1.1, inflation aspects: x_i <- xbar + alpha (x_i - xbar), which scales
 * the ensemble covariance by alpha^2; then the prep of enkf_obs_prep with center = 1).
 * One pass over X_B:
 *   XB   nstate x nens, ld ldb, in/out: overwritten by the inflated ensemble.
 *   dXB  nstate x nens, ld ldx, output (nullable): deviations of the inflated ensemble
 *        from the mean (the mean is unchanged by inflation).
 *   V    nobs x nens, ld ldv, output: H dX_B / sqrt(Nens - 1), H = rows 0, obs_stride, ...
 *   Y, D nobs x nens (both or neither): D = Y - H X_B of the inflated ensemble.
 * precision ENKF_FP64 or ENKF_FP32 (element type of every array); alpha >= 0 (1 = no
 * inflation); nens >= 2; (nobs - 1) * obs_stride < nstate.  Means in FP64.
 */
ENKF_API enkf_status enkf_inflate_prep(int64_t nstate, int64_t nobs, int32_t nens, int32_t precision,
                                       int32_t obs_stride, double alpha, void* XB, int64_t ldb, void* dXB,
                                       int64_t ldx, const void* Y, int64_t ldy, void* V, int64_t ldv, void* D,
                                       int64_t ldd, void* stream);

/*
 * enkf_localized_update -- partial localization of the analysis increment (Sec. 3.1.2,
 * eq. localized-correction-component and its matrix form):
 *   X_A = X_B + (Delta o (S V^T)) Z,   S = dX_B / sqrt(Nens - 1),
 *   dX_A[i, l] = sum_k S[i, k] sum_j delta_ij V[j, k] Z[j, l],
 * with delta_ij = exp(-d / length) when radius < 0 or d <= radius, else 0, and d the
 * periodic distance between state index i and the observed state index j * obs_stride
 * on the ring of nstate points (the Lorenz-96 weights of Sec. 4.2 are length = nstate,
 * no cut-off).  It replaces the unlocalized X_A = X_B + dX_B M of enkf_ism_analysis:
 * call enkf_ism_analysis for Z (dXB = NULL), then this.
 *   dXB  nstate x nens deviations (ld ldx); V nobs x nens (ld ldv); Z nobs x nens (ld ldz);
 *   XB   nstate x nens (ld ldb); XA nstate x nens output (ld lda).  XA may be XB itself
 *        (same pointer and ld); any other overlap of XA with an input is ENKF_ERR_ARG.
 * precision ENKF_FP64 or ENKF_FP32; 2 <= nens <= 256; length > 0 (+inf gives delta = 1
 * inside the radius); radius < 0 means no cut-off.  Every pair (i, j) within the radius
 * costs 4 Nens flops (FP32 or FP64 CUDA cores); with a radius only the band of each
 * 32-row tile is visited.  Allocates nothing.
 */
ENKF_API enkf_status enkf_localized_update(int64_t nstate, int64_t nobs, int32_t nens, int32_t precision,
                                           int32_t obs_stride, double length, double radius, const void* dXB,
                                           int64_t ldx, const void* V, int64_t ldv, const void* Z, int64_t ldz,
                                           const void* XB, int64_t ldb, void* XA, int64_t lda, void* stream);

/*
 * Block-diagonal R = diag(R_1, ..., R_nblk) (Sec. 3.1: R^{-1} applied block by block in
 * Step 1).  Block b covers observation rows [b bs, min(nobs, (b + 1) bs)) and is stored
 * dense, column-major, FP64, in the leading part of the bs x bs matrix at
 * Rblk + b bs bs (nblk = ceil(nobs / bs) blocks, 1 <= bs <= 32).  With R = L L^T the
 * system (R + V V^T) Z = D is (I + V~ V~^T) Z~ = D~ with V~ = L^{-1} V, D~ = L^{-1} D and
 * Z = L^{-T} Z~; V^T Z = V~^T Z~, so the analysis of the whitened data with r = 1 gives
 * the same gamma_k, M and X_A.  Sequence: enkf_rblock_factor once per R, then per analysis
 * enkf_rblock_whiten (V and D in place), enkf_ism_analysis with r = 1, and
 * enkf_rblock_unwhiten on Z when Z itself is wanted.
 *   enkf_rblock_factor:   Lblk <- lower Cholesky factors (same layout as Rblk, upper parts
 *                         zero).  A block that is not positive definite gets NaN factors,
 *                         which the analysis then reports as ENKF_ERR_NUMERIC.
 *   enkf_rblock_whiten:   V <- L^{-1} V and, when D != NULL, D <- L^{-1} D (nobs x nens).
 *   enkf_rblock_unwhiten: Z <- L^{-T} Z (nobs x ncols).
 * precision ENKF_FP64 or ENKF_FP32 (element type of V, D, Z; the factors are FP64 and the
 * substitutions run in FP64).  All pointers are device pointers.  Allocates nothing.
 */
ENKF_API enkf_status enkf_rblock_factor(int64_t nobs, int32_t bs, const double* Rblk, double* Lblk, void* stream);
ENKF_API enkf_status enkf_rblock_whiten(int64_t nobs, int32_t nens, int32_t precision, int32_t bs,
                                        const double* Lblk, void* V, int64_t ldv, void* D, int64_t ldd,
                                        void* stream);
ENKF_API enkf_status enkf_rblock_unwhiten(int64_t nobs, int32_t ncols, int32_t precision, int32_t bs,
                                          const double* Lblk, void* Z, int64_t ldz, void* stream);

/*
 * enkf_ism_solve_pivot -- the solve Z = (R + V V^T)^{-1} D with the optional pivoting of
 * Sec. 3.4 (eq. EnKSM:gamma-value): before level k the remaining column with the largest
 * |1 + v_i^T u_i^(k-1)| is taken (ties to the lowest index), which the paper offers to
 * reduce round-off.  Z is the same in exact arithmetic; only the level order changes.
 *   r, V, D     as for enkf_ism_analysis (R = diag(r)); V and D are not written.
 *   Z           nobs x nens output (ld ldz), required.
 *   M           nens x nens output (column-major, ld nens, nullable; nens >= 2):
 *               V^T Z / sqrt(Nens - 1) in the caller's member order.
 *   perm        device int32[nens] (nullable): perm[k] = member column used at level k.
 *   gamma       device double[nens] (nullable): gamma_k of level k.
 *   workspace   >= enkf_ism_pivot_workspace bytes, 256-byte aligned, caller-owned.
 *   status      host int or NULL; when given, the call synchronises and stores the
 *               device status word (r_j <= 0, non-finite values, gamma_k < 1 - tol).
 * precision ENKF_FP64 or ENKF_FP32 (dots accumulated in FP64); 1 <= nens <= 256.  Four
 * launches per level (choice, dots, reduction, update) with no grid-wide wait inside a
 * kernel; the reductions run in a fixed order, so results are reproducible.
 */
ENKF_API enkf_status enkf_ism_pivot_workspace(int64_t nobs, int32_t nens, int32_t precision, size_t* bytes);
ENKF_API enkf_status enkf_ism_solve_pivot(int64_t nobs, int32_t nens, int32_t precision, const void* r,
                                          const void* V, int64_t ldv, const void* D, int64_t ldd, void* Z,
                                          int64_t ldz, void* M, int32_t* perm, double* gamma, void* workspace,
                                          size_t workspace_bytes, void* stream, int32_t* status);

/*
 * Kernel-phase timing (tracing aid).  enkf_ism_profile(plan, 1) makes every later
 * enkf_obs_prep / enkf_ism_analysis call on the plan record CUDA events around
 * each of its kernel phases on the caller's stream (up to 4096 phases between
 * reads).  enkf_ism_profile_read synchronises on the last recorded event, adds
 * the elapsed milliseconds of each phase into ms[phase] and the number of
 * launches into count[phase] (arrays of ENKF_PROFILE_PHASES, caller-owned host
 * memory), and clears the record.  Phases: 0 obs prep, 1 level streaming (Step 1
 * and Step 2), 2 Gram V^T U, 3 assembly of M, 4 X_A update, 5 refinement; and two
 * kernels inside those phases, each timed alone: 6 the panel kernel of phase 1
 * (panel modes), 7 the refinement's correction sweep (inside phase 5).
 */
/*
 * enkf_ism_gamma -- the level denominators gamma_k = 1 + v_k^T u_k^(k-1), k = 1..nens
 * (Sec. 3.1, eq. SM-step-2-h; Theorem 2: gamma_k >= 1), of the last enkf_ism_analysis
 * call made with this plan and workspace.  Waits for that call to finish, then copies
 * nens doubles into gamma (caller-owned host memory).  Status codes only; no device
 * memory is touched but the workspace's gamma entries.
 */
ENKF_API enkf_status enkf_ism_gamma(enkf_ism_plan_t plan, const void* workspace, double* gamma);

#define ENKF_PROFILE_PHASES 8
ENKF_API enkf_status enkf_ism_profile(enkf_ism_plan_t plan, int32_t enable);
ENKF_API enkf_status enkf_ism_profile_read(enkf_ism_plan_t plan, double* ms, int32_t* count);

/*
 * enkf_ism_solve_noalloc -- the solve Z = (R + V V^T)^{-1} D of enkf_ism_analysis
 * (the same plain level-streaming kernel) without a caller-provided workspace.  The
 * paper has no counterpart; this entry point exists for callers that cannot
 * allocate device memory, such as a plugin whose host application already owns
 * the GPU's memory through its own pool, or a process whose device-memory budget
 * is fixed at start-up.
 *
 *   nobs, nens    sizes as for enkf_ism_plan (1 <= nens <= 1024).
 *   precision     ENKF_FP64 or ENKF_FP32 (element type of r, V, D, Z).
 *   r, V, D, Z    device pointers as for enkf_ism_analysis; Z (nobs x nens, ld ldz)
 *                 is the output.
 *   stream        cudaStream_t.
 *   status        host int or NULL; when given, the call synchronises the stream and
 *                 stores the device status word (0 = ok) there, and returns that
 *                 status when it is not 0.  With NULL the call stays asynchronous and
 *                 device-side errors (r_j <= 0, non-finite values, gamma_k < 1 - tol,
 *                 an expired bounded wait) are not reported at all: the next call
 *                 clears the control block.  Unlike enkf_ism_analysis, nothing is
 *                 latched for a later call, so a caller that must know whether Z is
 *                 valid passes status.
 *
 * Scratch lives in one static device array of ENKF_NOALLOC_SCRATCH_BYTES (32 MiB)
 * that every GPU loading the library keeps until the process exits; the call
 * allocates nothing.  Sizes whose scratch (U plus per-CTA partials, about
 * w * nobs * nens bytes) exceeds the array are rejected with ENKF_ERR_WORKSPACE.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it: make that first
 * call before any stream capture.  All calls share the array; calls that overlap
 * on the GPU race on it.
 */
#define ENKF_NOALLOC_SCRATCH_BYTES (32u << 20)
ENKF_API enkf_status enkf_ism_solve_noalloc(int64_t nobs, int32_t nens, int32_t precision, const void* r,
                                            const void* V, int64_t ldv, const void* D, int64_t ldd,
                                            void* Z, int64_t ldz, void* stream, int32_t* status);

/*
 * enkf_fma_peak_launch -- launches a CUDA-core multiply-add microbenchmark on
 * `stream`: every thread of ctas_per_sm (1..8) x SM-count CTAs of 256 threads runs
 * 16 independent FMA chains of `iters` steps in registers.  The paper has no
 * counterpart; it measures the FP32 and FP64 CUDA-core peaks against which the
 * ALU-bound kernels are reported.  precision: ENKF_FP32 or ENKF_FP64.  sink: a
 * device word of that type (never written in practice).  *flops (host) receives
 * the exact number of floating-point operations of the launch (2 per FMA); the
 * caller times the launch with CUDA events.
 */
ENKF_API enkf_status enkf_fma_peak_launch(int32_t precision, int32_t iters, int32_t ctas_per_sm, void* sink,
                                          void* stream, double* flops);

/*
 * Row-sharded analysis: the data path of one block of observation rows.  The rows of
 * V, D, U, Z and r are split into blocks (one per rank; every rank holds all N columns
 * of its rows).  Step 1 (Sec. 3.1, eq. SM-step-1) is local to a block; level k of Step 2
 * (eqs. SM-step-2-h/Z/u) needs the dots of v_k with z_0..z_{N-1} and u_k..u_{N-1} summed
 * over every block, which the caller forms by summing the blocks' partial dots (one
 * all-reduce of 2N doubles per level); every block then applies the level to its own
 * rows.  Sequence per rank (arrays: device memory, column-major, caller-owned):
 *   enkf_rows_level(k = -1)            U = R^-1 V, Z = R^-1 D on the block, and the block's
 *                                      partial dots of level 0 into part;
 *   for k = 0 .. N-1:  coef <- sum over ranks of part;
 *     enkf_rows_level(k)               level k on the block with the reduced dots coef
 *                                      (records C[k][:] = coef[0..N), gamma[k] = 1 +
 *                                      coef[N + k]), and the partial dots of level k + 1;
 *   enkf_rows_gram                     the block's partial Q[k][m] = v_k^T u_m (k < m) of the
 *                                      final U columns; Q <- sum over ranks;
 *   enkf_rows_assemble                 M = (I - triu(Q,1)) diag(1/gamma) C / sqrt(N - 1)
 *                                      (= V^T Z / sqrt(N - 1), Sec. 3.1) on every rank;
 *   enkf_rows_xa                       X_A = X_B + dX_B M on the rank's block of state rows.
 * coef and part: 2N doubles, entry i = v_k^T z_i, entry N + i = v_k^T u_i (i >= k; the
 * other entries of part are zero).  C: N x N doubles (row k = level k), gamma: N doubles.
 * precision ENKF_FP64 or ENKF_FP32 (element type of r, V, D, U, Z, X_B, dX_B, X_A, M);
 * dots, C, gamma and Q are FP64.  Each call launches on `stream` and returns; device-side
 * checks (r_j <= 0, non-finite values, gamma_k < 1 - tol) latch a status word in the
 * workspace (cleared by the k = -1 call) that enkf_rows_status reads (synchronising the
 * stream).  Workspace: enkf_rows_workspace(nobs, nens) bytes, one per rank and stream.
 * Errors: ENKF_ERR_ARG (NULL or out-of-range argument), ENKF_ERR_SHAPE (sizes, leading
 * dimensions), ENKF_ERR_WORKSPACE, ENKF_ERR_CUDA.
 */
ENKF_API enkf_status enkf_rows_workspace(int64_t nobs, int32_t nens, size_t* bytes);
ENKF_API enkf_status enkf_rows_level(int32_t precision, int64_t nobs, int32_t nens, int32_t k, const void* r,
                                     const void* V, int64_t ldv, const void* D, int64_t ldd, void* U, int64_t ldu,
                                     void* Z, int64_t ldz, const double* coef, double* C, double* gamma,
                                     double* part, void* workspace, size_t workspace_bytes, void* stream);
ENKF_API enkf_status enkf_rows_gram(int32_t precision, int64_t nobs, int32_t nens, const void* V, int64_t ldv,
                                    const void* U, int64_t ldu, double* Q, void* workspace, size_t workspace_bytes,
                                    void* stream);
ENKF_API enkf_status enkf_rows_assemble(int32_t precision, int32_t nens, const double* Q, const double* C,
                                        const double* gamma, void* M, void* stream);
ENKF_API enkf_status enkf_rows_xa(int32_t precision, int64_t nstate, int32_t nens, const void* XB, int64_t ldb,
                                  const void* dXB, int64_t ldx, const void* M, void* XA, int64_t lda, void* stream);
ENKF_API enkf_status enkf_rows_status(void* workspace, void* stream, int32_t* status);

/* Human-readable name of a status code (static string). */
ENKF_API const char* enkf_status_string(enkf_status s);

/* Detail text of the last error raised on the calling thread (thread-local). */
ENKF_API const char* enkf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ENKF_ISM_H */
