/*
 * Plain FP64 CPU oracle of the iterative Sherman-Morrison EnKF analysis
 * (Nino-Ruiz, Sandu and Anderson, "An Efficient Implementation of the Ensemble
 * Kalman Filter Based on an Iterative Sherman-Morrison Formula").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The CUDA library shares no code,
 * header or constant with it, and neither links the other.
 *
 * Every routine follows the paper's definition step by step, in double
 * precision, with no blocking, fusion or reordering beyond what the paper
 * writes.  Sums over observations run in ascending row order.  Parallelism is
 * only over independent columns (or state rows), so the result does not depend
 * on the thread count.  Compile with -fno-fast-math -ffp-contract=off.
 *
 * Storage: column-major, one ensemble member per column, leading dimension ld.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Ensemble statistics and observation space (Sec. 2 and Sec. 3)           */
/* ------------------------------------------------------------------------ */

/*
 * Ensemble mean and deviations, eq. (ensemble-background-mean):
 *   xbar = X_B 1 / Nens,   dX_B[:, e] = X_B[:, e] - xbar.
 * The paper's S (eq. EnSM:Matrix-member-deviations) is dX_B / sqrt(Nens - 1).
 */
void oracle_ensemble_deviations(int64_t nstate, int32_t nens, const double* XB, int64_t ldb,
                                double* xbar, double* dXB, int64_t ldx) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nstate; ++i) {
        double s = 0.0;
        for (int32_t e = 0; e < nens; ++e) s += XB[e * ldb + i];
        double m = s / (double)nens;
        if (xbar) xbar[i] = m;
        for (int32_t e = 0; e < nens; ++e) dXB[e * ldx + i] = XB[e * ldb + i] - m;
    }
}

/*
 * Observation-space ensemble deviations, eq. (EnKSM:member-observations):
 *   V = H S = H dX_B / sqrt(Nens - 1),
 * with H selecting state rows 0, stride, 2*stride, ... (nobs rows).
 */
void oracle_observe_deviations(int64_t nobs, int32_t nens, int32_t stride, const double* dXB, int64_t ldx,
                               double* V, int64_t ldv) {
    double scale = 1.0 / sqrt((double)(nens - 1));
#pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < nens; ++e)
        for (int64_t j = 0; j < nobs; ++j) V[e * ldv + j] = dXB[e * ldx + j * (int64_t)stride] * scale;
}

/*
 * Innovations, eq. (EnKSM:system-rhs):  D = Y - H X_B.
 */
void oracle_innovations(int64_t nobs, int32_t nens, int32_t stride, const double* Y, int64_t ldy,
                        const double* XB, int64_t ldb, double* D, int64_t ldd) {
#pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < nens; ++e)
        for (int64_t j = 0; j < nobs; ++j) D[e * ldd + j] = Y[e * ldy + j] - XB[e * ldb + j * (int64_t)stride];
}

/* ------------------------------------------------------------------------ */
/* Iterative Sherman-Morrison formula S_*(R, V, D), Sec. 3.1               */
/* ------------------------------------------------------------------------ */

/*
 * Step 1, eq. (SM-step-1):  Z^(0) = R^{-1} D,  U^(0) = R^{-1} V,  R = diag(r).
 * Each row j is divided by r_j.  nrhs is the number of columns of D
 * (Nens in the paper).  Adds nobs * (nens + nrhs) long operations (one
 * division per entry; 2 Nobs Nens when nrhs = Nens, eq.
 * EnKSM:operations-count-step-one) to *longops when longops is not NULL.
 */
void oracle_ism_step1(int64_t nobs, int32_t nens, int32_t nrhs, const double* r,
                      const double* V, int64_t ldv, const double* D, int64_t ldd,
                      double* U, int64_t ldu, double* Z, int64_t ldz, int64_t* longops) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < nrhs; ++i)
        for (int64_t j = 0; j < nobs; ++j) Z[i * ldz + j] = D[i * ldd + j] / r[j];
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < nens; ++i)
        for (int64_t j = 0; j < nobs; ++j) U[i * ldu + j] = V[i * ldv + j] / r[j];
    if (longops) *longops += (int64_t)nobs * (nens + nrhs);
}

/* v^T x over rows 0..nobs-1, ascending. */
static double dot_asc(int64_t nobs, const double* v, const double* x) {
    double s = 0.0;
    for (int64_t j = 0; j < nobs; ++j) s += v[j] * x[j];
    return s;
}

/*
 * The same sum, as accurate as if formed in twice the working precision and rounded once:
 * the Dot2 algorithm of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
 * Sci. Comput. 26, 2005) -- every product split exactly into p + e by a fused
 * multiply-add, every partial sum into s + q by Knuth's TwoSum, the errors accumulated
 * and added at the end.  Used for V^T Z, whose entries are the part of Z in range(V) and
 * so cancel to ~1e-6 of sum |v||z| at the large workloads: the plain ascending sum would
 * lose ~1e-10 of them, this one keeps ~1e-16 of the sum as given.  (The rounding error of
 * an FP64 solve's Z is a larger effect on M at such gamma; ism_solve_refined in the Python
 * module removes it by one step of refinement.)
 */
static double dot2_asc(int64_t nobs, const double* v, const double* x) {
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < nobs; ++j) {
        const double p = v[j] * x[j];
        const double e = fma(v[j], x[j], -p);
        const double t = s + p;
        const double z = t - s;
        const double q = (s - (t - z)) + (p - z);
        s = t;
        c += q + e;
    }
    return s + c;
}

/*
 * Step 2, eqs. (SM-step-2-h), (SM-step-2-Z), (SM-step-2-u): for levels
 * k = 1..Nens (0-based k = 0..Nens-1 here):
 *   gamma_k = 1 + v_k^T u_k^(k-1)
 *   h_k     = u_k^(k-1) / gamma_k
 *   Z^(k)   = Z^(k-1) - h_k (v_k^T Z^(k-1))                 (every column of Z)
 *   u_i^(k) = u_i^(k-1) - h_k (v_k^T u_i^(k-1)),  i > k     (later columns of U only)
 * Column u_k is not touched at level k or after (Sec. 3.1: at iteration k only
 * columns k < i <= Nens are updated).  All three lines read level-(k-1) data.
 *
 * gamma (length nens) receives gamma_k when not NULL.  Long operations (products
 * and divisions, as counted in Sec. 3.2) are added to *longops when not NULL.
 * Returns 0, or k+1 when gamma_k is not finite or not positive (the level at
 * which the recurrence cannot proceed, Sec. 3.3).
 */
int oracle_ism_step2(int64_t nobs, int32_t nens, int32_t nrhs, const double* V, int64_t ldv,
                     double* U, int64_t ldu, double* Z, int64_t ldz, double* gamma, int64_t* longops) {
    double* h = (double*)malloc(sizeof(double) * (size_t)(nobs > 0 ? nobs : 1));
    if (!h) return -1;
    int status = 0;
    for (int32_t k = 0; k < nens; ++k) {
        const double* vk = V + k * ldv;
        const double* uk = U + k * ldu;
        double g = 1.0 + dot_asc(nobs, vk, uk);
        if (gamma) gamma[k] = g;
        if (!(g > 0.0) || !isfinite(g)) { status = k + 1; break; }
        for (int64_t j = 0; j < nobs; ++j) h[j] = uk[j] / g;
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t i = 0; i < nrhs; ++i) {
            double* z = Z + i * ldz;
            double c = dot_asc(nobs, vk, z);
            for (int64_t j = 0; j < nobs; ++j) z[j] -= h[j] * c;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t i = k + 1; i < nens; ++i) {
            double* u = U + i * ldu;
            double c = dot_asc(nobs, vk, u);
            for (int64_t j = 0; j < nobs; ++j) u[j] -= h[j] * c;
        }
        if (longops) *longops += 2 * nobs + 2 * nobs * (int64_t)nrhs + 2 * nobs * (int64_t)(nens - 1 - k);
    }
    free(h);
    return status;
}

/*
 * S_*(R, V, D): Step 1 then Step 2.  U is caller-provided scratch (nobs x nens).
 */
int oracle_ism_solve(int64_t nobs, int32_t nens, int32_t nrhs, const double* r,
                     const double* V, int64_t ldv, const double* D, int64_t ldd,
                     double* U, int64_t ldu, double* Z, int64_t ldz, double* gamma, int64_t* longops) {
    oracle_ism_step1(nobs, nens, nrhs, r, V, ldv, D, ldd, U, ldu, Z, ldz, longops);
    return oracle_ism_step2(nobs, nens, nrhs, V, ldv, U, ldu, Z, ldz, gamma, longops);
}

/* ------------------------------------------------------------------------ */
/* Analysis assembly, Sec. 3.1 (SMEnKF)                                     */
/* ------------------------------------------------------------------------ */

/*
 * M = V^T Z / sqrt(Nens - 1)  (nens x nrhs, column-major, ld = nens), so that
 * S V^T Z = dX_B M with S = dX_B / sqrt(Nens - 1).  Each entry is the plain definition,
 * summed in ascending row order with the Dot2 compensation (dot2_asc).
 */
void oracle_vtz(int64_t nobs, int32_t nens, int32_t nrhs, const double* V, int64_t ldv,
                const double* Z, int64_t ldz, double* M) {
    double scale = 1.0 / sqrt((double)(nens - 1));
#pragma omp parallel for schedule(static) collapse(2)
    for (int32_t i = 0; i < nrhs; ++i)
        for (int32_t m = 0; m < nens; ++m) M[i * nens + m] = dot2_asc(nobs, V + m * ldv, Z + i * ldz) * scale;
}

/*
 * X_A = X_B + S V^T Z = X_B + dX_B M  (SMEnKF analysis, Sec. 3.1).  The sum over
 * ensemble members runs in ascending order.  XA may alias XB.
 */
void oracle_analysis_update(int64_t nstate, int32_t nens, int32_t nrhs, const double* XB, int64_t ldb,
                            const double* dXB, int64_t ldx, const double* M, double* XA, int64_t lda) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nstate; ++i) {
        for (int32_t e = 0; e < nrhs; ++e) {
            double s = 0.0;
            for (int32_t m = 0; m < nens; ++m) s += dXB[m * ldx + i] * M[e * nens + m];
            XA[e * lda + i] = XB[e * ldb + i] + s;
        }
    }
}

/*
 * Residual of the analysis linear system, eq. (EnKSM:system-to-solve-V):
 *   Res = D - (R + V V^T) Z = D - (r o Z + V (V^T Z)).
 * P = V^T Z is formed first (nens x nrhs, each entry by dot2_asc: its entries cancel, and
 * an error in P enters Res undamped), then each entry of Res.
 */
int oracle_residual(int64_t nobs, int32_t nens, int32_t nrhs, const double* r, const double* V, int64_t ldv,
                    const double* D, int64_t ldd, const double* Z, int64_t ldz, double* Res, int64_t ldr) {
    double* P = (double*)malloc(sizeof(double) * (size_t)nens * (size_t)(nrhs > 0 ? nrhs : 1));
    if (!P) return -1;
#pragma omp parallel for schedule(static) collapse(2)
    for (int32_t i = 0; i < nrhs; ++i)
        for (int32_t m = 0; m < nens; ++m) P[i * nens + m] = dot2_asc(nobs, V + m * ldv, Z + i * ldz);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < nrhs; ++i) {
        for (int64_t j = 0; j < nobs; ++j) {
            double s = 0.0;
            for (int32_t m = 0; m < nens; ++m) s += V[m * ldv + j] * P[i * nens + m];
            Res[i * ldr + j] = D[i * ldd + j] - (r[j] * Z[i * ldz + j] + s);
        }
    }
    free(P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lorenz-96 forecast model, Sec. 4.2 eq. (eqn:Lorenz96), integrated by RK4 */
/* ------------------------------------------------------------------------ */

/*
 * dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F with periodic indices
 * (0-based here; the paper writes the wrap-around cases i = 1 and i = Nstate
 * explicitly).
 */
void oracle_l96_rhs(int64_t n, const double* x, double F, double* dx) {
    for (int64_t i = 0; i < n; ++i) {
        double xp1 = x[(i + 1) % n];
        double xm1 = x[(i - 1 + n) % n];
        double xm2 = x[(i - 2 + 2 * n) % n];
        dx[i] = (xp1 - xm2) * xm1 - x[i] + F;
    }
}

/*
 * Classical fourth-order Runge-Kutta, nsteps steps of size dt, applied to every
 * ensemble member (column) of X independently:
 *   k1 = f(x), k2 = f(x + dt/2 k1), k3 = f(x + dt/2 k2), k4 = f(x + dt k3),
 *   x <- x + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 */
int oracle_l96_rk4(int64_t nstate, int32_t nens, double* X, int64_t ld, double F, double dt, int32_t nsteps) {
    int status = 0;
#pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < nens; ++e) {
        double* x = X + e * ld;
        double* w = (double*)malloc(sizeof(double) * (size_t)nstate * 5);
        if (!w) { status = -1; continue; }
        double *k1 = w, *k2 = w + nstate, *k3 = w + 2 * nstate, *k4 = w + 3 * nstate, *t = w + 4 * nstate;
        for (int32_t s = 0; s < nsteps; ++s) {
            oracle_l96_rhs(nstate, x, F, k1);
            for (int64_t i = 0; i < nstate; ++i) t[i] = x[i] + 0.5 * dt * k1[i];
            oracle_l96_rhs(nstate, t, F, k2);
            for (int64_t i = 0; i < nstate; ++i) t[i] = x[i] + 0.5 * dt * k2[i];
            oracle_l96_rhs(nstate, t, F, k3);
            for (int64_t i = 0; i < nstate; ++i) t[i] = x[i] + dt * k3[i];
            oracle_l96_rhs(nstate, t, F, k4);
            for (int64_t i = 0; i < nstate; ++i)
                x[i] = x[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        }
        free(w);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Inflation, localization and block-diagonal R (Sec. 3.1.1, 3.1.2, 3.1)    */
/* ------------------------------------------------------------------------ */

/*
 * Multiplicative inflation (Sec. 3.1.1, inflation aspects): every member is
 * pushed away from the ensemble mean by the factor alpha,
 *   x_i <- xbar + alpha (x_i - xbar),   1 <= i <= Nens,
 * so the ensemble covariance grows by alpha^2.  In place on X (nstate x nens).
 */
void oracle_inflate(int64_t nstate, int32_t nens, double alpha, double* X, int64_t ld) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nstate; ++i) {
        double s = 0.0;
        for (int32_t e = 0; e < nens; ++e) s += X[e * ld + i];
        double m = s / (double)nens;
        for (int32_t e = 0; e < nens; ++e) X[e * ld + i] = m + alpha * (X[e * ld + i] - m);
    }
}

/*
 * Impact factor delta_{i,j} of observation j on state component i (Sec. 3.1.2,
 * partial localization; the Lorenz-96 choice of Sec. 4.2 is length = Nstate and
 * no cut-off): the distance d between state index i and the observed state index
 * j * stride, taken on the periodic ring of nstate points, gives
 *   delta = exp(-d / length)   when radius < 0 or d <= radius,
 *   delta = 0                  outside the radius of influence.
 */
static double loc_delta(int64_t nstate, int32_t stride, double length, double radius, int64_t i, int64_t j) {
    int64_t d = i - j * (int64_t)stride;
    if (d < 0) d = -d;
    if (nstate - d < d) d = nstate - d;
    if (radius >= 0.0 && (double)d > radius) return 0.0;
    return exp(-(double)d / length);
}

/*
 * Partial localization, eq. (localized-correction-component), written out as
 * printed: for every state component i and member l,
 *   dX[i, l] = sum_k S[i, k] sum_j delta_{i,j} V[j, k] Z[j, l],
 * with S = dX_B / sqrt(Nens - 1) (k over the nens members, j over the nobs
 * observations; V is nobs x nens, so the paper's V_{k,j} is V[j, k] here).
 * Costs Nstate * nrhs * Nens * Nobs products: tiny inputs only.  Writes the
 * increment dX (nstate x nrhs, ld ldo).
 */
void oracle_localized_increment_literal(int64_t nstate, int64_t nobs, int32_t nens, int32_t nrhs, int32_t stride,
                                        double length, double radius, const double* dXB, int64_t ldx,
                                        const double* V, int64_t ldv, const double* Z, int64_t ldz,
                                        double* dX, int64_t ldo) {
    double scale = 1.0 / sqrt((double)(nens - 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nstate; ++i) {
        for (int32_t l = 0; l < nrhs; ++l) {
            double outer = 0.0;
            for (int32_t k = 0; k < nens; ++k) {
                double inner = 0.0;
                for (int64_t j = 0; j < nobs; ++j)
                    inner += loc_delta(nstate, stride, length, radius, i, j) * V[k * ldv + j] * Z[l * ldz + j];
                outer += dXB[k * ldx + i] * scale * inner;
            }
            dX[l * ldo + i] = outer;
        }
    }
}

/*
 * Partial localization in the matrix form the paper gives beside the component
 * formula (Sec. 3.1.2):  dX = (Delta o (S V^T)) Z,  Delta = (delta_{i,j}) of size
 * Nstate x Nobs, o the Schur product.  For each state row i: the row
 * t_j = delta_{i,j} (S V^T)[i, j] over all observations j (sum over members in
 * ascending order), then dX[i, l] = sum_j t_j Z[j, l] (ascending j), and
 *   X_A = X_B + dX.
 * XA may alias XB.
 */
int oracle_localized_update(int64_t nstate, int64_t nobs, int32_t nens, int32_t nrhs, int32_t stride, double length,
                            double radius, const double* dXB, int64_t ldx, const double* V, int64_t ldv,
                            const double* Z, int64_t ldz, const double* XB, int64_t ldb, double* XA, int64_t lda) {
    double scale = 1.0 / sqrt((double)(nens - 1));
    int status = 0;
#pragma omp parallel
    {
        double* t = (double*)malloc(sizeof(double) * (size_t)(nobs > 0 ? nobs : 1));
        if (!t) {
#pragma omp atomic write
            status = -1;
        } else {
#pragma omp for schedule(static)
            for (int64_t i = 0; i < nstate; ++i) {
                for (int64_t j = 0; j < nobs; ++j) {
                    double sv = 0.0;
                    for (int32_t k = 0; k < nens; ++k) sv += dXB[k * ldx + i] * scale * V[k * ldv + j];
                    t[j] = loc_delta(nstate, stride, length, radius, i, j) * sv;
                }
                for (int32_t l = 0; l < nrhs; ++l) {
                    double s = 0.0;
                    for (int64_t j = 0; j < nobs; ++j) s += t[j] * Z[l * ldz + j];
                    XA[l * lda + i] = XB[l * ldb + i] + s;
                }
            }
            free(t);
        }
    }
    return status;
}

/*
 * Step 1 with a block-diagonal R (Sec. 3.1: R^{-1} = diag(R_b^{-1}) is applied
 * block by block):  Z^(0) = R^{-1} D,  U^(0) = R^{-1} V.  Block b covers rows
 * [b*bs, min(nobs, (b+1)*bs)) and is stored dense, column-major, in the leading
 * m x m part of the bs x bs matrix at Rblk + b*bs*bs (m = rows of the block).
 * Each block is factored R_b = L L^T (Cholesky) and every column is solved by
 * forward then backward substitution.  Returns 0, or -(b+1) when block b is not
 * positive definite.
 */
int oracle_ism_step1_blockdiag(int64_t nobs, int32_t nens, int32_t nrhs, int32_t bs, const double* Rblk,
                               const double* V, int64_t ldv, const double* D, int64_t ldd, double* U, int64_t ldu,
                               double* Z, int64_t ldz) {
    int64_t nblk = (nobs + bs - 1) / bs;
    int status = 0;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
        int64_t r0 = b * bs;
        int32_t m = (int32_t)((nobs - r0) < bs ? (nobs - r0) : bs);
        const double* A = Rblk + b * (int64_t)bs * bs;
        double* L = (double*)calloc((size_t)m * m, sizeof(double));
        double* x = (double*)malloc(sizeof(double) * (size_t)m);
        if (!L || !x) {
            free(L);
            free(x);
#pragma omp atomic write
            status = -1;
            continue;
        }
        int ok = 1;
        for (int32_t c = 0; c < m && ok; ++c) {
            double s = A[c * bs + c];
            for (int32_t p = 0; p < c; ++p) s -= L[p * m + c] * L[p * m + c];
            if (!(s > 0.0)) { ok = 0; break; }
            double lcc = sqrt(s);
            L[c * m + c] = lcc;
            for (int32_t q = c + 1; q < m; ++q) {
                double t = A[c * bs + q];
                for (int32_t p = 0; p < c; ++p) t -= L[p * m + q] * L[p * m + c];
                L[c * m + q] = t / lcc;
            }
        }
        if (!ok) {
#pragma omp atomic write
            status = (int)-(b + 1);
        } else {
            for (int32_t col = 0; col < nens + nrhs; ++col) {
                const double* in = col < nens ? V + col * ldv + r0 : D + (col - nens) * ldd + r0;
                double* out = col < nens ? U + col * ldu + r0 : Z + (col - nens) * ldz + r0;
                for (int32_t q = 0; q < m; ++q) {          /* L y = rhs */
                    double t = in[q];
                    for (int32_t p = 0; p < q; ++p) t -= L[p * m + q] * x[p];
                    x[q] = t / L[q * m + q];
                }
                for (int32_t q = m - 1; q >= 0; --q) {     /* L^T out = y */
                    double t = x[q];
                    for (int32_t p = q + 1; p < m; ++p) t -= L[q * m + p] * out[p];
                    out[q] = t / L[q * m + q];
                }
            }
        }
        free(L);
        free(x);
    }
    return status;
}

/*
 * Step 2 with pivoting (Sec. 3.4, eq. EnKSM:gamma-value): before level k the
 * candidate with the largest |1 + v_i^T u_i^(k-1)| over k <= i < Nens (0-based;
 * ties go to the lowest index) is found, and columns k and that index are
 * interchanged in V and U^(k-1) (the columns of Z are right-hand sides and stay
 * where they are); then level k runs as in oracle_ism_step2.  V is copied first
 * (the caller's V is not modified).  perm[k] receives the original column index
 * that level k used; gamma[k] its gamma_k.  Long operations as in
 * oracle_ism_step2 plus Nobs products per candidate (Sec. 3.4 counts every
 * candidate, the pivot included, on top of T_SMF).
 */
int oracle_ism_step2_pivot(int64_t nobs, int32_t nens, int32_t nrhs, const double* V, int64_t ldv, double* U,
                           int64_t ldu, double* Z, int64_t ldz, double* gamma, int32_t* perm, int64_t* longops) {
    double* Vc = (double*)malloc(sizeof(double) * (size_t)(nobs > 0 ? nobs : 1) * (size_t)(nens > 0 ? nens : 1));
    double* h = (double*)malloc(sizeof(double) * (size_t)(nobs > 0 ? nobs : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)(nens > 0 ? nens : 1));
    if (!Vc || !h || !g) {
        free(Vc);
        free(h);
        free(g);
        return -1;
    }
    for (int32_t i = 0; i < nens; ++i) {
        memcpy(Vc + i * nobs, V + i * ldv, sizeof(double) * (size_t)nobs);
        perm[i] = i;
    }
    int status = 0;
    for (int32_t k = 0; k < nens; ++k) {
#pragma omp parallel for schedule(static)
        for (int32_t i = k; i < nens; ++i) g[i] = 1.0 + dot_asc(nobs, Vc + i * nobs, U + i * ldu);
        if (longops) *longops += (int64_t)(nens - k) * nobs;
        int32_t ind = k;
        for (int32_t i = k + 1; i < nens; ++i)
            if (fabs(g[i]) > fabs(g[ind])) ind = i;
        if (ind != k) {
            for (int64_t j = 0; j < nobs; ++j) {
                double t = Vc[k * nobs + j];
                Vc[k * nobs + j] = Vc[ind * nobs + j];
                Vc[ind * nobs + j] = t;
                t = U[k * ldu + j];
                U[k * ldu + j] = U[ind * ldu + j];
                U[ind * ldu + j] = t;
            }
            int32_t t = perm[k];
            perm[k] = perm[ind];
            perm[ind] = t;
        }
        const double* vk = Vc + k * nobs;
        const double* uk = U + k * ldu;
        double gk = g[ind];
        if (gamma) gamma[k] = gk;
        if (!(gk > 0.0) || !isfinite(gk)) { status = k + 1; break; }
        for (int64_t j = 0; j < nobs; ++j) h[j] = uk[j] / gk;
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t i = 0; i < nrhs; ++i) {
            double* z = Z + i * ldz;
            double c = dot_asc(nobs, vk, z);
            for (int64_t j = 0; j < nobs; ++j) z[j] -= h[j] * c;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t i = k + 1; i < nens; ++i) {
            double* u = U + i * ldu;
            double c = dot_asc(nobs, vk, u);
            for (int64_t j = 0; j < nobs; ++j) u[j] -= h[j] * c;
        }
        if (longops) *longops += 2 * nobs + 2 * nobs * (int64_t)nrhs + 2 * nobs * (int64_t)(nens - 1 - k);
    }
    free(Vc);
    free(h);
    free(g);
    return status;
}
