// C ABI of libenkf_ism (declared in include/enkf_ism.h): plans, argument
// validation, workspace layout and the orchestration of one analysis.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/enkf_ism.h"
#include "internal.h"

using namespace enkf;

namespace {

thread_local char g_last_error[1024] = "";

enkf_status fail(enkf_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

enkf_status cuda_fail(cudaError_t e, const char* what) {
    return fail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CU(call, what)                                  \
    do {                                                \
        cudaError_t e__ = (call);                       \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }

}  // namespace

void enkf::set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

struct enkf_ism_plan_s {
    int64_t nstate, nobs;
    int32_t nens, mode, panel_b;
    uint32_t flags;
    int device;
    bool fp64;
    bool small;          // the whole analysis in one CTA (small.cu)
    bool tc5;            // three-piece BF16 panel solve on tcgen05 (ism_panel_tc05.cu)
    Tc5Launch T5;
    size_t w;                 // element size
    LevelLaunch L;
    PanelLaunch P;
    int32_t nsplit;
    int64_t ldu, ldzw;
    // workspace layout (byte offsets)
    size_t off_ctl, off_U, off_Z, off_part, off_coefg, off_C, off_gamma, off_Qpart, off_Q, off_M, off_M64, off_Msplit,
        off_delta, off_P, off_Md, off_rnorm, off_vp, off_up, off_vpc, off_upc, off_ufc, off_wfin, off_Cd, total;
    int64_t ldp;              // row pitch of the 16-bit operand pieces (tensor-core panel modes)
    bool refine;
    // latched status of the previous call
    int* h_status;            // pinned host word
    cudaEvent_t done;
    bool pending;
    // kernel-phase timing
    bool prof;
    int nprof;
    cudaEvent_t* prof_ev;     // [2 * kProfCap]
    int* prof_phase;          // [kProfCap]
};

namespace {
constexpr int kProfCap = 4096;

// Records the start event of a phase; returns the slot or -1.
int prof_begin(enkf_ism_plan_s* p, int phase, cudaStream_t s) {
    if (!p->prof || p->nprof >= kProfCap) return -1;
    const int i = p->nprof++;
    p->prof_phase[i] = phase;
    cudaEventRecord(p->prof_ev[2 * i], s);
    return i;
}

void prof_end(enkf_ism_plan_s* p, int slot, cudaStream_t s) {
    if (slot >= 0) cudaEventRecord(p->prof_ev[2 * slot + 1], s);
}

// A phase slot whose two events the caller records itself (around one launch inside a
// phase); -1 when profiling is off or the record is full.
int prof_reserve(enkf_ism_plan_s* p, int phase) {
    if (!p->prof || p->nprof >= kProfCap) return -1;
    const int i = p->nprof++;
    p->prof_phase[i] = phase;
    return i;
}
}  // namespace

extern "C" {

const char* enkf_status_string(enkf_status s) {
    switch (s) {
        case ENKF_OK: return "ENKF_OK";
        case ENKF_ERR_ARG: return "ENKF_ERR_ARG";
        case ENKF_ERR_SHAPE: return "ENKF_ERR_SHAPE";
        case ENKF_ERR_CUDA: return "ENKF_ERR_CUDA";
        case ENKF_ERR_NUMERIC: return "ENKF_ERR_NUMERIC";
        case ENKF_ERR_TIMEOUT: return "ENKF_ERR_TIMEOUT";
        case ENKF_ERR_UNSUPPORTED: return "ENKF_ERR_UNSUPPORTED";
        case ENKF_ERR_WORKSPACE: return "ENKF_ERR_WORKSPACE";
    }
    return "ENKF_UNKNOWN_STATUS";
}

const char* enkf_last_error(void) { return g_last_error; }

enkf_status enkf_ism_plan(enkf_ism_plan_t* out, int64_t nstate, int64_t nobs, int32_t nens, int32_t mode,
                          int32_t panel_b, uint32_t flags, size_t* workspace_bytes) {
    if (!out || !workspace_bytes) return fail(ENKF_ERR_ARG, "enkf_ism_plan: NULL out or workspace_bytes");
    *out = nullptr;
    if (nstate < 1 || nobs < 1 || nens < 1)
        return fail(ENKF_ERR_SHAPE, "enkf_ism_plan: need nstate, nobs, nens >= 1 (got %lld, %lld, %d)",
                    (long long)nstate, (long long)nobs, nens);
    if (nens > 1024) return fail(ENKF_ERR_SHAPE, "enkf_ism_plan: nens %d > 1024", nens);
    if (nobs > ((int64_t)1 << 40) || nstate > ((int64_t)1 << 40))
        return fail(ENKF_ERR_SHAPE, "enkf_ism_plan: size too large");
    const bool panel = (mode == ENKF_PANEL_FP32 || mode == ENKF_PANEL_BF16 || mode == ENKF_PANEL_FP16 ||
                        mode == ENKF_PANEL_BF16X3);
    if (mode != ENKF_FP64 && mode != ENKF_FP32 && !panel) return fail(ENKF_ERR_ARG, "enkf_ism_plan: bad mode %d", mode);
    if (panel && (panel_b < 0 || panel_b > panel_max_b()))
        return fail(ENKF_ERR_ARG, "enkf_ism_plan: panel_b %d out of [1, %d]", panel_b, panel_max_b());
    if (flags & ~(ENKF_FLAG_REFINE | ENKF_FLAG_NO_CHECKS | ENKF_FLAG_TEST_TIMEOUT))
        return fail(ENKF_ERR_ARG, "enkf_ism_plan: unknown flag bits 0x%x", flags);
    enkf_ism_plan_s* p = new (std::nothrow) enkf_ism_plan_s();
    if (!p) return fail(ENKF_ERR_ARG, "enkf_ism_plan: out of host memory");
    p->nstate = nstate;
    p->nobs = nobs;
    p->nens = nens;
    p->mode = mode;
    p->panel_b = panel ? (panel_b > 0 ? panel_b : panel_max_b()) : 0;
    p->flags = flags;
    p->fp64 = (mode == ENKF_FP64);
    p->w = p->fp64 ? 8 : 4;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) {
        if (panel) {
            const int prec = mode == ENKF_PANEL_BF16     ? 1
                             : mode == ENKF_PANEL_FP16   ? 2
                             : mode == ENKF_PANEL_BF16X3 ? 3
                                                         : 0;
            e = panel_plan(nobs, nens, p->panel_b, prec, &p->P);
            p->L.grid = p->P.grid;
            if (e == cudaSuccess && prec == 3 && p->panel_b == tc5_panel_b()) {
                e = tc5_plan(nobs, nens, &p->T5);
                p->tc5 = e == cudaSuccess;
                if (p->tc5 && p->T5.grid > p->L.grid) p->L.grid = p->T5.grid;
            }
        } else {
            e = level_plan(p->fp64, nobs, nens, &p->L);
            p->small = !(flags & ENKF_FLAG_TEST_TIMEOUT) && small_fits(p->fp64, nobs, nens);
        }
    }
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "enkf_ism_plan: level_plan");
    }
    p->nsplit = gram_upper_nsplit(nobs, nens);
    p->ldu = pad32(nobs);
    p->ldzw = pad32(nobs);
    const size_t N = (size_t)nens;
    size_t o = 0;
    p->off_ctl = o; o = align256(o + sizeof(Control));
    p->off_U = o; o = align256(o + p->w * (size_t)p->ldu * N);
    p->off_Z = o; o = align256(o + p->w * (size_t)p->ldzw * N);
    const size_t part_per_cta = panel ? (size_t)p->P.part_stride : 2 * N;
    const size_t coef_len = panel ? (size_t)p->P.part_stride : 2 * N;
    p->off_part = o; o = align256(o + sizeof(double) * (size_t)p->L.grid * part_per_cta);
    p->off_coefg = o; o = align256(o + sizeof(double) * coef_len);
    p->off_C = o; o = align256(o + sizeof(double) * N * N);
    p->off_gamma = o; o = align256(o + sizeof(double) * N);
    p->off_Qpart = o; o = align256(o + sizeof(double) * (size_t)p->nsplit * N * N);
    p->off_Q = o; o = align256(o + sizeof(double) * N * N);
    p->off_M = o; o = align256(o + p->w * N * N);
    p->off_M64 = o; o = align256(o + sizeof(double) * N * N);
    p->off_Msplit = o; o = align256(o + xa_split_bytes(nens));
    {
        // tensor-core panel modes: pieces of V ([pieces][N][ldp]) and of two panels' U_P
        // ([2][pieces][b_max][ldp]), 16-bit
        const int pieces = panel ? panel_pieces(p->P.prec) : 0;
        p->ldp = (nobs + 63 + 7) / 8 * 8;
        p->off_vp = o; o = align256(o + sizeof(uint16_t) * (size_t)pieces * N * p->ldp);
        p->off_up = o; o = align256(o + sizeof(uint16_t) * 2 * (size_t)pieces * panel_max_b() * p->ldp);
        p->off_vpc = o; o = align256(o + (p->tc5 ? tc5_vpc_bytes(nobs, nens) : 0));
        p->off_upc = o; o = align256(o + (p->tc5 ? tc5_upc_bytes(nobs) : 0));
    }
    p->refine = panel && (flags & ENKF_FLAG_REFINE);
    if (p->refine) {
        p->off_delta = o; o = align256(o + sizeof(float) * (size_t)p->ldzw * N);
        p->off_P = o; o = align256(o + sizeof(double) * N * N);
        p->off_Md = o; o = align256(o + sizeof(double) * N * N);
        p->off_rnorm = o; o = align256(o + sizeof(double) * 1040);   // residual-norm partials + result
        // the tensor-core solve's stored factors for its correction sweep
        p->off_ufc = o; o = align256(o + (p->tc5 ? tc5_vpc_bytes(nobs, nens) : 0));
        p->off_wfin = o; o = align256(o + (p->tc5 ? tc5_wfin_bytes(nens) : 0));
        p->off_Cd = o; o = align256(o + (p->tc5 ? sizeof(double) * N * N : 0));
    }
    p->total = o;
    e = cudaMallocHost(&p->h_status, sizeof(int));   // pinned host word, not device memory
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (p->h_status) cudaFreeHost(p->h_status);
        delete p;
        return cuda_fail(e, "enkf_ism_plan: host status");
    }
    *p->h_status = 0;
    p->pending = false;
    *workspace_bytes = p->total;
    *out = p;
    return ENKF_OK;
}

void enkf_ism_plan_destroy(enkf_ism_plan_t p) {
    if (!p) return;
    if (p->pending) cudaEventSynchronize(p->done);
    cudaEventDestroy(p->done);
    cudaFreeHost(p->h_status);
    if (p->prof_ev) {
        for (int i = 0; i < 2 * kProfCap; ++i) cudaEventDestroy(p->prof_ev[i]);
        free(p->prof_ev);
        free(p->prof_phase);
    }
    delete p;
}

enkf_status enkf_ism_profile(enkf_ism_plan_t p, int32_t enable) {
    if (!p) return fail(ENKF_ERR_ARG, "enkf_ism_profile: NULL plan");
    if (enable && !p->prof_ev) {
        p->prof_ev = (cudaEvent_t*)calloc(2 * kProfCap, sizeof(cudaEvent_t));
        p->prof_phase = (int*)calloc(kProfCap, sizeof(int));
        if (!p->prof_ev || !p->prof_phase) return fail(ENKF_ERR_ARG, "enkf_ism_profile: out of host memory");
        for (int i = 0; i < 2 * kProfCap; ++i) CU(cudaEventCreate(&p->prof_ev[i]), "cudaEventCreate");
    }
    p->prof = enable != 0;
    p->nprof = 0;
    return ENKF_OK;
}

enkf_status enkf_ism_profile_read(enkf_ism_plan_t p, double* ms, int32_t* count) {
    if (!p || !ms || !count) return fail(ENKF_ERR_ARG, "enkf_ism_profile_read: NULL argument");
    for (int i = 0; i < p->nprof; ++i) {
        // phases nest (a kernel's own slot inside its phase), so the last slot is not always
        // the last event recorded: wait for each
        CU(cudaEventSynchronize(p->prof_ev[2 * i + 1]), "cudaEventSynchronize");
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, p->prof_ev[2 * i], p->prof_ev[2 * i + 1]), "cudaEventElapsedTime");
        const int ph = p->prof_phase[i];
        if (ph >= 0 && ph < ENKF_PROFILE_PHASES) {
            ms[ph] += (double)t;
            count[ph] += 1;
        }
    }
    p->nprof = 0;
    return ENKF_OK;
}

enkf_status enkf_ism_gamma(enkf_ism_plan_t p, const void* workspace, double* gamma) {
    if (!p || !workspace || !gamma) return fail(ENKF_ERR_ARG, "enkf_ism_gamma: NULL argument");
    CU(cudaSetDevice(p->device), "cudaSetDevice");
    if (p->pending) CU(cudaEventSynchronize(p->done), "cudaEventSynchronize");
    CU(cudaMemcpy(gamma, (const char*)workspace + p->off_gamma, sizeof(double) * (size_t)p->nens,
                  cudaMemcpyDeviceToHost),
       "enkf_ism_gamma: copy");
    return ENKF_OK;
}

static enkf_status take_latched(enkf_ism_plan_t p) {
    if (!p->pending) return ENKF_OK;
    if (cudaEventQuery(p->done) != cudaSuccess) return ENKF_OK;   // not finished yet: checked later
    p->pending = false;
    const int st = *p->h_status;
    *p->h_status = 0;
    if (st != 0) return fail((enkf_status)st, "device status of a previous call: %s", enkf_status_string((enkf_status)st));
    return ENKF_OK;
}

static bool ld_ok(int64_t ld, int64_t rows) { return ld >= rows && ld >= 1; }

enkf_status enkf_obs_prep(enkf_ism_plan_t p, int32_t obs_stride, int32_t center, const void* XB, int64_t ldb, void* dXB,
                          int64_t ldx, const void* Y, int64_t ldy, void* V, int64_t ldv, void* D, int64_t ldd,
                          void* stream) {
    if (!p) return fail(ENKF_ERR_ARG, "enkf_obs_prep: NULL plan");
    if (obs_stride < 1) return fail(ENKF_ERR_SHAPE, "enkf_obs_prep: obs_stride %d < 1", obs_stride);
    if ((p->nobs - 1) * (int64_t)obs_stride >= p->nstate)
        return fail(ENKF_ERR_SHAPE, "enkf_obs_prep: (nobs-1)*stride >= nstate");
    if (p->nens < 2) return fail(ENKF_ERR_SHAPE, "enkf_obs_prep: nens must be >= 2");
    if (!dXB || !V) return fail(ENKF_ERR_ARG, "enkf_obs_prep: NULL dXB or V");
    if ((center || Y) && !XB) return fail(ENKF_ERR_ARG, "enkf_obs_prep: XB required");
    if (Y && !D) return fail(ENKF_ERR_ARG, "enkf_obs_prep: D required with Y");
    if (!ld_ok(ldx, p->nstate) || !ld_ok(ldv, p->nobs) || ((center || Y) && !ld_ok(ldb, p->nstate)) ||
        (Y && (!ld_ok(ldy, p->nobs) || !ld_ok(ldd, p->nobs))))
        return fail(ENKF_ERR_SHAPE, "enkf_obs_prep: leading dimension smaller than rows");
    CU(cudaSetDevice(p->device), "cudaSetDevice");
    const int slot = prof_begin(p, 0, (cudaStream_t)stream);
    CU(obs_prep(p->fp64, p->nstate, p->nobs, p->nens, obs_stride, center, XB, ldb, dXB, ldx, Y, ldy, V, ldv, D, ldd,
                (cudaStream_t)stream),
       "enkf_obs_prep launch");
    prof_end(p, slot, (cudaStream_t)stream);
    return ENKF_OK;
}

enkf_status enkf_ism_analysis(enkf_ism_plan_t p, const void* r, const void* V, int64_t ldv, const void* D, int64_t ldd,
                              const void* dXB, int64_t ldx, const void* XB, int64_t ldb, void* XA, int64_t lda, void* Z,
                              int64_t ldz, void* M, void* workspace, size_t workspace_bytes, void* stream,
                              enkf_ism_info* info) {
    if (!p) return fail(ENKF_ERR_ARG, "enkf_ism_analysis: NULL plan");
    if (!r || !V || !D) return fail(ENKF_ERR_ARG, "enkf_ism_analysis: NULL r, V or D");
    if (!ld_ok(ldv, p->nobs) || !ld_ok(ldd, p->nobs) || (Z && !ld_ok(ldz, p->nobs)))
        return fail(ENKF_ERR_SHAPE, "enkf_ism_analysis: ldv/ldd/ldz smaller than nobs");
    if (dXB) {
        if (!XB || !XA) return fail(ENKF_ERR_ARG, "enkf_ism_analysis: XB and XA required with dXB");
        if (!ld_ok(ldx, p->nstate) || !ld_ok(ldb, p->nstate) || !ld_ok(lda, p->nstate))
            return fail(ENKF_ERR_SHAPE, "enkf_ism_analysis: ldx/ldb/lda smaller than nstate");
        if (XA == XB && lda != ldb) return fail(ENKF_ERR_ARG, "enkf_ism_analysis: XA aliases XB with lda != ldb");
    }
    if ((dXB || M) && p->nens < 2)
        return fail(ENKF_ERR_SHAPE, "enkf_ism_analysis: M and X_A need nens >= 2 (S divides by sqrt(Nens-1))");
    if (!workspace || workspace_bytes < p->total)
        return fail(ENKF_ERR_WORKSPACE, "enkf_ism_analysis: workspace %zu bytes < required %zu", workspace_bytes,
                    p->total);
    if ((uintptr_t)workspace % 256 != 0) return fail(ENKF_ERR_WORKSPACE, "enkf_ism_analysis: workspace not 256-aligned");
    const uintptr_t wmask = p->w - 1;
    if (((uintptr_t)r | (uintptr_t)V | (uintptr_t)D | (uintptr_t)dXB | (uintptr_t)XB | (uintptr_t)XA | (uintptr_t)Z |
         (uintptr_t)M) & wmask)
        return fail(ENKF_ERR_ARG, "enkf_ism_analysis: pointer not aligned to the element size");

    enkf_status latched = take_latched(p);
    if (latched != ENKF_OK) return latched;

    CU(cudaSetDevice(p->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    Control* ctl = (Control*)(ws + p->off_ctl);
    CU(cudaMemsetAsync(ctl, 0, sizeof(Control), s), "cudaMemsetAsync(control)");

    void* Zp = Z ? Z : (void*)(ws + p->off_Z);
    const int64_t ldzp = Z ? ldz : p->ldzw;
    LevelArgs a;
    a.nobs = p->nobs;
    a.nens = p->nens;
    a.r = r;
    a.V = V;
    a.ldv = ldv;
    a.D = D;
    a.ldd = ldd;
    a.U = ws + p->off_U;
    a.ldu = p->ldu;
    a.Z = Zp;
    a.ldz = ldzp;
    a.part = (double*)(ws + p->off_part);
    a.coefg = (double*)(ws + p->off_coefg);
    a.C = (double*)(ws + p->off_C);
    a.gamma = (double*)(ws + p->off_gamma);
    a.ctl = ctl;
    a.rows_per_blk = p->L.rows_per_blk;
    a.rows_chunk = p->L.rows_chunk;
    a.check = (p->flags & ENKF_FLAG_NO_CHECKS) ? 0 : 1;
    a.test_skip_arrival = (p->flags & ENKF_FLAG_TEST_TIMEOUT) ? 1 : 0;
    a.timeout_ns = (p->flags & ENKF_FLAG_TEST_TIMEOUT) ? 20000000ull : 2000000000ull;
    int slot = prof_begin(p, 1, s);
    if (p->small) {
        SmallArgs sa;
        sa.nobs = (int32_t)p->nobs;
        sa.nens = p->nens;
        sa.nstate = p->nstate;
        sa.r = r;
        sa.V = V;
        sa.ldv = ldv;
        sa.D = D;
        sa.ldd = ldd;
        sa.dXB = dXB;
        sa.ldx = ldx;
        sa.XB = XB;
        sa.ldb = ldb;
        sa.XA = XA;
        sa.lda = lda;
        sa.Z = Z;
        sa.ldz = ldz;
        sa.M = M;
        sa.gamma = a.gamma;
        sa.ctl = ctl;
        sa.check = a.check;
        CU(small_launch(p->fp64, sa, s), "small-problem launch");
        prof_end(p, slot, s);
    } else {
    PanelArgs panel_args;
    bool solved_tc5 = false;
    if (p->mode == ENKF_PANEL_FP32 || p->mode == ENKF_PANEL_BF16 || p->mode == ENKF_PANEL_FP16 ||
        p->mode == ENKF_PANEL_BF16X3) {
        PanelArgs pa;
        pa.nobs = p->nobs;
        pa.nens = p->nens;
        pa.r = r;
        pa.V = V;
        pa.ldv = ldv;
        pa.D = D;
        pa.ldd = ldd;
        pa.U = a.U;
        pa.ldu = a.ldu;
        pa.Z = a.Z;
        pa.ldz = a.ldz;
        pa.part = a.part;
        pa.part_stride = p->P.part_stride;
        pa.coefg = a.coefg;
        pa.C = a.C;
        pa.gamma = a.gamma;
        pa.ctl = ctl;
        pa.rows_per_blk = p->P.rows_per_blk;
        pa.panel_b = p->panel_b;
        pa.check = a.check;
        pa.vec_ok = (((uintptr_t)a.U | (uintptr_t)a.Z | (uintptr_t)V | (uintptr_t)D) % 16 == 0) && (a.ldu % 4 == 0) &&
                    (ldd % 4 == 0) &&
                    (a.ldz % 4 == 0) && (ldv % 4 == 0) && (p->P.rows_per_blk % 4 == 0);
        pa.timeout_ns = a.timeout_ns;
        pa.refine = 0;
        pa.Qg = nullptr;
        pa.vp = (unsigned short*)(ws + p->off_vp);
        pa.up = (unsigned short*)(ws + p->off_up);
        pa.ldp = p->ldp;
        cudaError_t et = cudaErrorNotSupported;
        if (p->tc5) {
            const int k6 = prof_reserve(p, 6);
            et = tc5_solve(p->T5, pa, ws + p->off_vpc, ws + p->off_upc, p->refine ? ws + p->off_ufc : nullptr,
                           p->refine ? (float*)(ws + p->off_wfin) : nullptr, s, k6 >= 0 ? p->prof_ev[2 * k6] : nullptr,
                           k6 >= 0 ? p->prof_ev[2 * k6 + 1] : nullptr);
            if (et != cudaSuccess && k6 >= 0) --p->nprof;      // nothing was recorded in the slot
            if (et == cudaErrorNotSupported) (void)cudaGetLastError();
            else CU(et, "tensor-core panel launch");
            solved_tc5 = et == cudaSuccess;
        }
        if (et == cudaErrorNotSupported) {
            const int k6 = prof_begin(p, 6, s);
            CU(panel_launch(p->P, pa, s), "panel launch");
            prof_end(p, k6, s);
        }
        panel_args = pa;
    } else {
        CU(level_launch(p->fp64, p->L, a, s), "level-streaming launch");
    }
    prof_end(p, slot, s);

    if (M || dXB || p->refine) {
        double* Q = (double*)(ws + p->off_Q);
        void* Mp = M ? M : (void*)(ws + p->off_M);
        double* M64 = (double*)(ws + p->off_M64);
        if (!p->refine) {
            slot = prof_begin(p, 2, s);
            CU(gram_upper(p->fp64, p->nobs, p->nens, V, ldv, a.U, p->ldu, (double*)(ws + p->off_Qpart), p->nsplit, Q,
                          ctl, a.timeout_ns, s),
               "gram launch");
            prof_end(p, slot, s);
            slot = prof_begin(p, 3, s);
            CU(assemble_M(p->fp64, p->nens, Q, a.C, a.gamma, Mp, M64, s), "assemble_M launch");
            prof_end(p, slot, s);
        } else {
            // One step of iterative refinement: P = V^T Z1 from the coefficient identity of the
            // solve, the scaled residual R^-1 (D - r o Z1 - V P), the solve's stored factors applied
            // to it giving delta, then Z = Z1 + delta and M = (P + V^T delta) / sqrt(N - 1).  An
            // error e in P enters M only as (I + V^T R^-1 V)^-1 e (~e / gamma): the correction
            // takes up V e in the residual.
            slot = prof_begin(p, 5, s);
            double* P = (double*)(ws + p->off_P);
            double* Pd = (double*)(ws + p->off_Md);
            double* part = (double*)(ws + p->off_Qpart);
            float* delta = (float*)(ws + p->off_delta);
            // P from the identity needs the solve's own e = V^T Z1 - P well below gamma times the
            // target: true for the FP32-class and split-BF16 solves (e ~ u gamma |M| with u <= 2^-17),
            // not for the FP16 solve (u = 2^-11), which takes V^T Z1 summed exactly instead
            const bool p_identity = p->mode != ENKF_PANEL_FP16;
            if (info || !p_identity) {
                // V^T Z1 summed exactly, and (diagnostic) the true relative residual of Z1
                // (fixed-point digits on the tensor cores when V and Z are TMA-aligned, else
                // compensated FP32 sums on CUDA cores)
                cudaError_t eg = gram_exact(p->nobs, p->nens, (const float*)V, ldv, (const float*)Zp, ldzp, part,
                                            p->nsplit, P, ctl, a.timeout_ns, s);
                if (eg == cudaErrorNotSupported) {
                    (void)cudaGetLastError();
                    eg = gram_comp(p->nobs, p->nens, (const float*)V, ldv, (const float*)Zp, ldzp, part, p->nsplit,
                                   P, s);
                }
                CU(eg, "refine Gram V^T Z");
                CU(refine_residual(p->nobs, p->nens, (const float*)r, (const float*)V, ldv, (const float*)D, ldd,
                                   (const float*)Zp, ldzp, P, (float*)Mp, ws + p->off_Msplit, delta, p->ldzw, ctl,
                                   a.timeout_ns, s),
                   "refine residual (exact V^T Z1)");
                if (info)
                    CU(refine_resid_norm(p->nobs, p->nens, delta, p->ldzw, (const float*)r, (const float*)D, ldd,
                                         (double*)(ws + p->off_rnorm), (double*)(ws + p->off_rnorm) + 1024, s),
                       "refine residual norm");
            }
            // Q = V^T U of the final columns (the full Gram where the CUDA-core correction needs
            // its diagonal and lower part too), then P = (I - triu(Q,1)) diag(1/gamma) C
            const bool qfull = !solved_tc5;
            if (qfull)
                CU(gram_full(false, p->nobs, p->nens, V, ldv, a.U, p->ldu, part, p->nsplit, Q, ctl, a.timeout_ns, s),
                   "refine Gram V^T U");
            else
                CU(gram_upper(false, p->nobs, p->nens, V, ldv, a.U, p->ldu, part, p->nsplit, Q, ctl, a.timeout_ns,
                              s),
                   "refine Gram V^T U (upper)");
            if (p_identity) {
                CU(assemble_P(p->nens, Q, a.C, a.gamma, P, s), "refine P");
                // Mp (M's output, written last by refine_apply) holds -P in FP32 until then
                CU(refine_residual(p->nobs, p->nens, (const float*)r, (const float*)V, ldv, (const float*)D, ldd,
                                   (const float*)Zp, ldzp, P, (float*)Mp, ws + p->off_Msplit, delta, p->ldzw, ctl,
                                   a.timeout_ns, s),
                   "refine residual");
            }
            PanelArgs ra = panel_args;
            ra.Z = delta;
            ra.ldz = p->ldzw;
            CU(cudaMemsetAsync(&ctl->barrier, 0, sizeof(unsigned), s), "barrier reset");
            cudaError_t ec = cudaErrorNotSupported;
            double* Cd = (double*)(ws + p->off_Cd);
            if (solved_tc5) {
                ra.C = Cd;
                // the tensor-core solve's own stored factors (final-column pieces, per-panel
                // diag(1/gamma) (I + L)^-1)
                const int k7 = prof_begin(p, 7, s);
                ec = tc5_correct(p->T5, ra, ws + p->off_vpc, ws + p->off_ufc, (const float*)(ws + p->off_wfin), s);
                prof_end(p, k7, s);
                if (ec == cudaErrorNotSupported) (void)cudaGetLastError();
                else CU(ec, "stored-factor correction (tensor cores)");
            }
            if (ec == cudaErrorNotSupported) {
                if (!qfull)
                    CU(gram_full(false, p->nobs, p->nens, V, ldv, a.U, p->ldu, part, p->nsplit, Q, ctl, a.timeout_ns,
                                 s),
                       "refine Gram V^T U");
                ra.Qg = Q;
                ra.refine = 1;
                ra.vec_ok = panel_args.vec_ok && (p->ldzw % 4 == 0);
                const int k7 = prof_begin(p, 7, s);
                CU(panel_launch(p->P, ra, s), "stored-factor correction");
                prof_end(p, k7, s);
            }
            if (ec == cudaSuccess)
                // V^T delta from the correction's own per-level coefficients (the identity above)
                CU(assemble_P(p->nens, Q, Cd, a.gamma, Pd, s), "refine V^T delta");
            else
                CU(gram_full(false, p->nobs, p->nens, V, ldv, delta, p->ldzw, part, p->nsplit, Pd, ctl, a.timeout_ns,
                             s),
                   "refine Gram V^T delta");
            CU(refine_apply(p->nobs, p->nens, (float*)Zp, ldzp, delta, p->ldzw, P, Pd, M64, (float*)Mp, s),
               "refine apply");
            prof_end(p, slot, s);
        }
        if (dXB) {
            slot = prof_begin(p, 4, s);
            if (p->fp64)
                CU(xa_update(true, p->nstate, p->nens, XB, ldb, dXB, ldx, Mp, XA, lda, s), "xa_update launch");
            else
                CU(xa_update_tc05(p->nstate, p->nens, (const float*)XB, ldb, (const float*)dXB, ldx, (const float*)Mp,
                                  ws + p->off_Msplit, (float*)XA, lda, nullptr, p->refine ? 3 : 2, ctl,
                                  a.timeout_ns, s),
                   "xa_update_tc05 launch");
            prof_end(p, slot, s);
        }
    }
    }   // not the small-problem path
    CU(cudaMemcpyAsync(p->h_status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy");
    CU(cudaEventRecord(p->done, s), "cudaEventRecord");
    p->pending = true;

    if (info) {
        CU(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        p->pending = false;
        const int st = *p->h_status;
        *p->h_status = 0;
        memset(info, 0, sizeof(*info));
        info->status = st;
        info->grid_ctas = p->L.grid;
        info->panel_b = p->panel_b;
        double* g = (double*)malloc(sizeof(double) * (size_t)p->nens);
        if (!g) return fail(ENKF_ERR_ARG, "out of host memory");
        cudaError_t e = cudaMemcpy(g, a.gamma, sizeof(double) * (size_t)p->nens, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            free(g);
            return cuda_fail(e, "gamma copy");
        }
        double gmin = INFINITY, gmax = -INFINITY;
        for (int k = 0; k < p->nens; ++k) {
            gmin = fmin(gmin, g[k]);
            gmax = fmax(gmax, g[k]);
        }
        free(g);
        info->gamma_min = gmin;
        info->gamma_max = gmax;
        info->refine_resid = 0.0;
        if (p->refine) {
            e = cudaMemcpy(&info->refine_resid, (double*)(ws + p->off_rnorm) + 1024, sizeof(double),
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "refine residual norm copy");
        }
        {
            Control hc;
            cudaMemcpy(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost);
            if (st == 0 && hc.pad[42] != 0)
                return fail(ENKF_ERR_CUDA, "shared-memory guard bands corrupted: %x, first bad word %08x at %d",
                            hc.pad[42], hc.pad[43], hc.pad[44]);
        }
        if (st != 0) {
            Control hc;
            cudaMemcpy(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost);
            if (hc.pad[0] != 0) {
                char msg[900];
                snprintf(msg, sizeof(msg),
                         "device status %s (level %d; wait site %d, CTA %d, tile %d, parity %d, thread %d, phase %d; "
                         "expired waits per site 1-15: %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d; progress %d %d %d "
                         "%d; as_full %08x %08x as_empty %08x %08x d2_full %08x %08x; waited %08x %08x; guards %x %08x at %d)",
                         enkf_status_string((enkf_status)st), hc.fail_level, hc.pad[0], hc.pad[1], hc.pad[2], hc.pad[3],
                         hc.pad[4], hc.pad[5], hc.pad[11], hc.pad[12], hc.pad[13], hc.pad[14], hc.pad[15], hc.pad[16],
                         hc.pad[17], hc.pad[18], hc.pad[19], hc.pad[20], hc.pad[21], hc.pad[22], hc.pad[23], hc.pad[24],
                         hc.pad[25], hc.pad[30], hc.pad[31], hc.pad[32], hc.pad[33], hc.pad[34], hc.pad[35], hc.pad[36],
                         hc.pad[37], hc.pad[38], hc.pad[39], hc.pad[40], hc.pad[41], hc.pad[42], hc.pad[43], hc.pad[44]);
                return fail((enkf_status)st, "%s", msg);
            }
            return fail((enkf_status)st, "device status %s (level %d)", enkf_status_string((enkf_status)st),
                        hc.fail_level);
        }
    }
    return ENKF_OK;
}

enkf_status enkf_forecast_workspace(int64_t nstate, int32_t nens, int32_t method, size_t* bytes) {
    if (!bytes) return fail(ENKF_ERR_ARG, "enkf_forecast_workspace: NULL bytes");
    if (nstate < 1 || nens < 1) return fail(ENKF_ERR_SHAPE, "enkf_forecast_workspace: bad sizes");
    if (method == ENKF_FORECAST_RK4) {
        *bytes = 0;
        return ENKF_OK;
    }
    if (method == ENKF_FORECAST_SURROGATE) {
        *bytes = surrogate_forecast_ws(nstate, nens);
        return ENKF_OK;
    }
    return fail(ENKF_ERR_UNSUPPORTED, "enkf_forecast_workspace: method %d not built", method);
}

enkf_status enkf_forecast(void* X, int64_t ld, int64_t nstate, int32_t nens, int32_t precision, double F, double dt,
                          int32_t nsteps, int32_t method, const void* weights, void* workspace,
                          size_t workspace_bytes, void* stream) {
    (void)weights;
    (void)workspace;
    (void)workspace_bytes;
    if (!X) return fail(ENKF_ERR_ARG, "enkf_forecast: NULL X");
    if (precision != ENKF_FP64 && precision != ENKF_FP32) return fail(ENKF_ERR_ARG, "enkf_forecast: bad precision");
    if (nstate < 4 || nens < 1 || ld < nstate || nsteps < 0)
        return fail(ENKF_ERR_SHAPE, "enkf_forecast: need nstate >= 4, nens >= 1, ld >= nstate, nsteps >= 0");
    const bool fp64 = precision == ENKF_FP64;
    if ((uintptr_t)X % (fp64 ? 8 : 4)) return fail(ENKF_ERR_ARG, "enkf_forecast: X misaligned");
    if (method == ENKF_FORECAST_RK4) {
        if (nstate > (fp64 ? 6144 : 12288)) return fail(ENKF_ERR_SHAPE, "enkf_forecast: nstate too large for RK4");
        if (nsteps == 0) return ENKF_OK;
        CU(l96_rk4(fp64, X, ld, nstate, nens, F, dt, nsteps, (cudaStream_t)stream), "l96_rk4 launch");
        return ENKF_OK;
    }
    if (method == ENKF_FORECAST_SURROGATE) {
        if (fp64) return fail(ENKF_ERR_UNSUPPORTED, "enkf_forecast: the surrogate runs on FP32 states");
        if (!weights) return fail(ENKF_ERR_ARG, "enkf_forecast: NULL surrogate weights");
        if (nstate < 5 || nstate > (1 << 28)) return fail(ENKF_ERR_SHAPE, "enkf_forecast: surrogate needs nstate >= 5");
        const size_t need = surrogate_forecast_ws(nstate, nens);
        if (!workspace || workspace_bytes < need || (uintptr_t)workspace % 256)
            return fail(ENKF_ERR_WORKSPACE, "enkf_forecast: surrogate workspace %zu < %zu bytes (or misaligned)",
                        workspace_bytes, need);
        if ((uintptr_t)weights % 256) return fail(ENKF_ERR_ARG, "enkf_forecast: weights not 256-byte aligned");
        CU(surrogate_forecast((float*)X, ld, nstate, nens, nsteps, weights, workspace, (cudaStream_t)stream),
           "surrogate forecast");
        return ENKF_OK;
    }
    return fail(ENKF_ERR_UNSUPPORTED, "enkf_forecast: method %d not built", method);
}

enkf_status enkf_surrogate_sizes(int64_t nstate, int32_t nbatch, int64_t* n_params, size_t* packed_bytes,
                                 size_t* train_workspace_bytes) {
    if (nstate < 5 || nbatch < 1) return fail(ENKF_ERR_SHAPE, "enkf_surrogate_sizes: need nstate >= 5, nbatch >= 1");
    if (n_params) *n_params = surrogate_n_params();
    if (packed_bytes) *packed_bytes = surrogate_packed_bytes();
    if (train_workspace_bytes) *train_workspace_bytes = surrogate_train_ws(nstate, nbatch);
    return ENKF_OK;
}

enkf_status enkf_surrogate_pack(const float* master, void* packed, void* stream) {
    if (!master || !packed) return fail(ENKF_ERR_ARG, "enkf_surrogate_pack: NULL argument");
    if ((uintptr_t)packed % 256) return fail(ENKF_ERR_ARG, "enkf_surrogate_pack: packed not 256-byte aligned");
    CU(surrogate_pack(master, packed, (cudaStream_t)stream), "surrogate pack");
    return ENKF_OK;
}

enkf_status enkf_surrogate_train_step(float* master, float* adam_m, float* adam_v, int32_t step, float lr,
                                      void* packed, const float* X, const float* target, int64_t nstate,
                                      int32_t nbatch, void* workspace, size_t workspace_bytes, float* sq_err,
                                      float* grad, void* stream) {
    if (!master || !packed || !X || !target || !sq_err || (step > 0 && (!adam_m || !adam_v)))
        return fail(ENKF_ERR_ARG, "enkf_surrogate_train_step: NULL argument");
    if (nstate < 5 || nbatch < 1 || (int64_t)nstate * nbatch > ((int64_t)1 << 31))
        return fail(ENKF_ERR_SHAPE, "enkf_surrogate_train_step: bad sizes");
    const size_t need = surrogate_train_ws(nstate, nbatch);
    if (!workspace || workspace_bytes < need || (uintptr_t)workspace % 256)
        return fail(ENKF_ERR_WORKSPACE, "enkf_surrogate_train_step: workspace %zu < %zu bytes", workspace_bytes, need);
    CU(surrogate_train_step(master, adam_m, adam_v, step, lr, packed, X, target, nstate, nbatch, workspace, sq_err,
                            grad, (cudaStream_t)stream),
       "surrogate train step");
    return ENKF_OK;
}

}  // extern "C"
