// C ABI of the batched analyses (declared in include/enkf_ism.h): plan (validation,
// longest-first order, workspace layout, size classes), autotuner of the panel
// width per size class with a persisted cache, and the CUDA-graph launch.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/enkf_ism.h"
#include "internal.h"

using namespace enkf;

namespace {

enkf_status bfail(enkf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

enkf_status bcuda(cudaError_t e, const char* what) {
    return bfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define BCU(call, what)                                     \
    do {                                                    \
        cudaError_t e__ = (call);                           \
        if (e__ != cudaSuccess) return bcuda(e__, what);   \
    } while (0)

constexpr int kClasses = 16;
constexpr int kWidths[4] = {1, 8, 16, 32};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int size_class(int64_t nobs, int32_t nens) {
    int ec = (nens + 31) / 32 - 1;
    ec = ec < 0 ? 0 : (ec > 3 ? 3 : ec);
    const int oc = nobs < 64 ? 0 : nobs < 256 ? 1 : nobs < 1024 ? 2 : 3;
    return ec * 4 + oc;
}

std::string gpu_key() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string name(prop.name);
    for (auto& c : name)
        if (c == ' ' || c == '\t') c = '_';
    char buf[64];
    snprintf(buf, sizeof(buf), "_sm%d%d", prop.major, prop.minor);
    return name + buf;
}

// Cache file: one line per entry "<gpu_key> <class> <b>"; later lines win.
void load_cache(const char* path, const std::string& key, int* widths, bool* found) {
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return;
    char k[256];
    int c, b;
    while (fscanf(f, "%255s %d %d", k, &c, &b) == 3) {
        if (key == k && c >= 0 && c < kClasses && (b == 1 || b == 8 || b == 16 || b == 32)) {
            widths[c] = b;
            found[c] = true;
        }
    }
    fclose(f);
}

}  // namespace

struct enkf_ism_batch_plan_s {
    int32_t nprob;
    int device;
    uint32_t flags;
    int grid;
    std::vector<BatchDesc> desc;
    std::vector<int> order;            // longest first
    std::vector<int> cls;              // size class per problem
    std::vector<int> by_class;         // problem ids grouped by class (for tuning)
    int class_begin[kClasses + 1];
    int widths[kClasses];
    size_t off_ctl, off_desc, off_order, off_class, off_iter, total;
    BatchDesc* h_desc;                 // pinned host copies for the uploads
    int* h_order;
    int* h_status;
    // captured graph
    cudaStream_t cap;
    cudaGraphExec_t exec;
    bool have_exec;
    const void* g_in;
    void* g_out;
    void* g_ws;
};

extern "C" {

enkf_status enkf_ism_batch_plan(enkf_ism_batch_plan_t* out, int32_t nprob, const enkf_ism_problem* problems,
                                int32_t mode, uint32_t flags, size_t* workspace_bytes) {
    if (!out || !workspace_bytes || (!problems && nprob > 0)) return bfail(ENKF_ERR_ARG, "enkf_ism_batch_plan: NULL");
    *out = nullptr;
    if (nprob < 0) return bfail(ENKF_ERR_SHAPE, "enkf_ism_batch_plan: nprob < 0");
    if (mode != ENKF_FP32) return bfail(ENKF_ERR_UNSUPPORTED, "enkf_ism_batch_plan: only ENKF_FP32 is built");
    if (flags & ~(uint32_t)ENKF_FLAG_NO_CHECKS) return bfail(ENKF_ERR_ARG, "enkf_ism_batch_plan: unknown flags");
    for (int32_t i = 0; i < nprob; ++i) {
        const enkf_ism_problem& p = problems[i];
        if (p.nobs < 1 || p.nobs > (1 << 30) || p.nens < 4 || p.nens > 128 || p.nens % 4 != 0)
            return bfail(ENKF_ERR_SHAPE, "problem %d: need nobs >= 1 and 4 <= nens <= 128, nens %% 4 == 0", i);
        if (p.ldv < p.nobs || p.ldd < p.nobs || (p.Z >= 0 && p.ldz < p.nobs))
            return bfail(ENKF_ERR_SHAPE, "problem %d: leading dimension smaller than nobs", i);
        if (p.r < 0 || p.V < 0 || p.D < 0) return bfail(ENKF_ERR_ARG, "problem %d: negative input offset", i);
    }
    enkf_ism_batch_plan_s* pl = new (std::nothrow) enkf_ism_batch_plan_s();
    if (!pl) return bfail(ENKF_ERR_ARG, "out of host memory");
    pl->nprob = nprob;
    pl->flags = flags;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e == cudaSuccess) e = batch_configure(&pl->grid);
    if (e != cudaSuccess) {
        delete pl;
        return bcuda(e, "enkf_ism_batch_plan: configure");
    }
    // default widths, then the autotune cache
    for (int c = 0; c < kClasses; ++c) pl->widths[c] = 16;
    bool found[kClasses] = {};
    load_cache(getenv("ENKF_AUTOTUNE_CACHE"), gpu_key(), pl->widths, found);

    pl->desc.resize(nprob);
    pl->cls.resize(nprob);
    size_t ws_floats = 0;
    std::vector<double> cost(nprob);
    for (int32_t i = 0; i < nprob; ++i) {
        const enkf_ism_problem& p = problems[i];
        BatchDesc& d = pl->desc[i];
        d.nobs = (int32_t)p.nobs;
        d.nens = p.nens;
        d.ldX = 2 * p.nens;
        d.ldVr = p.nens;
        d.pad = 0;
        d.r = p.r;
        d.V = p.V;
        d.D = p.D;
        d.Z = p.Z;
        d.M = p.M;
        d.ldv = p.ldv;
        d.ldd = p.ldd;
        d.ldz = p.ldz;
        d.X = (int64_t)ws_floats;
        ws_floats += ((size_t)p.nobs * d.ldX + 63) / 64 * 64;
        d.Vr = (int64_t)ws_floats;
        ws_floats += ((size_t)p.nobs * d.ldVr + 63) / 64 * 64;
        d.Ch = (int64_t)ws_floats;
        ws_floats += ((size_t)p.nens * p.nens + 63) / 64 * 64;
        d.Qw = (int64_t)ws_floats;
        ws_floats += ((size_t)p.nens * p.nens + 63) / 64 * 64;
        pl->cls[i] = size_class(p.nobs, p.nens);
        d.b = pl->widths[pl->cls[i]];
        cost[i] = (double)p.nobs * p.nens * p.nens + 64.0 * p.nens * p.nens;
    }
    pl->order.resize(nprob);
    std::iota(pl->order.begin(), pl->order.end(), 0);
    std::stable_sort(pl->order.begin(), pl->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // problems grouped by class (each group longest first)
    pl->by_class.clear();
    for (int c = 0; c < kClasses; ++c) {
        pl->class_begin[c] = (int)pl->by_class.size();
        for (int i : pl->order)
            if (pl->cls[i] == c) pl->by_class.push_back(i);
    }
    pl->class_begin[kClasses] = (int)pl->by_class.size();

    size_t o = 0;
    pl->off_ctl = o; o = al256(o + sizeof(Control));
    pl->off_desc = o; o = al256(o + sizeof(BatchDesc) * (size_t)(nprob > 0 ? nprob : 1));
    pl->off_order = o; o = al256(o + sizeof(int) * (size_t)(nprob > 0 ? nprob : 1));
    pl->off_class = o; o = al256(o + sizeof(int) * (size_t)(nprob > 0 ? nprob : 1));
    pl->off_iter = o; o = al256(o + sizeof(float) * ws_floats);
    pl->total = o;

    e = cudaMallocHost(&pl->h_desc, sizeof(BatchDesc) * (size_t)(nprob > 0 ? nprob : 1));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_order, sizeof(int) * 2 * (size_t)(nprob > 0 ? nprob : 1));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_status, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (pl->h_desc) cudaFreeHost(pl->h_desc);
        if (pl->h_order) cudaFreeHost(pl->h_order);
        if (pl->h_status) cudaFreeHost(pl->h_status);
        delete pl;
        return bcuda(e, "enkf_ism_batch_plan: host buffers");
    }
    pl->have_exec = false;
    *workspace_bytes = pl->total;
    *out = pl;
    return ENKF_OK;
}

void enkf_ism_batch_plan_destroy(enkf_ism_batch_plan_t pl) {
    if (!pl) return;
    cudaStreamSynchronize(pl->cap);
    if (pl->have_exec) cudaGraphExecDestroy(pl->exec);
    cudaStreamDestroy(pl->cap);
    cudaFreeHost(pl->h_desc);
    cudaFreeHost(pl->h_order);
    cudaFreeHost(pl->h_status);
    delete pl;
}

static enkf_status batch_check_ws(enkf_ism_batch_plan_t pl, const void* in, void* outp, void* ws, size_t bytes) {
    if (!pl) return bfail(ENKF_ERR_ARG, "NULL batch plan");
    if (!in || !outp) return bfail(ENKF_ERR_ARG, "NULL base_in or base_out");
    if (!ws || bytes < pl->total || (uintptr_t)ws % 256)
        return bfail(ENKF_ERR_WORKSPACE, "batch workspace %zu bytes < required %zu (or not 256-aligned)", bytes,
                     pl->total);
    if (((uintptr_t)in | (uintptr_t)outp) & 3) return bfail(ENKF_ERR_ARG, "base pointers not float-aligned");
    return ENKF_OK;
}

// Uploads the descriptors (with the current widths) and the order list.
static enkf_status batch_upload(enkf_ism_batch_plan_t pl, void* ws, cudaStream_t s) {
    char* w = (char*)ws;
    for (int i = 0; i < pl->nprob; ++i) {
        pl->h_desc[i] = pl->desc[i];
        pl->h_desc[i].b = pl->widths[pl->cls[i]];
    }
    for (int i = 0; i < pl->nprob; ++i) pl->h_order[i] = pl->order[i];
    for (int i = 0; i < pl->nprob; ++i) pl->h_order[pl->nprob + i] = pl->by_class[i];
    if (pl->nprob > 0) {
        BCU(cudaMemcpyAsync(w + pl->off_desc, pl->h_desc, sizeof(BatchDesc) * pl->nprob, cudaMemcpyHostToDevice, s),
            "descriptor upload");
        BCU(cudaMemcpyAsync(w + pl->off_order, pl->h_order, sizeof(int) * pl->nprob, cudaMemcpyHostToDevice, s),
            "order upload");
        BCU(cudaMemcpyAsync(w + pl->off_class, pl->h_order + pl->nprob, sizeof(int) * pl->nprob,
                            cudaMemcpyHostToDevice, s),
            "class order upload");
    }
    // the pinned buffers are reused by later uploads: finish this one first
    BCU(cudaStreamSynchronize(s), "upload sync");
    return ENKF_OK;
}

enkf_status enkf_ism_batch_autotune(enkf_ism_batch_plan_t pl, const void* base_in, void* base_out, void* workspace,
                                    size_t workspace_bytes, void* stream, const char* cache_path, int32_t* widths) {
    enkf_status st = batch_check_ws(pl, base_in, base_out, workspace, workspace_bytes);
    if (st != ENKF_OK) return st;
    BCU(cudaSetDevice(pl->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)workspace;
    st = batch_upload(pl, workspace, s);
    if (st != ENKF_OK) return st;
    Control* ctl = (Control*)(w + pl->off_ctl);
    const BatchDesc* d_desc = (const BatchDesc*)(w + pl->off_desc);
    const int* d_class = (const int*)(w + pl->off_class);
    float* iter = (float*)(w + pl->off_iter);
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0), "cudaEventCreate");
    BCU(cudaEventCreate(&e1), "cudaEventCreate");
    const int check = (pl->flags & ENKF_FLAG_NO_CHECKS) ? 0 : 1;
    for (int c = 0; c < kClasses; ++c) {
        const int beg = pl->class_begin[c], cnt = pl->class_begin[c + 1] - beg;
        if (cnt == 0) continue;
        float best = 1e30f;
        int best_b = pl->widths[c];
        for (int wi = 0; wi < 4; ++wi) {
            const int b = kWidths[wi];
            float ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                BCU(cudaMemsetAsync(ctl, 0, sizeof(Control), s), "memset");
                BCU(cudaEventRecord(e0, s), "event");
                BCU(batch_launch(pl->grid, d_desc, d_class + beg, cnt, (const float*)base_in, (float*)base_out, iter,
                                 ctl, check, b, s),
                    "batch launch (tune)");
                BCU(cudaEventRecord(e1, s), "event");
                BCU(cudaEventSynchronize(e1), "event sync");
                float t = 0.f;
                BCU(cudaEventElapsedTime(&t, e0, e1), "elapsed");
                if (rep > 0) ms += t;   // first run warms up
            }
            if (ms < best) {
                best = ms;
                best_b = b;
            }
        }
        pl->widths[c] = best_b;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (widths)
        for (int c = 0; c < kClasses; ++c) widths[c] = pl->widths[c];
    for (int i = 0; i < pl->nprob; ++i) pl->desc[i].b = pl->widths[pl->cls[i]];
    if (pl->have_exec) {   // descriptors changed: recapture on the next run
        cudaGraphExecDestroy(pl->exec);
        pl->have_exec = false;
    }
    const char* path = cache_path ? cache_path : getenv("ENKF_AUTOTUNE_CACHE");
    if (path) {
        FILE* f = fopen(path, "a");
        if (!f) return bfail(ENKF_ERR_ARG, "cannot open autotune cache %s", path);
        const std::string key = gpu_key();
        for (int c = 0; c < kClasses; ++c)
            if (pl->class_begin[c + 1] > pl->class_begin[c]) fprintf(f, "%s %d %d\n", key.c_str(), c, pl->widths[c]);
        fclose(f);
    }
    return ENKF_OK;
}

enkf_status enkf_ism_batch(enkf_ism_batch_plan_t pl, const void* base_in, void* base_out, void* workspace,
                           size_t workspace_bytes, void* stream, int32_t* status) {
    enkf_status st = batch_check_ws(pl, base_in, base_out, workspace, workspace_bytes);
    if (st != ENKF_OK) return st;
    BCU(cudaSetDevice(pl->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)workspace;
    Control* ctl = (Control*)(w + pl->off_ctl);
    if (!pl->have_exec || pl->g_in != base_in || pl->g_out != base_out || pl->g_ws != workspace) {
        if (pl->have_exec) {
            cudaGraphExecDestroy(pl->exec);
            pl->have_exec = false;
        }
        st = batch_upload(pl, workspace, s);
        if (st != ENKF_OK) return st;
        const int check = (pl->flags & ENKF_FLAG_NO_CHECKS) ? 0 : 1;
        cudaGraph_t g;
        BCU(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e1 = cudaMemsetAsync(ctl, 0, sizeof(Control), pl->cap);
        cudaError_t e2 = batch_launch(pl->grid, (const BatchDesc*)(w + pl->off_desc), (const int*)(w + pl->off_order),
                                      pl->nprob, (const float*)base_in, (float*)base_out, (float*)(w + pl->off_iter),
                                      ctl, check, 0, pl->cap);
        cudaError_t e3 = cudaStreamEndCapture(pl->cap, &g);
        if (e1 != cudaSuccess) return bcuda(e1, "capture memset");
        if (e2 != cudaSuccess) return bcuda(e2, "capture launch");
        if (e3 != cudaSuccess) return bcuda(e3, "end capture");
        cudaError_t e4 = cudaGraphInstantiate(&pl->exec, g, 0);
        cudaGraphDestroy(g);
        if (e4 != cudaSuccess) return bcuda(e4, "graph instantiate");
        pl->have_exec = true;
        pl->g_in = base_in;
        pl->g_out = base_out;
        pl->g_ws = workspace;
    }
    BCU(cudaGraphLaunch(pl->exec, s), "graph launch");
    if (status) {
        BCU(cudaMemcpyAsync(pl->h_status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy");
        BCU(cudaStreamSynchronize(s), "sync");
        *status = *pl->h_status;
        if (*status != 0) return bfail((enkf_status)*status, "batch device status %d", *status);
    }
    return ENKF_OK;
}

}  // extern "C"
