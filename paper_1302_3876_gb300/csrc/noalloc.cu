// enkf_ism_solve_noalloc: the solve of enkf_ism_analysis for callers that cannot
// allocate device memory.
//
// Who needs this: code that runs inside a host application which already owns
// the device memory -- a plugin whose host reserved the whole GPU through its own
// pool allocator, or a process whose device-memory budget is fixed when it
// starts.  There cudaMalloc either fails or bypasses the host's accounting, so
// such a caller cannot create the workspace that enkf_ism_analysis needs.
//
// This entry point needs no workspace: its scratch (the control block, U, the
// per-CTA partial dots, the reduced coefficients, gamma) lives in one
// file-scope __device__ array of ENKF_NOALLOC_SCRATCH_BYTES.  Every GPU that loads
// the library holds that array until the process exits.  The call allocates
// nothing (no cudaMalloc, cudaFree or allocating library routine) and launches the
// same level-streaming kernel as enkf_ism_analysis.
//
// The host cannot use the array's name as a device address (in host code it names
// a host-side stand-in).  The first call on each device, with that device
// current, asks the runtime for the array's device address with
// cudaGetSymbolAddress and caches it per device; make that first call before any
// stream capture.  All calls share the one array, which keeps the last call's
// contents: the control block is cleared on every call, and calls that overlap on
// the GPU (two streams, or two host threads, at once) race on the scratch.  Device-
// side errors reach the caller only through the optional status word (which makes
// the call synchronous); with status NULL they are dropped, not latched.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "../../include/enkf_ism.h"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = ENKF_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

enkf_status nfail(enkf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    enkf::set_last_error(buf);
    return s;
}

enkf_status ncuda(cudaError_t e, const char* what) {
    return nfail(ENKF_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Device address of the scratch array on the current device (set up once per device).
enkf_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nfail(ENKF_ERR_UNSUPPORTED, "enkf_ism_solve_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ENKF_OK;
}

}  // namespace

extern "C" enkf_status enkf_ism_solve_noalloc(int64_t nobs, int32_t nens, int32_t precision, const void* r,
                                              const void* V, int64_t ldv, const void* D, int64_t ldd, void* Z,
                                              int64_t ldz, void* stream, int32_t* status) {
    using namespace enkf;
    if (!r || !V || !D || !Z) return nfail(ENKF_ERR_ARG, "enkf_ism_solve_noalloc: NULL r, V, D or Z");
    if (precision != ENKF_FP64 && precision != ENKF_FP32)
        return nfail(ENKF_ERR_ARG, "enkf_ism_solve_noalloc: precision must be ENKF_FP64 or ENKF_FP32");
    if (nobs < 1 || nens < 1 || nens > 1024)
        return nfail(ENKF_ERR_SHAPE, "enkf_ism_solve_noalloc: need nobs >= 1 and 1 <= nens <= 1024");
    if (ldv < nobs || ldd < nobs || ldz < nobs)
        return nfail(ENKF_ERR_SHAPE, "enkf_ism_solve_noalloc: ldv/ldd/ldz smaller than nobs");
    const bool fp64 = precision == ENKF_FP64;
    const size_t w = fp64 ? 8 : 4;
    if (((uintptr_t)r | (uintptr_t)V | (uintptr_t)D | (uintptr_t)Z) & (w - 1))
        return nfail(ENKF_ERR_ARG, "enkf_ism_solve_noalloc: pointer not aligned to the element size");

    LevelLaunch L;
    cudaError_t e = level_plan(fp64, nobs, nens, &L);
    if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: launch shape");
    const int64_t ldu = (nobs + 31) / 32 * 32;
    const size_t N = (size_t)nens;
    const size_t off_U = al256(sizeof(Control));
    const size_t off_part = al256(off_U + w * (size_t)ldu * N);
    const size_t off_coefg = al256(off_part + sizeof(double) * (size_t)L.grid * 2 * N);
    const size_t off_C = al256(off_coefg + sizeof(double) * 2 * N);
    const size_t off_gamma = al256(off_C + sizeof(double) * N * N);
    const size_t need = al256(off_gamma + sizeof(double) * N);
    if (need > kScratchBytes)
        return nfail(ENKF_ERR_WORKSPACE,
                     "enkf_ism_solve_noalloc: nobs=%lld, nens=%d needs %zu bytes of scratch, more than the "
                     "%zu-byte static array; use enkf_ism_analysis with a workspace",
                     (long long)nobs, nens, need, kScratchBytes);

    void* base = nullptr;
    enkf_status st = scratch_address(&base);
    if (st != ENKF_OK) return st;
    char* sc = static_cast<char*>(base);
    cudaStream_t s = (cudaStream_t)stream;
    Control* ctl = reinterpret_cast<Control*>(sc);
    e = cudaMemsetAsync(ctl, 0, sizeof(Control), s);
    if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: clearing the control block");

    LevelArgs a;
    a.nobs = nobs;
    a.nens = nens;
    a.r = r;
    a.V = V;
    a.ldv = ldv;
    a.D = D;
    a.ldd = ldd;
    a.U = sc + off_U;
    a.ldu = ldu;
    a.Z = Z;
    a.ldz = ldz;
    a.part = reinterpret_cast<double*>(sc + off_part);
    a.coefg = reinterpret_cast<double*>(sc + off_coefg);
    a.C = reinterpret_cast<double*>(sc + off_C);
    a.gamma = reinterpret_cast<double*>(sc + off_gamma);
    a.ctl = ctl;
    a.rows_per_blk = L.rows_per_blk;
    a.rows_chunk = L.rows_chunk;
    a.check = 1;
    a.test_skip_arrival = 0;
    a.timeout_ns = 2000000000ull;
    e = level_launch(fp64, L, a, s);
    if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: level-streaming launch");
    if (status) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: cudaStreamSynchronize");
        int dst = 0;
        e = cudaMemcpy(&dst, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return ncuda(e, "enkf_ism_solve_noalloc: status read");
        *status = dst;
        if (dst != 0) return nfail((enkf_status)dst, "enkf_ism_solve_noalloc: device status %d", dst);
    }
    return ENKF_OK;
}
