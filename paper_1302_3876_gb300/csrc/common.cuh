// Device-side helpers shared by the kernels of libenkf_ism: status codes, the
// bounded grid barrier used by the persistent level-streaming kernel, and small
// reductions.  No arithmetic of the filter lives here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace enkf {

// Device status codes (same values as enkf_status in include/enkf_ism.h).
enum : int {
    kOk = 0,
    kErrNumeric = 4,
    kErrTimeout = 5,
};

// Workspace control block (first 256 bytes of every workspace).
struct Control {
    int status;          // latched device status (0 = ok)
    unsigned barrier;    // monotonically increasing arrival counter of the grid barrier
    int fail_level;      // level at which a numeric check failed (diagnostic)
    int pad[61];
};
static_assert(sizeof(Control) == 256, "control block is 256 bytes");

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_s32(const int* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(Control* ctl, int code) {
    atomicCAS(&ctl->status, 0, code);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Thread 0
// of each CTA arrives on a monotonically increasing counter and spins, with both
// an iteration limit and a wall-clock limit, until every CTA of the current
// epoch has arrived.  On expiry it latches kErrTimeout.  Returns true when the
// grid may proceed (no timeout, no latched error).  Must be called by every
// thread of the CTA.
__device__ __forceinline__ bool grid_barrier(Control* ctl, unsigned nblocks, unsigned& epoch,
                                             uint64_t timeout_ns, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        ++epoch;
        __threadfence();
        atomicAdd(&ctl->barrier, 1u);
        const unsigned target = epoch * nblocks;
        const uint64_t t0 = global_timer_ns();
        unsigned it = 0;
        while (ld_volatile_u32(&ctl->barrier) < target) {
            __nanosleep(32);
            if ((++it & 63u) == 0) {
                if (global_timer_ns() - t0 > timeout_ns || it > (1u << 27)) {
                    set_status(ctl, kErrTimeout);
                    ok = 0;
                    break;
                }
                if (ld_volatile_s32(&ctl->status) == kErrTimeout) { ok = 0; break; }
            }
        }
        __threadfence();
        if (ok && ld_volatile_s32(&ctl->status) != 0) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, then a fixed pass over warps).
// scratch must hold blockDim.x / 32 doubles.  Result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += scratch[w];
    return s;
}

}  // namespace enkf
