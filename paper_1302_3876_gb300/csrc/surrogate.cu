// Learned forecast surrogate for the Lorenz-96 ensemble (replaces the model
// propagation of the forecast step, eq. forecast-step, between analyses):
//   x_next = x + s_out * f(x),  f = 4 periodic 1-D convolutions over the state index
//   (channels 1 -> 64 -> 64 -> 64 -> 1, kernel 5, circular padding 2, GELU-tanh between).
//
// Storage: activations channels-last in BF16, act[m][p][c] (64 channels = 128 bytes
// per position); master parameters FP32 in the flat order W1 (64,1,5), b1, W2
// (64,64,5), b2, W3, b3, W4 (1,64,5), b4; the packed inference copy holds
//   W1 [o][t] f32, b1, W2 [o][t][i] bf16, b2, W3 [o][t][i] bf16, b3, W4 [t][i] f32, b4,
//   WT2 / WT3 [i][t][o] bf16 with WT[i][t][o] = W[o][i][4-t]   (backward data).
//
// The 64 -> 64 convolutions are implicit GEMMs on BF16 tensor cores (mma.sync
// m16n8k16, FP32 accumulation): a CTA computes 128 positions x 64 channels with
// K = 5 taps x 64 channels staged in shared memory.  The same kernel with the
// transposed, tap-flipped weights gives the data gradient (epilogue: times
// gelu'(pre-activation)).  Layers 1 and 4, weight gradients (per-CTA partials
// reduced in a fixed order) and Adam run on FP32 CUDA cores.
#include <cuda_bf16.h>
#include <math.h>

#include "internal.h"

namespace enkf {
namespace {

constexpr int CH = 64;
constexpr int KT = 5;
constexpr float SHIFT = 2.5f, SCALE_IN = 0.25f, SCALE_OUT = 1.0f;
constexpr float GELU_C = 0.7978845608028654f, GELU_A = 0.044715f;

__device__ __forceinline__ float gelu(float u) {
    return 0.5f * u * (1.f + tanhf(GELU_C * (u + GELU_A * u * u * u)));
}
__device__ __forceinline__ float gelu_grad(float u) {
    const float k = GELU_C * (u + GELU_A * u * u * u);
    const float th = tanhf(k);
    return 0.5f * (1.f + th) + 0.5f * u * (1.f - th * th) * GELU_C * (1.f + 3.f * GELU_A * u * u);
}

__device__ __forceinline__ int wrap(int p, int P) { return p < 0 ? p + P : (p >= P ? p - P : p); }

// ---------------------------------------------------------------------------
// layer 1: z0 = (x - shift) scale_in; y1 = conv(z0) + b1; a1 = gelu(y1)
// ---------------------------------------------------------------------------
__global__ void l1_fwd_kernel(const float* __restrict__ X, int64_t ldx, int P, int nm, const SurrogatePacked w,
                              __nv_bfloat16* __restrict__ y1, __nv_bfloat16* __restrict__ a1) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nm * P) return;
    const int m = (int)(idx / P), p = (int)(idx % P);
    const float* x = X + (int64_t)m * ldx;
    float z[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) z[t] = (x[wrap(p + t - 2, P)] - SHIFT) * SCALE_IN;
    __align__(16) __nv_bfloat16 yo[CH], ao[CH];
#pragma unroll 8
    for (int o = 0; o < CH; ++o) {
        float v = w.b1[o];
#pragma unroll
        for (int t = 0; t < KT; ++t) v = fmaf(w.W1[o * KT + t], z[t], v);
        yo[o] = __float2bfloat16(v);
        ao[o] = __float2bfloat16(gelu(v));
    }
    uint4* da = reinterpret_cast<uint4*>(a1 + idx * CH);
#pragma unroll
    for (int q = 0; q < CH / 8; ++q) da[q] = reinterpret_cast<const uint4*>(ao)[q];
    if (y1) {
        uint4* dy = reinterpret_cast<uint4*>(y1 + idx * CH);
#pragma unroll
        for (int q = 0; q < CH / 8; ++q) dy[q] = reinterpret_cast<const uint4*>(yo)[q];
    }
}

// ---------------------------------------------------------------------------
// 64 -> 64 convolution on tensor cores.  MODE 0: forward, out_y = pre-activation
// (nullable), out_a = gelu.  MODE 1: data gradient, out_a = acc * gelu'(yprev).
// Weights Wk[o][t][i] (bf16, K index = t*64 + i).
// ---------------------------------------------------------------------------
constexpr int TP = 128;            // positions per CTA
constexpr int IN_LD = CH + 8;      // padded smem row (bf16)
constexpr int W_LD = KT * CH + 8;

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int MODE>
__global__ void __launch_bounds__(256) conv64_kernel(const __nv_bfloat16* __restrict__ in, int P, int nm,
                                                     const __nv_bfloat16* __restrict__ Wk,
                                                     const float* __restrict__ bias,
                                                     const __nv_bfloat16* __restrict__ yprev,
                                                     __nv_bfloat16* __restrict__ out_y,
                                                     __nv_bfloat16* __restrict__ out_a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* Ins = reinterpret_cast<__nv_bfloat16*>(smem_raw);      // [TP + 4][IN_LD]
    __nv_bfloat16* Ws = Ins + (TP + 4) * IN_LD;                          // [64][W_LD]
    const int tiles_per_member = (P + TP - 1) / TP;
    const int m = blockIdx.x / tiles_per_member;
    const int p0 = (blockIdx.x % tiles_per_member) * TP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const __nv_bfloat16* src = in + (int64_t)m * P * CH;
    // stage input rows p0-2 .. p0+TP+1 (periodic) and the weights, 16-byte vectors
    for (int e = tid; e < (TP + 4) * (CH / 8); e += 256) {
        const int r = e / (CH / 8), q = e % (CH / 8);
        const int p = wrap(((p0 - 2 + r) % P + P) % P, P);
        *reinterpret_cast<uint4*>(Ins + r * IN_LD + q * 8) =
            *reinterpret_cast<const uint4*>(src + (int64_t)p * CH + q * 8);
    }
    for (int e = tid; e < CH * (KT * CH / 8); e += 256) {
        const int o = e / (KT * CH / 8), q = e % (KT * CH / 8);
        *reinterpret_cast<uint4*>(Ws + o * W_LD + q * 8) = *reinterpret_cast<const uint4*>(Wk + o * KT * CH + q * 8);
    }
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
    const int r0 = warp * 16 + (lane >> 2);      // tile row of a0/a1 (before the tap offset)
    const int kq = (lane & 3) * 2;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
#pragma unroll
        for (int kc = 0; kc < CH / 16; ++kc) {
            uint32_t a[4];
            const __nv_bfloat16* ar = Ins + (r0 + t) * IN_LD + kc * 16 + kq;
            a[0] = *reinterpret_cast<const uint32_t*>(ar);
            a[1] = *reinterpret_cast<const uint32_t*>(ar + 8 * IN_LD);
            a[2] = *reinterpret_cast<const uint32_t*>(ar + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(ar + 8 * IN_LD + 8);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const __nv_bfloat16* br = Ws + (n * 8 + (lane >> 2)) * W_LD + t * CH + kc * 16 + kq;
                uint32_t b[2];
                b[0] = *reinterpret_cast<const uint32_t*>(br);
                b[1] = *reinterpret_cast<const uint32_t*>(br + 8);
                mma_bf16(acc[n], a, b);
            }
        }
    }
    // epilogue: rows r0 and r0 + 8, columns n*8 + kq, +1
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = p0 + r0 + 8 * h;
        if (p >= P) continue;
        const int64_t base = ((int64_t)m * P + p) * CH;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int o = n * 8 + kq;
            float v0 = acc[n][2 * h], v1 = acc[n][2 * h + 1];
            if (MODE == 0) {
                v0 += bias[o];
                v1 += bias[o + 1];
                if (out_y) *reinterpret_cast<__nv_bfloat162*>(out_y + base + o) = __floats2bfloat162_rn(v0, v1);
                *reinterpret_cast<__nv_bfloat162*>(out_a + base + o) = __floats2bfloat162_rn(gelu(v0), gelu(v1));
            } else {
                const __nv_bfloat162 yp = *reinterpret_cast<const __nv_bfloat162*>(yprev + base + o);
                v0 *= gelu_grad(__bfloat162float(yp.x));
                v1 *= gelu_grad(__bfloat162float(yp.y));
                *reinterpret_cast<__nv_bfloat162*>(out_a + base + o) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// layer 4: out = x + s_out (b4 + sum_t sum_i W4[t][i] a3[p+t-2][i]).
// TRAIN: also g4 = s_out * 2 (out - target) / n and the squared error per thread.
// ---------------------------------------------------------------------------
template <bool TRAIN>
__global__ void l4_fwd_kernel(const __nv_bfloat16* __restrict__ a3, const float* X, int64_t ldx, int P, int nm,
                              const SurrogatePacked w, float* Xout, int64_t ldo, const float* __restrict__ target,
                              float* __restrict__ g4, float* __restrict__ sqerr_part) {
    __shared__ float red[8];
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float se = 0.f;
    if (idx < (int64_t)nm * P) {
        const int m = (int)(idx / P), p = (int)(idx % P);
        float v = w.b4[0];
#pragma unroll
        for (int t = 0; t < KT; ++t) {
            const __nv_bfloat16* row = a3 + ((int64_t)m * P + wrap(p + t - 2, P)) * CH;
#pragma unroll 8
            for (int i = 0; i < CH; ++i) v = fmaf(w.W4[t * CH + i], __bfloat162float(row[i]), v);
        }
        const float out = X[(int64_t)m * ldx + p] + SCALE_OUT * v;
        if (TRAIN) {
            const float d = out - target[(int64_t)m * ldx + p];
            se = d * d;
            g4[idx] = SCALE_OUT * 2.f * d / (float)((int64_t)nm * P);
        } else {
            Xout[(int64_t)m * ldo + p] = out;
        }
    }
    if (TRAIN) {
        se = warp_sum(se);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
            sqerr_part[blockIdx.x] = s;
        }
    }
}

// layer 4 backward: gy3 = (sum_t W4[t][i] g4[p - t + 2]) * gelu'(y3); per-CTA partials of
// gW4[t][i] = sum g4[p] a3[p+t-2][i] and gb4 = sum g4.
__global__ void __launch_bounds__(256) l4_bwd_kernel(const float* __restrict__ g4, const __nv_bfloat16* __restrict__ a3,
                                                     const __nv_bfloat16* __restrict__ y3, int P, int nm,
                                                     const SurrogatePacked w, __nv_bfloat16* __restrict__ gy3,
                                                     float* __restrict__ part /* [grid][KT*CH + 1] */) {
    __shared__ float sacc[KT * CH + 1];
    for (int e = threadIdx.x; e < KT * CH + 1; e += blockDim.x) sacc[e] = 0.f;
    __syncthreads();
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < (int64_t)nm * P) {
        const int m = (int)(idx / P), p = (int)(idx % P);
        float gsh[KT];
#pragma unroll
        for (int t = 0; t < KT; ++t) gsh[t] = g4[(int64_t)m * P + wrap(p - t + 2, P)];
        const __nv_bfloat16* yr = y3 + idx * CH;
        __align__(16) __nv_bfloat16 go[CH];
#pragma unroll 8
        for (int i = 0; i < CH; ++i) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < KT; ++t) v = fmaf(w.W4[t * CH + i], gsh[t], v);
            go[i] = __float2bfloat16(v * gelu_grad(__bfloat162float(yr[i])));
        }
#pragma unroll
        for (int q = 0; q < CH / 8; ++q) reinterpret_cast<uint4*>(gy3 + idx * CH)[q] = reinterpret_cast<uint4*>(go)[q];
    }
    // weight gradient of layer 4: thread e accumulates entry e over the CTA's positions
    const int64_t first = blockIdx.x * (int64_t)blockDim.x;
    const int64_t last = min(first + (int64_t)blockDim.x, (int64_t)nm * P);
    for (int e = threadIdx.x; e < KT * CH + 1; e += blockDim.x) {
        float v = 0.f;
        if (e == KT * CH) {
            for (int64_t q = first; q < last; ++q) v += g4[q];
        } else {
            const int t = e / CH, i = e % CH;
            for (int64_t q = first; q < last; ++q) {
                const int m = (int)(q / P), p = (int)(q % P);
                v = fmaf(g4[q], __bfloat162float(a3[((int64_t)m * P + wrap(p + t - 2, P)) * CH + i]), v);
            }
        }
        part[(int64_t)blockIdx.x * (KT * CH + 1) + e] = v;
    }
}

// Weight gradient of a 64 -> 64 layer: gW[o][i][t] = sum gy[p][o] a[p+t-2][i], gb[o] = sum gy[p][o].
// CTA = 128 positions of one member; thread -> 8 output channels x (2 inputs x 5 taps).
__global__ void __launch_bounds__(256) conv64_wgrad_kernel(const __nv_bfloat16* __restrict__ gy,
                                                           const __nv_bfloat16* __restrict__ act, int P, int nm,
                                                           float* __restrict__ part /* [grid][64*64*5 + 64] */) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float (*G)[CH + 1] = reinterpret_cast<float (*)[CH + 1]>(smem_raw);                 // [TP][CH + 1]
    float (*A)[CH + 1] = reinterpret_cast<float (*)[CH + 1]>(smem_raw + sizeof(float) * TP * (CH + 1));   // [TP + 4][CH + 1]
    const int tiles_per_member = (P + TP - 1) / TP;
    const int m = blockIdx.x / tiles_per_member;
    const int p0 = (blockIdx.x % tiles_per_member) * TP;
    const int tid = threadIdx.x;
    for (int e = tid; e < TP * CH; e += 256) {
        const int r = e / CH, c = e % CH;
        const int p = p0 + r;
        G[r][c] = p < P ? __bfloat162float(gy[((int64_t)m * P + p) * CH + c]) : 0.f;
    }
    for (int e = tid; e < (TP + 4) * CH; e += 256) {
        const int r = e / CH, c = e % CH;
        const int p = ((p0 - 2 + r) % P + P) % P;
        A[r][c] = __bfloat162float(act[((int64_t)m * P + p) * CH + c]);
    }
    __syncthreads();
    const int og = tid >> 5, ig = tid & 31;     // o = og*8 + 0..7, i = ig*2 + 0..1
    float acc[8][2][KT];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int t = 0; t < KT; ++t) acc[a][b][t] = 0.f;
    float gb[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) gb[a] = 0.f;
    const int nr = min(TP, P - p0);
    for (int r = 0; r < nr; ++r) {
        float g[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) g[a] = G[r][og * 8 + a];
#pragma unroll
        for (int t = 0; t < KT; ++t) {
            const float x0 = A[r + t][ig * 2], x1 = A[r + t][ig * 2 + 1];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                acc[a][0][t] = fmaf(g[a], x0, acc[a][0][t]);
                acc[a][1][t] = fmaf(g[a], x1, acc[a][1][t]);
            }
        }
        if (ig == 0) {
#pragma unroll
            for (int a = 0; a < 8; ++a) gb[a] += g[a];
        }
    }
    float* out = part + (int64_t)blockIdx.x * (CH * CH * KT + CH);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int t = 0; t < KT; ++t) out[((og * 8 + a) * CH + ig * 2 + b) * KT + t] = acc[a][b][t];
    if (ig == 0)
#pragma unroll
        for (int a = 0; a < 8; ++a) out[CH * CH * KT + og * 8 + a] = gb[a];
}

// Layer 1 weight gradient: gW1[o][t] = sum gy1[p][o] z0[p+t-2], gb1[o] = sum gy1[p][o].
__global__ void __launch_bounds__(256) l1_wgrad_kernel(const __nv_bfloat16* __restrict__ gy1, const float* __restrict__ X,
                                                       int64_t ldx, int P, int nm, float* __restrict__ part /* [grid][64*6] */) {
    __shared__ float Z[TP + 4];
    const int tiles_per_member = (P + TP - 1) / TP;
    const int m = blockIdx.x / tiles_per_member;
    const int p0 = (blockIdx.x % tiles_per_member) * TP;
    for (int r = threadIdx.x; r < TP + 4; r += blockDim.x) {
        const int p = ((p0 - 2 + r) % P + P) % P;
        Z[r] = (X[(int64_t)m * ldx + p] - SHIFT) * SCALE_IN;
    }
    __syncthreads();
    const int nr = min(TP, P - p0);
    for (int e = threadIdx.x; e < CH * 6; e += blockDim.x) {
        const int o = e / 6, t = e % 6;     // t = 5: bias
        float v = 0.f;
        for (int r = 0; r < nr; ++r) {
            const float g = __bfloat162float(gy1[((int64_t)m * P + p0 + r) * CH + o]);
            v = fmaf(g, t < KT ? Z[r + t] : 1.f, v);
        }
        part[(int64_t)blockIdx.x * CH * 6 + e] = v;
    }
}

// Fixed-order sum of per-CTA partials: out[e] = sum_b part[b][e].
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, int len, float* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * len + e];
        out[e] = (float)s;
    }
}

// Scatter reduced gradients into the flat master order.
__global__ void gather_grads_kernel(const float* __restrict__ g1, const float* __restrict__ g2, const float* __restrict__ g3,
                                    const float* __restrict__ g4r, float* __restrict__ flat) {
    const int n1 = CH * KT, n2 = CH * CH * KT;
    const int total = n1 + CH + 2 * (n2 + CH) + KT * CH + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int q = e;
        float v;
        if (q < n1) {
            v = g1[(q / KT) * 6 + q % KT];
        } else if ((q -= n1) < CH) {
            v = g1[q * 6 + 5];
        } else if ((q -= CH) < n2) {
            v = g2[q];
        } else if ((q -= n2) < CH) {
            v = g2[n2 + q];
        } else if ((q -= CH) < n2) {
            v = g3[q];
        } else if ((q -= n2) < CH) {
            v = g3[n2 + q];
        } else if ((q -= CH) < KT * CH) {
            const int i = q / KT, t = q % KT;   // flat W4 (1, 64, 5): i*5 + t
            v = g4r[t * CH + i];
        } else {
            v = g4r[KT * CH];
        }
        flat[e] = v;
    }
}

// Adam on the flat FP32 master parameters (bias-corrected).
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ mom, float* __restrict__ vel,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * mom[e] + (1.f - b1) * gg;
        const float vv = b2 * vel[e] + (1.f - b2) * gg * gg;
        mom[e] = mm;
        vel[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// Derives the packed inference copy from the flat master parameters.
__global__ void pack_kernel(const float* __restrict__ flat, SurrogatePacked w) {
    const int n1 = CH * KT, n2 = CH * CH * KT;
    const float* W1 = flat;
    const float* B1 = W1 + n1;
    const float* W2 = B1 + CH;
    const float* B2 = W2 + n2;
    const float* W3 = B2 + CH;
    const float* B3 = W3 + n2;
    const float* W4 = B3 + CH;
    const float* B4 = W4 + KT * CH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        const int o = e / (CH * KT), rem = e % (CH * KT), i = rem / KT, t = rem % KT;   // flat (o, i, t)
        w.W2[(o * KT + t) * CH + i] = __float2bfloat16(W2[e]);
        w.W3[(o * KT + t) * CH + i] = __float2bfloat16(W3[e]);
        w.WT2[(i * KT + (KT - 1 - t)) * CH + o] = __float2bfloat16(W2[e]);
        w.WT3[(i * KT + (KT - 1 - t)) * CH + o] = __float2bfloat16(W3[e]);
        if (e < n1) w.W1[e] = W1[e];
        if (e < CH) {
            w.b1[e] = B1[e];
            w.b2[e] = B2[e];
            w.b3[e] = B3[e];
        }
        if (e < KT * CH) {
            const int i4 = e / KT, t4 = e % KT;
            w.W4[t4 * CH + i4] = W4[e];
        }
        if (e == 0) w.b4[0] = B4[0];
    }
}

}  // namespace

int64_t surrogate_n_params() { return CH * KT + CH + 2 * (CH * CH * KT + CH) + KT * CH + 1; }

size_t surrogate_packed_bytes() {
    return sizeof(float) * (CH * KT + 3 * CH + KT * CH + 4) + sizeof(__nv_bfloat16) * 4 * CH * CH * KT + 256;
}

SurrogatePacked surrogate_view(void* packed) {
    char* b = static_cast<char*>(packed);
    SurrogatePacked w;
    w.W2 = reinterpret_cast<__nv_bfloat16*>(b);
    w.W3 = w.W2 + CH * CH * KT;
    w.WT2 = w.W3 + CH * CH * KT;
    w.WT3 = w.WT2 + CH * CH * KT;
    float* f = reinterpret_cast<float*>(w.WT3 + CH * CH * KT);
    w.W1 = f;
    w.b1 = w.W1 + CH * KT;
    w.b2 = w.b1 + CH;
    w.b3 = w.b2 + CH;
    w.W4 = w.b3 + CH;
    w.b4 = w.W4 + KT * CH;
    return w;
}

size_t conv64_smem() { return sizeof(__nv_bfloat16) * ((TP + 4) * IN_LD + CH * W_LD); }

cudaError_t surrogate_pack(const float* flat, void* packed, cudaStream_t s) {
    pack_kernel<<<(CH * CH * KT + 255) / 256, 256, 0, s>>>(flat, surrogate_view(packed));
    return cudaGetLastError();
}

static cudaError_t conv64(int mode, const __nv_bfloat16* in, int P, int nm, const __nv_bfloat16* W, const float* b,
                          const __nv_bfloat16* yprev, __nv_bfloat16* out_y, __nv_bfloat16* out_a, cudaStream_t s) {
    const size_t smem = conv64_smem();
    const int grid = nm * ((P + TP - 1) / TP);
    cudaError_t e;
    if (mode == 0) {
        if ((e = cudaFuncSetAttribute(conv64_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        conv64_kernel<0><<<grid, 256, smem, s>>>(in, P, nm, W, b, yprev, out_y, out_a);
    } else {
        if ((e = cudaFuncSetAttribute(conv64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        conv64_kernel<1><<<grid, 256, smem, s>>>(in, P, nm, W, b, yprev, out_y, out_a);
    }
    return cudaGetLastError();
}

size_t surrogate_forecast_ws(int64_t nstate, int32_t nens) {
    return 2 * sizeof(__nv_bfloat16) * (size_t)CH * nstate * nens + 256;
}

cudaError_t surrogate_forecast(float* X, int64_t ld, int64_t nstate, int32_t nens, int32_t nsteps, const void* packed,
                               void* ws, cudaStream_t s) {
    const SurrogatePacked w = surrogate_view(const_cast<void*>(packed));
    const int P = (int)nstate;
    __nv_bfloat16* a = static_cast<__nv_bfloat16*>(ws);
    __nv_bfloat16* b = a + (size_t)CH * nstate * nens;
    const int64_t npos = (int64_t)nstate * nens;
    const int blk = (int)((npos + 255) / 256);
    for (int step = 0; step < nsteps; ++step) {
        l1_fwd_kernel<<<blk, 256, 0, s>>>(X, ld, P, nens, w, nullptr, a);
        cudaError_t e = conv64(0, a, P, nens, w.W2, w.b2, nullptr, nullptr, b, s);
        if (e != cudaSuccess) return e;
        if ((e = conv64(0, b, P, nens, w.W3, w.b3, nullptr, nullptr, a, s)) != cudaSuccess) return e;
        l4_fwd_kernel<false><<<blk, 256, 0, s>>>(a, X, ld, P, nens, w, X, ld, nullptr, nullptr, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Training workspace: y1 a1 y2 a2 y3 a3 gyA gyB (bf16, 64 per position), g4 (f32), partials.
size_t surrogate_train_ws(int64_t nstate, int32_t nbatch) {
    const size_t npos = (size_t)nstate * nbatch;
    const size_t tiles = (size_t)nbatch * ((nstate + TP - 1) / TP);
    const size_t blocks = (npos + 255) / 256;
    size_t part = tiles * (CH * CH * KT + CH);
    if (blocks * (KT * CH + 1) > part) part = blocks * (KT * CH + 1);
    return sizeof(__nv_bfloat16) * 8 * CH * npos +
           sizeof(float) * (npos + part + blocks + 2 * (CH * CH * KT + CH) + (KT * CH + 1) + CH * 6 +
                            (size_t)surrogate_n_params() + 8) + 4096;
}

cudaError_t surrogate_train_step(float* master, float* mom, float* vel, int32_t step, float lr, void* packed,
                                 const float* X, const float* target, int64_t nstate, int32_t nbatch, void* ws,
                                 float* loss, float* grad_out, cudaStream_t s) {
    const SurrogatePacked w = surrogate_view(packed);
    const int P = (int)nstate, nm = nbatch;
    const size_t npos = (size_t)nstate * nbatch;
    const size_t ntiles = (size_t)nbatch * ((nstate + TP - 1) / TP);
    const int blocks = (int)((npos + 255) / 256);
    __nv_bfloat16* act = static_cast<__nv_bfloat16*>(ws);
    __nv_bfloat16 *y1 = act, *a1 = y1 + CH * npos, *y2 = a1 + CH * npos, *a2 = y2 + CH * npos;
    __nv_bfloat16 *y3 = a2 + CH * npos, *a3 = y3 + CH * npos, *gA = a3 + CH * npos, *gB = gA + CH * npos;
    float* g4 = reinterpret_cast<float*>(gB + CH * npos);
    float* sq = g4 + npos;
    float* part = sq + blocks;
    size_t partlen = ntiles * (CH * CH * KT + CH);
    if ((size_t)blocks * (KT * CH + 1) > partlen) partlen = (size_t)blocks * (KT * CH + 1);
    float* gw2 = part + partlen;
    float* gw3 = gw2 + (CH * CH * KT + CH);
    float* gw4 = gw3 + (CH * CH * KT + CH);
    float* gw1 = gw4 + (KT * CH + 1);
    float* flat = gw1 + CH * 6;   // flat gradient (n_params floats) when grad_out is NULL
    cudaError_t e;
    // forward
    l1_fwd_kernel<<<blocks, 256, 0, s>>>(X, nstate, P, nm, w, y1, a1);
    if ((e = conv64(0, a1, P, nm, w.W2, w.b2, nullptr, y2, a2, s))) return e;
    if ((e = conv64(0, a2, P, nm, w.W3, w.b3, nullptr, y3, a3, s))) return e;
    l4_fwd_kernel<true><<<blocks, 256, 0, s>>>(a3, X, nstate, P, nm, w, nullptr, 0, target, g4, sq);
    reduce_parts_kernel<<<1, 32, 0, s>>>(sq, blocks, 1, loss);   // sum of squared errors
    // backward
    l4_bwd_kernel<<<blocks, 256, 0, s>>>(g4, a3, y3, P, nm, w, gA, part);
    reduce_parts_kernel<<<(KT * CH + 1 + 255) / 256, 256, 0, s>>>(part, blocks, KT * CH + 1, gw4);
    const size_t wsm = sizeof(float) * (2 * TP + 4) * (CH + 1);
    if ((e = cudaFuncSetAttribute(conv64_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm))) return e;
    conv64_wgrad_kernel<<<(int)ntiles, 256, wsm, s>>>(gA, a2, P, nm, part);
    reduce_parts_kernel<<<(CH * CH * KT + CH + 255) / 256, 256, 0, s>>>(part, (int)ntiles, CH * CH * KT + CH, gw3);
    if ((e = conv64(1, gA, P, nm, w.WT3, nullptr, y2, nullptr, gB, s))) return e;   // gy2
    conv64_wgrad_kernel<<<(int)ntiles, 256, wsm, s>>>(gB, a1, P, nm, part);
    reduce_parts_kernel<<<(CH * CH * KT + CH + 255) / 256, 256, 0, s>>>(part, (int)ntiles, CH * CH * KT + CH, gw2);
    if ((e = conv64(1, gB, P, nm, w.WT2, nullptr, y1, nullptr, gA, s))) return e;   // gy1
    l1_wgrad_kernel<<<(int)ntiles, 256, 0, s>>>(gA, X, nstate, P, nm, part);
    reduce_parts_kernel<<<2, 256, 0, s>>>(part, (int)ntiles, CH * 6, gw1);
    float* gflat = grad_out ? grad_out : flat;
    gather_grads_kernel<<<(int)((surrogate_n_params() + 255) / 256), 256, 0, s>>>(gw1, gw2, gw3, gw4, gflat);
    if (step > 0) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
        adam_kernel<<<(int)((surrogate_n_params() + 255) / 256), 256, 0, s>>>(master, mom, vel, gflat,
                                                                              (int)surrogate_n_params(), lr, b1, b2,
                                                                              1e-8f, c1, c2);
        pack_kernel<<<(CH * CH * KT + 255) / 256, 256, 0, s>>>(master, w);
    }
    return cudaGetLastError();
}

}  // namespace enkf
