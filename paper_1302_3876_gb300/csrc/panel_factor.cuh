// b x b factor of one panel of the iterative Sherman-Morrison recurrence (eqs.
// SM-step-2-h/u restricted to b levels), shared by the single-problem panel kernel
// and the batched kernel.  S is any shared-memory view with the float arrays Gh, Gl
// (the panel Gram G = Gh + Gl), Bt, cb, Lt, W, Bf and the double array gam, all with
// row stride kFB.
#pragma once

#include "common.cuh"

namespace enkf {

constexpr int kFB = 32;   // largest panel width

// Knuth's TwoSum with explicitly rounded operations: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// W = B (I + L)^{-1} by backward substitution, lane q < bp forming row q:
//   W[q][l] = B[q][l] - sum_{m > l} W[q][m] L[m][l].  Reads Bt and Lt, writes W.
template <typename S>
__device__ void panel_w(const S& s, int bp) {
    const int q = threadIdx.x & 31;
    if (q < bp) {
        float w[kFB];
#pragma unroll
        for (int l = kFB - 1; l >= 0; --l) {
            if (l < bp) {
                float v = s.Bt[l * kFB + q];
#pragma unroll
                for (int m = l + 1; m < kFB; ++m)
                    if (m < bp) v = fmaf(-s.Lt[l * kFB + m], w[m], v);
                w[l] = v;
                s.W[q * kFB + l] = v;
            } else {
                w[l] = 0.f;
            }
        }
    }
    __syncwarp();
}

// b x b factor from the panel Gram G = Gh + Gl by one warp; lane j keeps the
// coefficient vector beta_j (u_j = U_P beta_j) in registers.  Per level m:
//   g_j = (G beta_j)_m (FP32), gamma_m = 1 + (G beta_m)_m in double-FP32 (exact
//   products, TwoSum butterfly over the lanes), B[:,m] = beta_m / gamma_m,
//   beta_j -= B[:,m] g_j (j > m).
// Then L = strictly lower part of G B and W = B (I + L)^{-1}.  No FP64 arithmetic:
// on GB300 a warp-wide FP64 instruction occupies the FP64 pipe for ~64 cycles.
// gamma is written to s.gam (FP64) and the final beta to s.Bf.
template <typename S>
__device__ void factor_warp(const S& s, int bp) {
    const int lane = threadIdx.x & 31;
    float beta[kFB];
#pragma unroll
    for (int u = 0; u < kFB; ++u) beta[u] = (u == lane) ? 1.f : 0.f;
    float ghi_l = 0.f, glo_l = 0.f, ginv_l = 0.f;   // gamma of this lane's level
    for (int m = 0; m < bp; ++m) {
        const float* gr = s.Gh + m * kFB;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
        for (int u = 0; u < kFB; u += 4) {
            const float4 gv = *reinterpret_cast<const float4*>(gr + u);
            g0 = fmaf(gv.x, beta[u], g0);
            g1 = fmaf(gv.y, beta[u + 1], g1);
            g2 = fmaf(gv.z, beta[u + 2], g2);
            g3 = fmaf(gv.w, beta[u + 3], g3);
        }
        const float gj = (g0 + g1) + (g2 + g3);
        if (lane == m) {
#pragma unroll
            for (int u = 0; u < kFB; ++u) s.cb[u] = beta[u];
        }
        __syncwarp();
        // gamma_m = 1 + sum_u G[m][u] beta[u][m]: lane u forms its term exactly as hi + lo
        const float bu = s.cb[lane];
        const float gh = gr[lane];
        float hi = __fmul_rn(gh, bu);
        float lo = __fmaf_rn(gh, bu, -hi);
        lo = __fmaf_rn(s.Gl[m * kFB + lane], bu, lo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            float t, e;
            two_sum(hi, h2, t, e);
            hi = t;
            lo = __fadd_rn(__fadd_rn(lo, l2), e);
        }
        float g_hi, e1;
        two_sum(1.f, hi, g_hi, e1);
        float g_lo = __fadd_rn(lo, e1);
        const float tmp = __fadd_rn(g_hi, g_lo);            // renormalise (|g_lo| << |g_hi|)
        g_lo = __fsub_rn(g_lo, __fsub_rn(tmp, g_hi));
        g_hi = tmp;
        const float ginv = 1.0f / g_hi;
        if (lane == m) ghi_l = g_hi, glo_l = g_lo, ginv_l = ginv;
        // B[:,m] = beta_m / gamma_m, kept transposed
        s.Bt[m * kFB + lane] = bu * ginv;
        __syncwarp();
        if (lane > m && lane < bp) {
            const float* bm = s.Bt + m * kFB;
#pragma unroll
            for (int u = 0; u < kFB; u += 4) {
                const float4 bv = *reinterpret_cast<const float4*>(bm + u);
                beta[u] = fmaf(-bv.x, gj, beta[u]);
                beta[u + 1] = fmaf(-bv.y, gj, beta[u + 1]);
                beta[u + 2] = fmaf(-bv.z, gj, beta[u + 2]);
                beta[u + 3] = fmaf(-bv.w, gj, beta[u + 3]);
            }
        }
        __syncwarp();
    }
    if (lane < bp) {
        s.gam[lane] = (double)ghi_l + (double)glo_l;
        // final beta_l (= gamma_l B[:,l]) for the panel's own columns; B[:,l] = beta_l / gamma_l
#pragma unroll
        for (int u = 0; u < kFB; ++u) s.Bf[u * kFB + lane] = beta[u];
        // L[m][l] = sum_u G[m][u] B[u][l] for m > l (lane l)
        float bl[kFB];
#pragma unroll
        for (int u = 0; u < kFB; ++u) bl[u] = beta[u] * ginv_l;
        for (int m = 0; m < bp; ++m) {
            float v = 0.f;
            if (m > lane) {
                const float* gr = s.Gh + m * kFB;
#pragma unroll
                for (int u = 0; u < kFB; u += 4) {
                    const float4 gv = *reinterpret_cast<const float4*>(gr + u);
                    v = fmaf(gv.x, bl[u], v);
                    v = fmaf(gv.y, bl[u + 1], v);
                    v = fmaf(gv.z, bl[u + 2], v);
                    v = fmaf(gv.w, bl[u + 3], v);
                }
            }
            s.Lt[lane * kFB + m] = v;
        }
    }
    __syncwarp();
    panel_w(s, bp);
}

}  // namespace enkf
