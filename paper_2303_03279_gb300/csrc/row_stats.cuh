// row_stats.cuh - per-row mean and sum of squared deviations for the time-domain metrics
// (COR, XCOR: the signals are centered before correlating, Supplementary Information 1),
// one warp per row, in double-float FP32 arithmetic.
#pragma once

#include "df32.cuh"

// Double-word sum over a warp by a butterfly of exact TwoSums: every lane ends with the same
// bits (TwoSum gives the same pair for (a, b) and (b, a)).
__device__ __forceinline__ void warp_df_allreduce(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        e = __fadd_rn(e, __fadd_rn(lo, ol));
        fast_two_sum(s, e, hi, lo);
    }
}

// Mean and sum of squared deviations of one warp's row x[0..N) without FP64 (which GB300
// runs at a small fraction of the FP32 rate). The row is first shifted by its first sample
// (y = x - x0, so a constant row is exactly 0 and stays so), y is summed as a double word,
// mean_y = sum / N as a double word (FMA remainder), and the deviations
// d = (y - mean_hi) - mean_lo are squared as exact two-products summed the same way.
struct RowStats {
    float x0, mean_hi, mean_lo;  // deviation of sample t: dev(x[t])
    float ss;                    // sum of dev^2, rounded once from its double word
    __device__ __forceinline__ float dev(float xt) const {
        return __fsub_rn(__fsub_rn(__fsub_rn(xt, x0), mean_hi), mean_lo);
    }
};

__device__ __forceinline__ RowStats warp_row_stats(const float* x, int N, int lane) {
    RowStats r;
    r.x0 = N > 0 ? x[0] : 0.f;
    float h = 0.f, l = 0.f;
    for (int t = lane; t < N; t += 32) {
        float s, e;
        two_sum(h, __fsub_rn(x[t], r.x0), s, e);
        h = s;
        l = __fadd_rn(l, e);
    }
    warp_df_allreduce(h, l);
    const float fN = (float)(N > 0 ? N : 1);
    r.mean_hi = __fdiv_rn(h, fN);
    r.mean_lo = __fdiv_rn(__fadd_rn(__fmaf_rn(-r.mean_hi, fN, h), l), fN);
    float qh = 0.f, ql = 0.f;
    for (int t = lane; t < N; t += 32) {
        const float d = r.dev(x[t]);
        float p, pe, s, e;
        two_prod(d, d, p, pe);
        two_sum(qh, p, s, e);
        qh = s;
        ql = __fadd_rn(ql, __fadd_rn(e, pe));
    }
    warp_df_allreduce(qh, ql);
    r.ss = __fadd_rn(qh, ql);
    return r;
}

