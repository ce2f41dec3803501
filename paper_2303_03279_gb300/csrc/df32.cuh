// df32.cuh - double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, giving
// about 48 significant bits. GB300 executes FP64 at a small fraction of its FP32 rate,
// so the FP64-class accumulators of the streaming update (running sums that are added
// to and subtracted from for every pushed trial) use these error-free transformations
// instead of DADD.
//
// Algorithms (restated from the published descriptions, not copied from any code):
//   two_sum       - Knuth's TwoSum (TAOCP vol. 2, 4.2.2): s + e == a + b exactly.
//   fast_two_sum  - Dekker's Fast2Sum (1971), requires |a| >= |b| (or a == 0).
//   two_prod      - product error via one FMA: p + e == a * b exactly (no underflow).
//   df_add_f      - double-word + float, "DWPlusFP" of Joldes, Muller, Popescu,
//                   ACM TOMS 44(4), 2017: relative error <= 2u^2, u = 2^-24.
//   df_add_df     - double-word + double-word, "AccurateDWPlusDW" of the same paper:
//                   relative error <= 3u^2 + 13u^3.
//
// Every operation is an explicit round-to-nearest intrinsic so that the compiler can
// neither contract a multiply-add nor reassociate: the same inputs give the same bits
// in every kernel that includes this header.
#pragma once

struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_make(float hi, float lo) {
    df32 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df32 df_add_f(df32 x, float y) {
    float sh, sl;
    two_sum(x.hi, y, sh, sl);
    float v = __fadd_rn(x.lo, sl);
    df32 z;
    fast_two_sum(sh, v, z.hi, z.lo);
    return z;
}

__device__ __forceinline__ df32 df_add_df(df32 x, df32 y) {
    float sh, sl, th, tl;
    two_sum(x.hi, y.hi, sh, sl);
    two_sum(x.lo, y.lo, th, tl);
    float c = __fadd_rn(sl, th);
    float vh, vl;
    fast_two_sum(sh, c, vh, vl);
    float w = __fadd_rn(tl, vl);
    df32 z;
    fast_two_sum(vh, w, z.hi, z.lo);
    return z;
}

__device__ __forceinline__ df32 df_neg(df32 x) { return df_make(-x.hi, -x.lo); }

// x * x for a double-word x, to about 2^-46 relative (hi*hi exact via two_prod,
// the cross term 2 hi lo in FP32, lo*lo dropped).
__device__ __forceinline__ df32 df_sqr(df32 x) {
    float p, e;
    two_prod(x.hi, x.hi, p, e);
    e = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, e);
    df32 z;
    fast_two_sum(p, e, z.hi, z.lo);
    return z;
}

// Exact square of a float as a double-word.
__device__ __forceinline__ df32 df_sqr_f(float a) {
    df32 z;
    two_prod(a, a, z.hi, z.lo);
    return z;
}

__device__ __forceinline__ float df_to_f(df32 x) { return __fadd_rn(x.hi, x.lo); }
