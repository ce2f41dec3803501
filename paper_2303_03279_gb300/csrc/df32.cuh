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

// ---------------------------------------------------------------------------------
// Packed forms for two independent lanes (x, y), using the FP32x2 instructions of
// sm_100+ (one issue slot for two correctly rounded operations). Each lane computes
// exactly the same bits as the scalar form.

// The operations are issued as inline PTX (add/mul/fma.rn.f32x2). The error-free
// transformations below rely on every operation being exactly one correctly rounded IEEE
// step. Measured on sm_103a: a packed multiply whose result feeds a packed add may be
// fused into one FMA by the backend, which drops the product's rounding; so a packed
// add/sub never takes a raw packed product as an operand in this library (such sums are
// done with scalar __fadd_rn, which is never contracted). Products as FMA addends, and
// sums of FMA/add results, are safe.
__device__ __forceinline__ unsigned long long pack_f2(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 unpack_f2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack_f2(a)), "l"(pack_f2(b)));
    return unpack_f2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack_f2(a)), "l"(pack_f2(b)));
    return unpack_f2(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack_f2(a)), "l"(pack_f2(b)), "l"(pack_f2(c)));
    return unpack_f2(d);
}
// a - b as fma(b, -1, a): one rounding, identical to a scalar subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    const float2 aa = sub2(s, bb);
    e = add2(sub2(a, aa), sub2(b, bb));
}

__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    e = sub2(b, sub2(s, a));
}

// Running-sum update (hi, lo) += y for one float term: DWPlusFP per lane (10 ops for 2 lanes).
__device__ __forceinline__ void acc2_f(float2& hi, float2& lo, float2 y) {
    float2 s, e;
    two_sum2(hi, y, s, e);
    fast_two_sum2(s, add2(lo, e), hi, lo);
}

// Running-sum update (hi, lo) += yh + yl for one double-word term (yh, yl) per lane.
__device__ __forceinline__ void acc2_d(float2& hi, float2& lo, float2 yh, float2 yl) {
    float2 s, e;
    two_sum2(hi, yh, s, e);
    fast_two_sum2(s, add2(add2(lo, e), yl), hi, lo);
}

// Lazy running sums for many terms in a row: hi takes the rounded sum, lo collects the exact
// TwoSum errors (and the low parts of double-word terms) in FP32, with no renormalization
// (7 ops for 2 lanes instead of 10). The identity hi + sum(errors) = sum(terms) is exact, so
// after k terms hi + lo is off by at most about k^2 u^2 of the summed magnitudes (u = 2^-24,
// the FP32 rounding of lo); renorm2 brings the pair back to a normalized double word.
__device__ __forceinline__ void acc2_f_lazy(float2& hi, float2& lo, float2 y) {
    float2 s, e;
    two_sum2(hi, y, s, e);
    hi = s;
    lo = add2(lo, e);
}

__device__ __forceinline__ void acc2_d_lazy(float2& hi, float2& lo, float2 yh, float2 yl) {
    float2 s, e;
    two_sum2(hi, yh, s, e);
    hi = s;
    lo = add2(lo, add2(e, yl));
}

__device__ __forceinline__ void renorm2(float2& hi, float2& lo) {
    float2 s, e;
    two_sum2(hi, lo, s, e);
    hi = s;
    lo = e;
}

// Running-sum update (hi, lo) += y1 + y2 for two float terms: two TwoSums into the
// leading part, their errors folded into lo, one renormalization (17 ops for 2 lanes).
__device__ __forceinline__ void acc2_ff(float2& hi, float2& lo, float2 y1, float2 y2) {
    float2 s1, e1, s2, e2;
    two_sum2(hi, y1, s1, e1);
    two_sum2(s1, y2, s2, e2);
    const float2 l = add2(add2(lo, e1), e2);
    fast_two_sum2(s2, l, hi, lo);
}

// Running-sum update (hi, lo) += (y1h + y1l) + (y2h + y2l) for two double-word terms.
__device__ __forceinline__ void acc2_dd(float2& hi, float2& lo, float2 y1h, float2 y1l, float2 y2h, float2 y2l) {
    float2 s1, e1, s2, e2;
    two_sum2(hi, y1h, s1, e1);
    two_sum2(s1, y2h, s2, e2);
    const float2 l = add2(add2(add2(lo, e1), add2(e2, y1l)), y2l);
    fast_two_sum2(s2, l, hi, lo);
}
