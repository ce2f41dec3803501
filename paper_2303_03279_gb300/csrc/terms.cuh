// terms.cuh - the per-pair, per-trial, per-bin terms that the running sums accumulate.
//
// For a node pair (i, j) and one trial's spectra X_i = a_i + i b_i, X_j = a_j + i b_j
// at one bin (Supplementary Information 1, Frequency Domain):
//   CSD_ij = X_i X_j*  ->  re = a_i a_j + b_i b_j,  im = b_i a_j - a_i b_j
//   sign(Im CSD_ij)    ->  exact, see below (PLI, USPLI)
//   u_i u_j*           ->  phasor product with u = X/|X| (PLV; 0 where X = 0)
// and the derived |im|, im^2 (WPLI, DSWPLI).
//
// The streaming update adds the terms of the new trial and subtracts those of the trial
// leaving the window; both come from these functions applied to the stored spectra,
// with explicit rounding intrinsics, so the subtracted value has exactly the bits that
// were added. Every step is sign-symmetric, so the terms of (X_i, -X_j) are the exact
// negations of those of (X_i, X_j): the streaming kernel subtracts a trial by staging
// its column spectra negated. The scalar and the packed (two pairs per instruction)
// forms perform the same correctly rounded operations lane by lane.
//
// Exact sign of b_i a_j - a_i b_j from FP32 operands: p = fl(b_i a_j), q = fl(a_i b_j).
// Rounding is monotone, so p > q implies b_i a_j > a_i b_j (and likewise for <). If
// p == q the sign is that of e - f with e = b_i a_j - p and f = a_i b_j - q, both exact
// FMA residuals; a rounded difference keeps the sign of the exact one. The residuals are
// exact when both factors of each product are 0 or at least 2^-50 in magnitude (the
// residual's last bit is then >= 2^-146, inside the subnormal range). A node with a
// nonzero component below 2^-50 is flagged when its spectra are staged and its pairs
// take an FP64 evaluation instead (FP32 x FP32 products are exact in FP64 and one
// rounded subtraction keeps the sign).
#pragma once

#include "df32.cuh"

// A nonzero component below 2^-50: FMA residuals of its products might be inexact.
__device__ __forceinline__ bool node_tiny(float2 X) {
    const float t = 8.8817841970012523e-16f;  // 2^-50
    return (X.x != 0.f && fabsf(X.x) < t) || (X.y != 0.f && fabsf(X.y) < t);
}

// u = X / |X| (0 for X == 0): the unit phasor e^{i Phi} used by PLV.
__device__ __forceinline__ float2 phasor_of(float2 X) {
    float m2 = __fmaf_rn(X.x, X.x, __fmul_rn(X.y, X.y));
    float r = (m2 > 0.0f) ? rsqrtf(m2) : 0.0f;
    return make_float2(__fmul_rn(X.x, r), __fmul_rn(X.y, r));
}

__device__ __forceinline__ void im_sign_fp64(float ai, float bi, float aj, float bj, float& im, int& s) {
    const double d = (double)bi * (double)aj - (double)ai * (double)bj;
    s = (d > 0.0) - (d < 0.0);
    im = (float)d;
}

__device__ __forceinline__ int sign_of(float t) { return (t > 0.f) - (t < 0.f); }

// The same FP64 evaluation kept out of line: a call is never if-converted, so a kernel that
// cannot tell tiny nodes apart in advance pays for it only when a node is tiny.
struct ImSign {
    float im;
    int s;
};
static __device__ __noinline__ ImSign im_sign_fp64_call(float ai, float bi, float aj, float bj) {
    ImSign v;
    im_sign_fp64(ai, bi, aj, bj, v.im, v.s);
    return v;
}

struct PairTerms {
    float re;  // Re(X_i X_j*)
    float im;  // Im(X_i X_j*), the correctly signed, nearly correctly rounded value
    int sgn;   // sign(Im(X_i X_j*)) in {-1, 0, 1}, exact
    float ure; // Re(u_i u_j*)
    float uim; // Im(u_i u_j*)
};

// Scalar form; tiny = node_tiny(X_i) || node_tiny(X_j).
__device__ __forceinline__ PairTerms pair_terms(float2 Xi, float2 Xj, float2 ui, float2 uj, bool tiny) {
    PairTerms t;
    const float ai = Xi.x, bi = Xi.y, aj = Xj.x, bj = Xj.y;
    t.re = __fmaf_rn(ai, aj, __fmul_rn(bi, bj));
    const float p = __fmul_rn(bi, aj), np = __fmul_rn(-bi, aj);
    const float q = __fmul_rn(ai, bj), nq = __fmul_rn(-ai, bj);
    const float e = __fmaf_rn(bi, aj, np);   // b_i a_j - p
    const float nf = __fmaf_rn(-ai, bj, q);  // -(a_i b_j - q)
    const float d1 = __fadd_rn(p, nq);       // fl(p - q)
    const float d2 = __fadd_rn(e, nf);       // fl(e - f)
    t.im = __fadd_rn(d1, d2);
    t.sgn = sign_of(d1 != 0.f ? d1 : d2);
    if (tiny) im_sign_fp64(ai, bi, aj, bj, t.im, t.sgn);
    t.ure = __fmaf_rn(ui.x, uj.x, __fmul_rn(ui.y, uj.y));
    t.uim = __fmaf_rn(ui.y, uj.x, __fmul_rn(-ui.x, uj.y));
    return t;
}

// Row-node constants of the packed form (one node i against two column nodes).
struct RowConst {
    float2 a, b, na, nb, ua, ub, nua;
    float as, bs;  // scalar a_i, b_i for the FP64 path
    bool tiny;
};
__device__ __forceinline__ RowConst row_const(float a, float b, float ua, float ub, bool tiny) {
    RowConst r;
    r.a = f2(a);
    r.b = f2(b);
    r.na = f2(-a);
    r.nb = f2(-b);
    r.ua = f2(ua);
    r.ub = f2(ub);
    r.nua = f2(-ua);
    r.as = a;
    r.bs = b;
    r.tiny = tiny;
    return r;
}

struct PairTerms2 {
    float2 re, im, ure, uim;
    int s0, s1;
};

// Packed form for pairs (i, j0) and (i, j1): aj = (a_j0, a_j1), bj = (b_j0, b_j1), ...
// TINY = false: the caller knows that none of the nodes is tiny, so the FP64 branch is
// not compiled in (it would otherwise be if-converted into the hot loop).
template <bool TINY = true>
__device__ __forceinline__ PairTerms2 pair_terms2(const RowConst& r, float2 aj, float2 bj, float2 uaj, float2 ubj,
                                                  bool tiny0, bool tiny1) {
    PairTerms2 t;
    t.re = fma2(r.a, aj, mul2(r.b, bj));
    const float2 p = mul2(r.b, aj), np = mul2(r.nb, aj);
    const float2 q = mul2(r.a, bj), nq = mul2(r.na, bj);
    const float2 e = fma2(r.b, aj, np);
    const float2 nf = fma2(r.na, bj, q);
    // fl(p) - fl(q) in scalar form: a packed add whose operand is a packed product can be
    // fused by the backend into one FMA (which would drop the rounding of the product);
    // the scalar round-to-nearest add is never contracted.
    const float2 d1 = make_float2(__fadd_rn(p.x, nq.x), __fadd_rn(p.y, nq.y));
    const float2 d2 = add2(e, nf);
    t.im = add2(d1, d2);
    t.s0 = sign_of(d1.x != 0.f ? d1.x : d2.x);
    t.s1 = sign_of(d1.y != 0.f ? d1.y : d2.y);
    if (TINY && (r.tiny || tiny0)) {
        const ImSign v = im_sign_fp64_call(r.as, r.bs, aj.x, bj.x);
        t.im.x = v.im;
        t.s0 = v.s;
    }
    if (TINY && (r.tiny || tiny1)) {
        const ImSign v = im_sign_fp64_call(r.as, r.bs, aj.y, bj.y);
        t.im.y = v.im;
        t.s1 = v.s;
    }
    t.ure = fma2(r.ua, uaj, mul2(r.ub, ubj));
    t.uim = fma2(r.ub, uaj, mul2(r.nua, ubj));
    return t;
}
