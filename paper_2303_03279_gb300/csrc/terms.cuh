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
// its column spectra negated. The packed form computes two pairs per instruction with
// correctly rounded operations lane by lane.
//
// Im = b_i a_j - a_i b_j by Kahan's 2x2 determinant algorithm: w = fl(a_i b_j),
// e = w - a_i b_j (exact, one FMA), f = fl(b_i a_j - w) (one FMA), im = fl(f + e).
// Jeannerod, Louvet and Muller (Math. Comp. 82, 2013) prove |im - Im| <= 2u |Im| without
// underflow, so im is 0 exactly when Im is and otherwise has its sign: the sign counts are
// exact. Directly: Im = F + e with F = b_i a_j - w; if |F| < ulp(w), F has at most 24
// significant bits, so f = F and im = fl(Im); otherwise |e| <= ulp(w) / 2 <= |F| / 2, so
// |Im| >= |F| / 2, far above the rounding error of f (<= u |F|). Both steps need exact residuals and no inexact subnormal result,
// which holds when every factor is 0 or at least 2^-50 in magnitude (each product is then a
// multiple of 2^-146, inside the subnormal grid). A node with a nonzero component below
// 2^-50 is flagged when its spectra are staged and its pairs take an FP64 evaluation
// instead (FP32 x FP32 products are exact in FP64 and one rounded subtraction keeps the
// sign).
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

// Packed Kahan determinant for two column nodes: Im(X_i X_j*) = b_i a_j - a_i b_j with
// bi = (b_i, b_i), ai = (a_i, a_i), nai = (-a_i, -a_i). Every add takes FMA results, never a
// raw product (a packed add of a packed product may be contracted into one FMA). Negating
// the column spectra negates every intermediate exactly, so the terms of (X_i, -X_j) are
// the exact negations of those of (X_i, X_j).
__device__ __forceinline__ float2 kahan_im2(float2 bi, float2 ai, float2 nai, float2 aj, float2 bj) {
    const float2 nw = mul2(nai, bj);              // -fl(a_i b_j)
    const float2 f = fma2(bi, aj, nw);            // fl(b_i a_j - w)
    const float2 me = fma2(ai, bj, nw);           // a_i b_j - w, exact
    return fma2(me, make_float2(-1.f, -1.f), f);  // fl(f - me)
}

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

// Row-node constants of the packed form (one node i against two column nodes).
struct RowConst {
    float2 a, b, na, ua, ub, nua;
    float as, bs;  // scalar a_i, b_i for the FP64 path
    bool tiny;
};
__device__ __forceinline__ RowConst row_const(float a, float b, float ua, float ub, bool tiny) {
    RowConst r;
    r.a = f2(a);
    r.b = f2(b);
    r.na = f2(-a);
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
    t.im = kahan_im2(r.b, r.a, r.na, aj, bj);
    t.s0 = sign_of(t.im.x);
    t.s1 = sign_of(t.im.y);
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
