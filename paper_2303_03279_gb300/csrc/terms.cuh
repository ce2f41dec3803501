// terms.cuh - the per-pair, per-trial, per-bin terms that the running sums accumulate.
//
// For a node pair (i, j) and one trial's spectra X_i = a_i + i b_i, X_j = a_j + i b_j
// at one bin (Supplementary Information 1, Frequency Domain):
//   CSD_ij = X_i X_j*  ->  re = a_i a_j + b_i b_j,  im = b_i a_j - a_i b_j
//   sign(Im CSD_ij)    ->  exact, see below (PLI, USPLI)
//   u_i u_j*           ->  phasor product with u = X/|X| (PLV; 0 where X = 0)
// and the derived |im|, im^2 (WPLI, DSWPLI).
//
// The streaming update adds the terms of the new trial and subtracts those of the
// trial leaving the window; both come from this one function applied to the stored
// spectra, with explicit rounding intrinsics, so the subtracted value has exactly the
// bits of the value that was added (no contraction differences between kernels).
//
// Exact sign of b_i a_j - a_i b_j from FP32 operands: p = fl(b_i a_j), q = fl(a_i b_j).
// Rounding is monotone, so p > q implies b_i a_j > a_i b_j (and likewise for <). If
// p == q the sign is that of e - f with e = b_i a_j - p and f = a_i b_j - q, both exact
// as FMA residuals and their rounded difference keeps its sign. The residuals are exact
// only while the products stay well above the subnormal range; when a nonzero product
// is below 2^-100 the sign is taken from an FP64 evaluation instead (FP32 x FP32 products
// are exact in FP64 and a single rounded subtraction keeps the sign).
#pragma once

struct PairTerms {
    float re;  // Re(X_i X_j*)
    float im;  // Im(X_i X_j*), the correctly signed, nearly correctly rounded value
    int sgn;   // sign(Im(X_i X_j*)) in {-1, 0, 1}, exact
    float ure; // Re(u_i u_j*)
    float uim; // Im(u_i u_j*)
};

// u = X / |X| (0 for X == 0): the unit phasor e^{i Phi} used by PLV.
__device__ __forceinline__ float2 phasor_of(float2 X) {
    float m2 = __fmaf_rn(X.x, X.x, __fmul_rn(X.y, X.y));
    float r = (m2 > 0.0f) ? rsqrtf(m2) : 0.0f;
    return make_float2(__fmul_rn(X.x, r), __fmul_rn(X.y, r));
}

__device__ __forceinline__ PairTerms pair_terms(float2 Xi, float2 Xj, float2 ui, float2 uj) {
    PairTerms t;
    const float ai = Xi.x, bi = Xi.y, aj = Xj.x, bj = Xj.y;
    t.re = __fmaf_rn(ai, aj, __fmul_rn(bi, bj));
    const float p = __fmul_rn(bi, aj);
    const float q = __fmul_rn(ai, bj);
    const float e = __fmaf_rn(bi, aj, -p);
    const float f = __fmaf_rn(ai, bj, -q);
    t.im = __fadd_rn(__fsub_rn(p, q), __fsub_rn(e, f));
    int s = (p > q) - (p < q);
    const int s2 = (e > f) - (e < f);
    s = (p == q) ? s2 : s;
    const float tiny = 7.88860905e-31f;  // 2^-100
    const bool p_tiny = fabsf(p) < tiny && bi != 0.0f && aj != 0.0f;
    const bool q_tiny = fabsf(q) < tiny && ai != 0.0f && bj != 0.0f;
    if (p_tiny || q_tiny) {
        const double d = (double)bi * (double)aj - (double)ai * (double)bj;
        s = (d > 0.0) - (d < 0.0);
        t.im = (float)d;
    }
    t.sgn = s;
    t.ure = __fmaf_rn(ui.x, uj.x, __fmul_rn(ui.y, uj.y));
    t.uim = __fmaf_rn(ui.y, uj.x, -__fmul_rn(ui.x, uj.y));
    return t;
}
