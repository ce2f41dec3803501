// pair_common.cuh - helpers shared by the pair kernels: packed pair index, tile masks,
// window facts and the per-bin metric finalize (Supplementary Information 1).
#pragma once

#include "df32.cuh"
#include "fc_internal.h"

namespace fcpair {

__device__ __forceinline__ long long packed_index(int i, int j, int n) {
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ float get4(const float4& v, int q) {
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set4(float4& v, int q, float x) {
    if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ int geti4(const int4& v, int q) {
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
__device__ __forceinline__ void seti4(int4& v, int q, int x) {
    if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
}

// Window facts read from the device control block.
struct WinFacts {
    long long end;     // trials accepted after this call (exclusive end of the window)
    long long start;   // first trial of the window
    int K;             // trials in the window
};
__device__ __forceinline__ WinFacts window_facts(const FcCtrl* c, int W, int count) {
    WinFacts w;
    w.end = c->pushed + count;
    w.start = (W > 0 && w.end > W) ? w.end - W : 0;
    w.K = (int)(w.end - w.start);
    return w;
}

// Window-length constants of the finalize (computed once per kernel, not per pair).
struct KConst {
    int K;
    float inv_K;    // 1/K
    float inv_KK1;  // 1/(K(K-1)); NaN for K < 2 (USPLI undefined)
};
__device__ __forceinline__ KConst make_kconst(int K) {
    KConst k;
    k.K = K;
    k.inv_K = 1.0f / (float)K;
    k.inv_KK1 = K >= 2 ? 1.0f / ((float)K * (float)(K - 1)) : __int_as_float(0x7fc00000);
    return k;
}

// |z| from |z|^2 as m2 * rsqrt(m2) (0 for 0).
__device__ __forceinline__ float mag_from_sq(float m2) {
    return m2 > 0.f ? __fmul_rn(m2, rsqrtf(m2)) : 0.f;
}

// x^2 - s for double-words x, s: x.hi^2 as an exact two-product plus the cross term
// 2 x.hi x.lo; the leading difference is exact when both sides are close (Sterbenz), so
// the cancellation of the debiased estimators keeps double-word accuracy (and gives an
// exact 0 for a single trial, where s holds the same two-product).
__device__ __forceinline__ float df_sq_minus(df32 x, df32 s) {
    float ph, pl;
    two_prod(x.hi, x.hi, ph, pl);
    pl = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, pl);
    return __fadd_rn(__fsub_rn(ph, s.hi), __fsub_rn(pl, s.lo));
}

// Exact float of an integer |v| < 2^22 on the FP32 pipe: v added to the integer image of
// 1.5 * 2^23 lands in the mantissa (unit spacing there), and subtracting 1.5 * 2^23 leaves v.
__device__ __forceinline__ float small_int_to_float(int v) {
    return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// Per-bin metrics from the sums of one pair-bin (Supplementary Information 1).
//   f[0..5]: CSD re, CSD im (= sum Im), phasor re, phasor im, sum |Im|, sum Im^2.
//   out[0..6]: COH, IMAGCOHY, PLV, PLI, USPLI, WPLI, DSWPLI.
// inv_i, inv_j = 1/sqrt(sum PSD); COHY = S_csd inv_i inv_j (the 1/K factors cancel).
// PLI = |S_sign| / K and USPLI = (S_sign^2 - K) / (K (K - 1)) come from the exact integer
// sign count; the ratios use the fast reciprocal division (a few ulp, far inside the
// 1e-5 tolerance).
__device__ __forceinline__ void finalize_bin(const df32* f, int sign, float inv_i, float inv_j,
                                             const KConst& kc, float* out) {
    const float cre = __fmul_rn(__fmul_rn(df_to_f(f[0]), inv_i), inv_j);
    const float cim = __fmul_rn(__fmul_rn(df_to_f(f[1]), inv_i), inv_j);
    out[0] = mag_from_sq(__fmaf_rn(cre, cre, __fmul_rn(cim, cim)));
    out[1] = cim;
    const float ure = df_to_f(f[2]), uim = df_to_f(f[3]);
    out[2] = __fmul_rn(mag_from_sq(__fmaf_rn(ure, ure, __fmul_rn(uim, uim))), kc.inv_K);
    // |S| and S^2 - K as floats, exactly: FP32-pipe arithmetic while |S^2 - K| < 2^22
    // (K <= 2048), else integer conversions (one rounding, as for any K)
    float pli_n, usn;
    if (kc.K <= 2048) {
        pli_n = small_int_to_float(abs(sign));
        usn = small_int_to_float(sign * sign - kc.K);
    } else {
        pli_n = (float)abs(sign);
        usn = kc.K <= 46340 ? (float)(sign * sign - kc.K) : (float)((long long)sign * sign - kc.K);
    }
    out[3] = __fmul_rn(pli_n, kc.inv_K);
    out[4] = __fmul_rn(usn, kc.inv_KK1);
    const float sabs = df_to_f(f[4]);
    out[5] = (sabs > 0.f) ? __fdividef(fabsf(df_to_f(f[1])), sabs) : 0.f;
    const float num = df_sq_minus(f[1], f[5]);
    const float den = df_sq_minus(f[4], f[5]);
    out[6] = (den != 0.f) ? __fdividef(num, den) : 0.f;
}

__device__ __forceinline__ void write_band(const PairArgs& a, int g, const float (*band)[4],
                                           int gi, int gj0, unsigned vmask, int nbins_group) {
    const float invB = 1.0f / (float)(a.fsel1 - a.fsel0);
    for (int m = 0; m < 7; ++m) {
        if (!(a.mask & (1u << (m + 2)))) continue;
        if (a.groups == 1) {
            float* dst = a.net_spec + (size_t)m * a.P;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (vmask & (1u << q)) dst[packed_index(gi, gj0 + q, a.n)] = __fmul_rn(band[m][q], invB);
        } else {
            float* dst = a.partial + ((size_t)g * 7 + m) * a.P;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (vmask & (1u << q)) dst[packed_index(gi, gj0 + q, a.n)] = band[m][q];
        }
    }
    (void)nbins_group;
}

__device__ __forceinline__ unsigned pair_mask(int ta, int tb, int li, int lj0, int n) {
    unsigned v = 0;
    const int gi = ta * FC_T + li;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int gj = tb * FC_T + lj0 + q;
        const bool ok = gi < n && gj < n && (ta != tb || lj0 + q > li);
        v |= ok ? (1u << q) : 0u;
    }
    return v;
}

}  // namespace fcpair
