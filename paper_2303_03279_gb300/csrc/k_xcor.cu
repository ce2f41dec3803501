// k_xcor.cu - cross-correlation (XCOR), Supplementary Information 1 (Time Domain) and
// Methods 2.4: "an FFT convolution, which consists of the creation of the signal spectra,
// multiplication of these spectra, and the transformation of the product back to the time
// domain. Subsequently, the highest correlation value and its index are returned."
//
// Per trial k and node i: x~_i = x_i - mean, energy E_i = sum x~_i^2, and the length-L
// real spectrum Z_i of x~_i zero-padded to L (power of two >= 2N - 1, so the circular
// correlation equals the linear one for |tau| <= N - 1). Per pair (i, j):
//   R(tau) = irfft(Z_i Z_j*)[tau mod L] = sum_t x~_i(t + tau) x~_j(t),
//   XCOR_k(i, j) = max_{|tau| <= N-1} R(tau) / sqrt(E_i E_j)   (0 if E_i E_j = 0),
// ties to the smallest |tau|, then the negative tau. The network is the mean over trials.
//
// Transforms are hand-written radix-2 FFTs in shared memory, one warp per signal: a real
// length-L transform is done as a complex length-M = L/2 transform plus the standard
// even/odd split (forward) or merge (inverse). Twiddles come from a host-built FP64 table
// rounded to FP32 (tw[k] = exp(-2 pi i k / L), k < L/2).
#include <climits>

#include "df32.cuh"
#include "fc_internal.h"
#include "row_stats.cuh"

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Pair (i, j), i < j, of packed index p (row r starts at r*n - r(r+1)/2).
// Row i of packed pair p: an FP32 estimate from the quadratic (FP64 runs at a small fraction
// of the FP32 rate here), corrected exactly in integers.
__device__ __forceinline__ void unpack_pair(long long p, int n, int& i, int& j) {
    const float b = 2.0f * (float)n - 1.0f;
    int r = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)p, 0.f))) * 0.5f);
    if (r < 0) r = 0;
    if (r > n - 2) r = n - 2;
    while (r > 0 && (long long)r * n - (long long)r * (r + 1) / 2 > p) --r;
    while (r < n - 2 && (long long)(r + 1) * n - (long long)(r + 1) * (r + 2) / 2 <= p) ++r;
    i = r;
    j = (int)(p - ((long long)r * n - (long long)r * (r + 1) / 2)) + r + 1;
}

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place radix-2 decimation-in-time FFT of buf[0..M) (already in bit-reversed order),
// executed by one warp. sign = -1: forward (exp(-i...)), +1: inverse (no 1/M scaling).
__device__ void warp_fft(float2* buf, int M, const float2* __restrict__ tw, int L, int sign) {
    const int lane = threadIdx.x & 31;
    for (int s = 1; s < M; s <<= 1) {
        const int step = L / (2 * s);
        for (int b = lane; b < M / 2; b += 32) {
            const int j = b & (s - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + s;
            float2 w = tw[j * step];
            if (sign > 0) w.y = -w.y;
            const float2 u = buf[i0], v = cmul(buf[i1], w);
            buf[i0] = cadd(u, v);
            buf[i1] = csub(u, v);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ node spectra
// One warp per (trial, node). Shared memory: M float2 per warp.
__global__ void k_xcor_spectra(XcorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    extern __shared__ float2 smem[];
    const int M = a.L / 2;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* buf = smem + (size_t)wib * M;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int ntr = a.count - a.write_from;
    if (warp >= ntr * a.n) return;
    const int tr = a.write_from + warp / a.n, node = warp % a.n;
    const float* x = a.x + ((size_t)tr * a.n + node) * a.N;
    // centered samples and their energy as double words on the FP32 pipes (row_stats.cuh)
    const RowStats st = warp_row_stats(x, a.N, lane);
    int bits = 0;
    while ((1 << bits) < M) ++bits;
    for (int m = lane; m < M; m += 32) {
        const int t0 = 2 * m, t1 = 2 * m + 1;
        const float v0 = t0 < a.N ? st.dev(x[t0]) : 0.f;
        const float v1 = t1 < a.N ? st.dev(x[t1]) : 0.f;
        buf[bitrev(m, bits)] = make_float2(v0, v1);
    }
    __syncwarp();
    warp_fft(buf, M, a.tw, a.L, -1);
    const long long g = c->pushed + tr;
    const int slot = (int)(g % a.slots);
    float2* out = a.spec + ((size_t)slot * a.n + node) * (M + 1);
    for (int k = lane; k <= M; k += 32) {
        const float2 zk = buf[k == M ? 0 : k];
        const float2 zc = cconj(buf[k == 0 ? 0 : M - k]);
        const float2 e = make_float2(0.5f * __fadd_rn(zk.x, zc.x), 0.5f * __fadd_rn(zk.y, zc.y));
        const float2 d = csub(zk, zc);  // 2i O[k]
        const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);  // d / (2i)
        const float2 w = (k < M) ? a.tw[k] : make_float2(-1.f, 0.f);
        out[k] = cadd(e, cmul(w, o));
    }
    if (lane == 0) a.energy[(size_t)slot * a.n + node] = st.ss;
}

// ------------------------------------------------------------------ pair correlations
// One warp per (pair, trial). Trials: the window (full mode) or the newest (stream mode).
__device__ __forceinline__ bool better(float v1, int t1, float v2, int t2) {
    if (v1 != v2) return v1 > v2;
    const int a1 = abs(t1), a2 = abs(t2);
    if (a1 != a2) return a1 < a2;
    return t1 < t2;
}

__global__ void k_xcor_pairs(XcorArgs a, long long n_items, long long first_trial, int n_trials) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    extern __shared__ float2 smem[];
    const int M = a.L / 2;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* buf = smem + (size_t)wib * M;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    if (item >= n_items) return;
    // trial-major: the warps of a CTA take consecutive pairs of one trial (pairs of one row
    // share its spectrum in L1; one trial's spectra stay in L2 while all pairs read them)
    const long long p = item % a.P;
    const long long trial = c->pushed + first_trial + item / a.P;
    if (trial < 0) return;  // window not yet full
    int i, j;
    unpack_pair(p, a.n, i, j);
    {
        const int slot = (int)(trial % a.slots);
        const float2* Zi = a.spec + ((size_t)slot * a.n + i) * (M + 1);
        const float2* Zj = a.spec + ((size_t)slot * a.n + j) * (M + 1);
        int bits = 0;
        while ((1 << bits) < M) ++bits;
        // Y[k] = E[k] + i O[k], E = (P[k] + conj P[M-k]) / 2, O = (P[k] - conj P[M-k]) e^{+2 pi i k/L} / 2
        for (int k = lane; k < M; k += 32) {
            const float2 pk = cmul(Zi[k], cconj(Zj[k]));
            const float2 pm = cconj(cmul(Zi[M - k], cconj(Zj[M - k])));
            const float2 e = make_float2(0.5f * __fadd_rn(pk.x, pm.x), 0.5f * __fadd_rn(pk.y, pm.y));
            const float2 dd = csub(pk, pm);
            float2 w = a.tw[k];
            w.y = -w.y;  // e^{+2 pi i k / L}
            const float2 o = cmul(make_float2(0.5f * dd.x, 0.5f * dd.y), w);
            buf[bitrev(k, bits)] = make_float2(__fsub_rn(e.x, o.y), __fadd_rn(e.y, o.x));  // e + i o
        }
        __syncwarp();
        warp_fft(buf, M, a.tw, a.L, +1);
        // r[2m] = Re y[m] / M, r[2m+1] = Im y[m] / M; scan lags |tau| <= N-1
        float best = -INFINITY;
        int best_tau = 0;
        const float invM = 1.0f / (float)M;
        for (int tau = -(a.N - 1) + lane; tau <= a.N - 1; tau += 32) {
            const int idx = tau >= 0 ? tau : a.L + tau;
            const float2 y = buf[idx >> 1];
            const float r = __fmul_rn((idx & 1) ? y.y : y.x, invM);
            if (better(r, tau, best, best_tau)) {
                best = r;
                best_tau = tau;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int ot = __shfl_xor_sync(0xffffffffu, best_tau, o);
            if (better(ov, ot, best, best_tau)) {
                best = ov;
                best_tau = ot;
            }
        }
        if (lane == 0) {
            const float ei = a.energy[(size_t)slot * a.n + i], ej = a.energy[(size_t)slot * a.n + j];
            const float den = __fmul_rn(sqrtf(ei), sqrtf(ej));
            float v = 0.f;
            int lag = 0;
            if (den > 0.f) {
                v = __fdiv_rn(best, den);
                lag = best_tau;
            }
            a.vals[(size_t)slot * a.P + p] = v;
            if (trial == c->pushed + a.count - 1) a.lag[p] = lag;
        }
    }
}

// Register form for transforms of M = 32 E 2^S complex points (E = 2 .. 64, S = 0 .. 2:
// trials up to 8,192 samples). The inverse transform runs as radix-2 decimation in
// frequency on natural-order input. With S >= 1 the first S stages split it into 2^S
// independent blocks of 32 E points (S = 1: top u + v, the even outputs; bottom (u - v) w,
// the odd outputs; S = 2 repeats the split on both halves, block b holding the outputs
// 4 k + bitrev2(b)); the blocks are transformed one after the other in the same registers,
// each forming its inputs from the product spectrum again. Within a block, lane l first
// holds elements l + 32 r, r < E: spans of 32 or more pair registers of the same lane;
// spans from 16 down to E (only when E <= 16) pair lanes through __shfl_xor_sync. One
// transpose through this warp's shared-memory buffer (a pad slot per E elements keeps both
// directions free of bank conflicts) then gives lane l the E consecutive elements l E + q,
// so the remaining spans (below E and below 32) pair registers of the same lane again, with
// twiddles that are the same for every lane. The output lands in bit-reversed order, which
// the scan over lags reads through the bit reversal of each position.
// CTAs per SM to keep registers for: at 512-point transforms one more than the register use
// alone would allow (shared memory holds four; the kernel is issue-bound and gains from
// warps); at 1024 points two, with the product-step twiddle table (three CTAs without the
// table and with 80 registers spilled and took 3 % longer once the products are staged
// in shared memory)
// 0: no minimum (the plain bound). The explicit minimum of one at 2048 points lets ptxas
// keep 240 registers instead of 188 (15 % faster); at 4096 points it made ptxas spill
// 564 bytes (22 % slower), so that form keeps the plain bound.
template <int E, int S> struct XcorMinBlocks { static constexpr int v = 0; };
template <> struct XcorMinBlocks<16, 0> { static constexpr int v = 4; };
template <> struct XcorMinBlocks<32, 0> { static constexpr int v = 2; };
template <> struct XcorMinBlocks<64, 0> { static constexpr int v = 1; };
// Forms without the product-step twiddle table stw (its odd entries come from the stage
// table): 8192 points, where it does not fit
template <int E, int S> struct XcorNoStw { static constexpr bool v = S == 2; };

template <int E, int S>
__device__ __forceinline__ void xcor_pairs_reg(const XcorArgs& a, long long n_items, long long first_trial,
                                               int n_trials) {
    constexpr int MS = 32 * E;  // points of one register transform
    constexpr int M = MS << S;  // points of the whole complex transform
    // dynamic shared memory: stw[M] = tw[k] = e^{-2 pi i k / L} (not in every form); sth[M] = the
    // butterflies' twiddles by stage, span h at sth[h + t] = tw[t M / h], t < h (a stage's
    // lanes read consecutive entries or one entry each, broadcast: no bank conflicts); then
    // one transpose buffer of MS + MS / E slots per warp. Without stw (see XcorNoStw):
    // tw[2t] = sth[M / 2 + t] and tw[2t + 1] = tw[2t] tw[1].
    constexpr bool NO_STW = XcorNoStw<E, S>::v;
    extern __shared__ float2 dsm[];
    float2* stw = dsm;
    float2* sth = dsm + (NO_STW ? 0 : M);
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        if (!NO_STW) stw[k] = a.tw[k];
        if (k > 0) {
            const int h = 1 << (31 - __clz(k));
            sth[k] = a.tw[(k - h) * (M / h)];
        }
    }
    const float2 tw1 = a.tw[1];
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    if (item >= n_items) return;
    // trial-major: the warps of a CTA take consecutive pairs of one trial (pairs of one row
    // share its spectrum in L1; one trial's spectra stay in L2 while all pairs read them)
    const long long p = item % a.P;
    const long long trial = c->pushed + first_trial + item / a.P;
    if (trial < 0) return;  // window not yet full
    int i, j;
    unpack_pair(p, a.n, i, j);
    const int slot = (int)(trial % a.slots);
    const float2* Zi = a.spec + ((size_t)slot * a.n + i) * (M + 1);
    const float2* Zj = a.spec + ((size_t)slot * a.n + j) * (M + 1);
    // Y[k] = E[k] + i O[k], E = (P[k] + conj P[M-k]) / 2, O = (P[k] - conj P[M-k]) e^{+2 pi i k/L} / 2
    auto prod = [&](int k) -> float2 {
        const float2 pk = cmul(Zi[k], cconj(Zj[k]));
        const float2 pm = cconj(cmul(Zi[M - k], cconj(Zj[M - k])));
        const float2 e = make_float2(0.5f * __fadd_rn(pk.x, pm.x), 0.5f * __fadd_rn(pk.y, pm.y));
        const float2 dd = csub(pk, pm);
        float2 w;  // e^{+2 pi i k / L}
        if (!NO_STW)
            w = cconj(stw[k]);
        else
            w = cconj((k & 1) ? cmul(sth[M / 2 + (k >> 1)], tw1) : sth[M / 2 + (k >> 1)]);
        const float2 o = cmul(make_float2(0.5f * dd.x, 0.5f * dd.y), w);
        return make_float2(__fsub_rn(e.x, o.y), __fadd_rn(e.y, o.x));
    };
    constexpr int bits = 5 + (E >= 2) + (E >= 4) + (E >= 8) + (E >= 16) + (E >= 32) + (E >= 64);  // log2 MS
    float best = -INFINITY;
    int best_tau = 0;
    const float invM = 1.0f / (float)M;
    const int L = 2 * M;
    float2* tb = sth + M + (size_t)wib * (MS + MS / E);
#pragma unroll 1
    for (int half = 0; half < (1 << S); ++half) {
        float2 x[E];
        if (S == 0) {
            // one pass: the products P[k] = Z_i[k] conj(Z_j[k]) of this lane's k into the warp's
            // transpose buffer (free until the transpose), P[M] (the Nyquist bin) in lane 0's
            // register; then the even/odd split with P[M - k] from the buffer, so each spectrum
            // element is loaded from memory once
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int k = lane + 32 * r;
                tb[k] = cmul(Zi[k], cconj(Zj[k]));
            }
            const float2 pnyq = lane == 0 ? cmul(Zi[M], cconj(Zj[M])) : make_float2(0.f, 0.f);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int k = lane + 32 * r;
                const float2 pk = tb[k];
                const float2 pm = cconj(k == 0 ? pnyq : tb[M - k]);
                const float2 e2 = make_float2(0.5f * __fadd_rn(pk.x, pm.x), 0.5f * __fadd_rn(pk.y, pm.y));
                const float2 dd = csub(pk, pm);
                float2 w;  // e^{+2 pi i k / L}
                if (!NO_STW)
                    w = cconj(stw[k]);
                else
                    w = cconj((k & 1) ? cmul(sth[M / 2 + (k >> 1)], tw1) : sth[M / 2 + (k >> 1)]);
                const float2 o = cmul(make_float2(0.5f * dd.x, 0.5f * dd.y), w);
                x[r] = make_float2(__fsub_rn(e2.x, o.y), __fadd_rn(e2.y, o.x));
            }
        }
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = lane + 32 * r;
            if (S == 0) {
                // formed above
            } else if (S == 1) {  // first stage, span MS: top half u + v, bottom half (u - v) e^{+2 pi i e / M}
                const float2 u = prod(e), v = prod(e + MS);
                x[r] = half == 0 ? cadd(u, v) : cmul(csub(u, v), cconj(sth[MS + e]));
            } else {  // stages of span 2 MS (top: half < 2) and MS (second split: half odd)
                const float2 p0 = prod(e), p1 = prod(e + MS), p2 = prod(e + 2 * MS), p3 = prod(e + 3 * MS);
                float2 t0, t1;
                if (half < 2) {
                    t0 = cadd(p0, p2);
                    t1 = cadd(p1, p3);
                } else {
                    t0 = cmul(csub(p0, p2), cconj(sth[2 * MS + e]));
                    t1 = cmul(csub(p1, p3), cconj(sth[3 * MS + e]));
                }
                x[r] = (half & 1) == 0 ? cadd(t0, t1) : cmul(csub(t0, t1), cconj(sth[MS + e]));
            }
        }
        // inverse transform (e^{+2 pi i ...}), decimation in frequency
#pragma unroll
        for (int h = MS / 2; h >= 32; h >>= 1) {  // partner in this lane's registers
            const int hr = h / 32;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                if ((r % (2 * hr)) >= hr) continue;
                const int e = lane + 32 * r;
                const float2 u = x[r], v = x[r + hr];
                const float2 w = cconj(sth[h + e % h]);
                x[r] = cadd(u, v);
                x[r + hr] = cmul(csub(u, v), w);
            }
        }
#pragma unroll
        for (int h = 16; h >= E; h >>= 1) {  // partner in lane ^ h (E <= 16 only)
            const bool upper = (lane & h) != 0;
            const float2 w = cconj(sth[h + lane % h]);
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float2 mine = x[r];
                const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, mine.x, h),
                                                 __shfl_xor_sync(0xffffffffu, mine.y, h));
                x[r] = upper ? cmul(csub(other, mine), w) : cadd(mine, other);
            }
        }
        // transpose: lane l takes elements l E + q, q < E
        __syncwarp();  // the previous half's reads of the buffer are done
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = lane + 32 * r;
            tb[e + e / E] = x[r];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < E; ++q) x[q] = tb[lane * (E + 1) + q];
        constexpr int HL = E / 2 < 16 ? E / 2 : 16;  // first span inside the lane after the transpose
#pragma unroll
        for (int h = HL; h >= 1; h >>= 1) {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                if ((q % (2 * h)) >= h) continue;
                const float2 u = x[q], v = x[q + h];
                const float2 w = cconj(sth[h + q % h]);  // (l E + q) mod h = q mod h
                x[q] = cadd(u, v);
                x[q + h] = cmul(csub(u, v), w);
            }
        }
        // position e holds this block's output bitrev(e), i.e. y[m] with m = 2^S bitrev(e) +
        // bitrev_S(block); r[2m] = Re y[m] / M, r[2m+1] = Im y[m] / M
        const int boff = S == 2 ? ((half & 1) << 1) | (half >> 1) : half;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int m = (bitrev(lane * E + r, bits) << S) + boff;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const int idx = 2 * m + part;
                const int tau = idx <= a.N - 1 ? idx : (idx >= L - (a.N - 1) ? idx - L : INT_MIN);
                if (tau == INT_MIN) continue;
                const float v = __fmul_rn(part ? x[r].y : x[r].x, invM);
                if (better(v, tau, best, best_tau)) {
                    best = v;
                    best_tau = tau;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int ot = __shfl_xor_sync(0xffffffffu, best_tau, o);
        if (better(ov, ot, best, best_tau)) {
            best = ov;
            best_tau = ot;
        }
    }
    if (lane == 0) {
        const float ei = a.energy[(size_t)slot * a.n + i], ej = a.energy[(size_t)slot * a.n + j];
        const float den = __fmul_rn(sqrtf(ei), sqrtf(ej));
        float v = 0.f;
        int lag = 0;
        if (den > 0.f) {
            v = __fdiv_rn(best, den);
            lag = best_tau;
        }
        a.vals[(size_t)slot * a.P + p] = v;
        if (trial == c->pushed + a.count - 1) a.lag[p] = lag;
    }
}

template <int E, int S>
__global__ void __launch_bounds__(256) k_xcor_pairs_reg(XcorArgs a, long long n_items, long long first_trial,
                                                       int n_trials) {
    xcor_pairs_reg<E, S>(a, n_items, first_trial, n_trials);
}
template <int E, int S>
__global__ void __launch_bounds__(256, XcorMinBlocks<E, S>::v) k_xcor_pairs_reg_mb(XcorArgs a, long long n_items,
                                                                                 long long first_trial, int n_trials) {
    xcor_pairs_reg<E, S>(a, n_items, first_trial, n_trials);
}

// ------------------------------------------------------------------ network update
__global__ void k_xcor_update(XcorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    df32 acc;
    if (a.mode == 0) {
        acc = df_make(a.acc[p], a.acc[a.P + p]);
        const long long tn = end - 1;
        acc = df_add_f(acc, a.vals[(size_t)(tn % a.slots) * a.P + p]);
        if (a.W > 0 && tn >= a.W) acc = df_add_f(acc, -a.vals[(size_t)((tn - a.W) % a.slots) * a.P + p]);
    } else {
        acc = df_make(0.f, 0.f);
        for (long long k = start; k < end; ++k) acc = df_add_f(acc, a.vals[(size_t)(k % a.slots) * a.P + p]);
    }
    a.acc[p] = acc.hi;
    a.acc[a.P + p] = acc.lo;
    if (a.finalize) a.net[p] = __fmul_rn(df_to_f(acc), 1.0f / (float)K);
}

}  // namespace

template <int E, int S>
cudaError_t launch_pairs_reg(const XcorArgs& a, long long items, long long first, int n_trials, cudaStream_t st) {
    constexpr int MS = 32 * E;
    // twiddle tables (2 M, or M without stw) and 8 warps x (MS + MS / E) transpose slots
    const int dyn = ((XcorNoStw<E, S>::v ? 1 : 2) * (MS << S) + 8 * (MS + MS / E)) * (int)sizeof(float2);
    const unsigned grid = (unsigned)((items + 7) / 8);
    if constexpr (XcorMinBlocks<E, S>::v > 0) {
        cudaError_t e = cudaFuncSetAttribute(k_xcor_pairs_reg_mb<E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        k_xcor_pairs_reg_mb<E, S><<<grid, 256, dyn, st>>>(a, items, first, n_trials);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_xcor_pairs_reg<E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        k_xcor_pairs_reg<E, S><<<grid, 256, dyn, st>>>(a, items, first, n_trials);
    }
    return cudaGetLastError();
}

cudaError_t launch_xcor_spectra(const XcorArgs& a, cudaStream_t st) {
    const long long warps = (long long)(a.count - a.write_from) * a.n;
    if (warps <= 0) return cudaSuccess;
    const int wpb = a.L / 2 > 4096 ? 2 : 4;  // M float2 per warp: 128 KB per block at M = 8192
    const size_t sm = (size_t)wpb * (a.L / 2) * sizeof(float2);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_xcor_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_xcor_spectra<<<(unsigned)((warps + wpb - 1) / wpb), wpb * 32, sm, st>>>(a);
    return cudaGetLastError();
}

// mode 1: every trial of the window; mode 0: the newest trial only.
cudaError_t launch_xcor_pairs(const XcorArgs& a, cudaStream_t st) {
    // trials relative to ctrl->pushed: newest = count - 1; window = [count - K, count)
    int n_trials;
    long long first;
    if (a.mode == 0) {
        n_trials = 1;
        first = a.count - 1;
    } else {
        n_trials = a.W;  // full mode always has W >= 1; the kernel clamps below
        first = a.count - a.W;
    }
    const long long items = a.P * n_trials;
    const int M = a.L / 2;
    // register form for M = 64 .. 8192 (8 warps per block), shared-memory form otherwise
    switch (M) {
        case 64: return launch_pairs_reg<2, 0>(a, items, first, n_trials, st);
        case 128: return launch_pairs_reg<4, 0>(a, items, first, n_trials, st);
        case 256: return launch_pairs_reg<8, 0>(a, items, first, n_trials, st);
        case 512: return launch_pairs_reg<16, 0>(a, items, first, n_trials, st);
        case 1024: return launch_pairs_reg<32, 0>(a, items, first, n_trials, st);
        case 2048: return launch_pairs_reg<64, 0>(a, items, first, n_trials, st);
        case 4096: return launch_pairs_reg<64, 1>(a, items, first, n_trials, st);
        case 8192: return launch_pairs_reg<64, 2>(a, items, first, n_trials, st);
        default: break;
    }
    const int wpb = 4;
    const size_t sm = (size_t)wpb * M * sizeof(float2);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_xcor_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_xcor_pairs<<<(unsigned)((items + wpb - 1) / wpb), wpb * 32, sm, st>>>(a, items, first, n_trials);
    return cudaGetLastError();
}

cudaError_t launch_xcor_update(const XcorArgs& a, cudaStream_t st) {
    k_xcor_update<<<(unsigned)((a.P + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}
