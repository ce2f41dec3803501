// k_nonlin.cu - the non-linear pair sums of the mixed-precision full-window path.
//
// The phase-lag metrics need sums that are not contractions (Supplementary Information 1):
//   PLI = |sum sign(Im CSD)| / K, USPLI from the same integer,
//   WPLI = |sum Im| / sum |Im|,  DSWPLI = ((sum Im)^2 - sum Im^2) / ((sum |Im|)^2 - sum Im^2),
// with Im = Im(X_i X_j*). Here they run on the CUDA cores beside the tensor-core linear
// sums (k_herk_tc.cu), which produce COH, IMAGCOHY and PLV. Im and its exact sign come from
// Kahan's 2x2 determinant (terms.cuh), so the sign counts equal those of exact arithmetic
// on the stored FP32 spectra.
//
// Sums. The signs are tallied as counts of positive and of negative terms in FP32 (exact
// integers below 2^24 trials). Im, |Im| and Im^2 are summed in FP32 over chunks of NK
// trials and each chunk's partial sums are added to double-word window sums; the debiased
// differences x^2 - s are then evaluated in double words with the exact square of their
// leading word (df_sq_minus). The FP32 chunk sums leave each of (sum Im)^2, (sum |Im|)^2
// and sum Im^2 off by up to ~m u (sum |Im|)^2 (m <= NK terms per chunk, u = 2^-24), so
// DSWPLI is off by up to ~6 m u (sum |Im|)^2 / ((sum |Im|)^2 - sum Im^2): small except
// where one term dominates a short window. Where at most one term of the window is
// nonzero both differences are exactly 0 (sum_{k != l} of products), and DSWPLI is 0, as
// the definition's zero denominator gives; the counts decide this exactly.
//
// Accumulator mode (ACC): the window sums of each bin are stored into the streaming
// accumulators (sum Im, sum |Im|, sum Im^2 as double words, the sign count) of the tile pairs
// of a list; this is the drift re-sum of a mixed-precision streaming session, whose linear
// sums come from the tensor cores. Here every term is added exactly as the streaming update
// adds it (Im, |Im| and the exact two-product of Im^2 into double words, renormalized every
// chunk): the update later subtracts a trial's terms from these sums, and sums rounded to
// FP32 would keep that trial's rounding (a residue of the size of the largest trial of the
// re-summed window) after it has left.
//
// Work split: a CTA of 128 threads takes one 32 x 32 tile pair and a group of bins; each
// thread holds a 2 x 4 register tile of pairs (rows 2 rg, 2 rg + 1; columns 4 cg .. 4 cg + 3),
// so every staged spectrum value feeds 4 or 2 pairs per load. Row spectra are staged as
// (a, a, b, b) and (-a, -a) so that they load straight into packed FP32x2 operands; column
// spectra as planes of a and b. Per pair and trial the loop issues the determinant (two
// packed FMAs, a packed multiply and FMA for two pairs), two compare-to-float tallies, one
// absolute add and a packed add and FMA for two pairs; it is unrolled four trials deep so
// that the shared-memory loads of later trials cover the latency of earlier ones. The next
// chunk of trials is copied by cp.async while the current one is computed, two adjacent
// nodes (16 bytes) per copy when the node count is even. Each bin's metrics are formed for
// two pairs per packed operation (CUDA's built-in FP32x2 operations, which round each lane
// like the scalar operation and are never contracted), bit for bit as the scalar finalize.
#include "df32.cuh"
#include "fc_internal.h"
#include "pair_common.cuh"
#include "terms.cuh"

#include <type_traits>

namespace {

using namespace fcpair;

constexpr int NK = 36;         // most trials per staged chunk (and per FP32 partial sum)
constexpr int NL_THREADS = 128;

// 1.0f if x > 0 (resp. x < 0) else 0.0f: one exact compare each.
__device__ __forceinline__ float gt0(float x) {
    float r;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lt0(float x) {
    float r;
    asm("set.lt.f32.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// x^2 - s for two lanes of double words x = xh + xl, s = sh + sl: the same correctly rounded
// steps as df_sq_minus per lane (exact square of the leading word by FMA, the cross term
// 2 xh xl, the two differences and their sum), on the packed FP32 pipe. The built-in packed
// operations round like their scalar counterparts and are never contracted.
__device__ __forceinline__ float2 sq_minus2(float2 xh, float2 xl, float2 sh, float2 sl) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 nph = __fmul2_rn(__fmul2_rn(xh, m1), xh);        // -fl(xh^2)
    float2 pl = __ffma2_rn(xh, xh, nph);                          // xh^2 - fl(xh^2), exact
    pl = __ffma2_rn(__fadd2_rn(xh, xh), xl, pl);                  // + 2 xh xl
    const float2 d1 = __fadd2_rn(nph, sh);                        // -(fl(xh^2) - sh)
    const float2 d2 = __ffma2_rn(sl, m1, pl);                     // pl - sl
    return __ffma2_rn(d1, m1, d2);                                // (fl(xh^2) - sh) + (pl - sl)
}

struct NlSmem {
    alignas(16) float2 raw[NK][2 * FC_T];  // the next chunk's spectra as copied (row tile, column tile)
    float4 rowv[NK][FC_T];  // row node i: (a, a, b, b)
    float2 rown[NK][FC_T];  // row node i: (-a, -a)
    float4 cola[NK][FC_T / 4];  // column nodes: a, four per vector
    float4 colb[NK][FC_T / 4];  //                b
    float band[4][FC_T][FC_T];  // band sums of PLI, USPLI, WPLI, DSWPLI per pair
};

template <bool ACC>
__global__ void __launch_bounds__(NL_THREADS, 3) k_nonlin(PairArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    if (K <= 0) return;
    const KConst kc = make_kconst(K);
    extern __shared__ __align__(16) unsigned char nl_smem_raw[];
    NlSmem& sm = *reinterpret_cast<NlSmem*>(nl_smem_raw);

    // bin group g: selected bins fsel0 + g group_bins .. (bins outside the selected band take
    // no part in the average and are not computed)
    const int tp = ACC ? a.tp_list[a.tp0 + blockIdx.x] : blockIdx.x, g = blockIdx.y;
    const int fa = a.fsel0 + g * a.group_bins, fb = min(a.fsel1, fa + a.group_bins);
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x, rg = tid >> 3, cg = tid & 7;
    const int li0 = 2 * rg, lj0 = 4 * cg;
    unsigned vmask = 0;  // bit 4 r + q: pair (li0 + r, lj0 + q)
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = ta * FC_T + li0 + r, gj = tb * FC_T + lj0 + q;
            if (gi < a.n && gj < a.n && (ta != tb || lj0 + q > li0 + r)) vmask |= 1u << (4 * r + q);
        }
    for (int e = tid; e < 4 * FC_TT; e += NL_THREADS) (&sm.band[0][0][0])[e] = 0.f;

    // Chunks of NK trials of the bins fa .. fb - 1 in order; the copy of chunk c + 1
    // (cp.async, asynchronous) runs while chunk c is computed. For an even node count a
    // thread copies and converts node pairs (16 bytes per copy): pair lp of the two tiles'
    // 32, trials kp0 + 4 q, each warp on one tile; the ring is the session's own device
    // allocation (256-byte aligned) and every (slot, bin) row starts at an even node offset,
    // so each pair starts on 16 bytes. For an odd node count: node l = tid % 64, trials
    // tid / 64 + 2 q.
    const bool pairs = (a.n & 1) == 0;
    const int lp = ((tid >> 5) & 1) * (FC_T / 2) + (tid & 15), kp0 = ((tid >> 6) << 1) | ((tid >> 4) & 1);
    const int l_node = pairs ? 2 * lp : tid & 63, kk0 = pairs ? kp0 : tid >> 6;
    const int node = l_node < FC_T ? ta * FC_T + l_node : tb * FC_T + l_node - FC_T;
    const bool node_ok = node < a.n;  // even count: node + 1 < n as well
    const int nchunk = (K + NK - 1) / NK;
    const int csize = (K + nchunk - 1) / nchunk;  // balanced chunks of at most NK trials
    const int slot_start = (int)(start % a.slots);
    constexpr int PER = NK * 2 * FC_T / NL_THREADS;  // elements per thread and chunk
    auto issue_copy = [&](int f, int k0) {
        const int kn = min(csize, K - k0);
        int slot = slot_start + k0 + kk0;
        while (slot >= a.slots) slot -= a.slots;
        const float2* src = a.ring + (size_t)f * a.n + node;
        const size_t slot_stride = (size_t)a.B * a.n;
        if (pairs) {
#pragma unroll
            for (int q = 0; q < PER / 2; ++q) {
                const int kk = kk0 + 4 * q;
                if (kk < kn && node_ok) cp_async16(&sm.raw[kk][l_node], src + (size_t)slot * slot_stride);
                slot += 4;
                if (slot >= a.slots) slot -= a.slots;
            }
        } else {
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int kk = kk0 + 2 * q;
                if (kk < kn && node_ok) cp_async8(&sm.raw[kk][l_node], src + (size_t)slot * slot_stride);
                slot += 2;
                if (slot >= a.slots) slot -= a.slots;
            }
        }
        cp_async_commit();
    };
    if (fa < fb) issue_copy(fa, 0);

    for (int f = fa; f < fb; ++f) {
        // window sums, packed pair q = 2 r + h covers pairs (li0 + r, lj0 + 2h + {0, 1});
        // pos / neg: counts of positive / negative terms (exact integers in FP32)
        float2 pos[4], neg[4], imh[4], iml[4], abh[4], abl[4], sqh[4], sql[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            pos[q] = neg[q] = imh[q] = iml[q] = abh[q] = abl[q] = sqh[q] = sql[q] = make_float2(0.f, 0.f);
        // nodes with a tiny component somewhere in the window (flags of the per-node sums
        // kernel) take the FP64 branch; bins without one (the rule) run a loop without it
        // (no flags given: every node takes it)
        auto tiny_at = [&](int node) { return a.tiny ? a.tiny[(size_t)f * a.n + min(node, a.n - 1)] != 0 : true; };
        unsigned tmask = 0;  // bits 0, 1: rows li0, li0 + 1; bits 2 .. 5: columns lj0 .. lj0 + 3
#pragma unroll
        for (int r = 0; r < 2; ++r) tmask |= tiny_at(ta * FC_T + li0 + r) ? 1u << r : 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) tmask |= tiny_at(tb * FC_T + lj0 + q) ? 4u << q : 0u;
        const bool bin_tiny = __syncthreads_or(tmask ? 1 : 0) != 0;
        for (int ci = 0; ci < nchunk; ++ci) {
            const int k0 = ci * csize;
            const int kn = min(csize, K - k0);
            cp_async_wait_all();
            __syncthreads();  // the chunk has landed; every thread is done with the previous one
            if (pairs) {
#pragma unroll
                for (int q = 0; q < PER / 2; ++q) {
                    const int kk = kk0 + 4 * q;
                    if (kk >= kn) break;  // trials past the chunk are never read
                    // a node past n is converted from whatever the buffer holds: its pairs are
                    // masked out and never stored
                    const float4 X = *reinterpret_cast<const float4*>(&sm.raw[kk][l_node]);
                    if (l_node < FC_T) {
                        sm.rowv[kk][l_node] = make_float4(X.x, X.x, X.y, X.y);
                        sm.rowv[kk][l_node + 1] = make_float4(X.z, X.z, X.w, X.w);
                        *reinterpret_cast<float4*>(&sm.rown[kk][l_node]) = make_float4(-X.x, -X.x, -X.z, -X.z);
                    } else {
                        *reinterpret_cast<float2*>(reinterpret_cast<float*>(sm.cola[kk]) + l_node - FC_T) = make_float2(X.x, X.z);
                        *reinterpret_cast<float2*>(reinterpret_cast<float*>(sm.colb[kk]) + l_node - FC_T) = make_float2(X.y, X.w);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int kk = kk0 + 2 * q;
                    float2 X = make_float2(0.f, 0.f);
                    if (kk < kn && node_ok) X = sm.raw[kk][l_node];
                    if (l_node < FC_T) {
                        sm.rowv[kk][l_node] = make_float4(X.x, X.x, X.y, X.y);
                        sm.rown[kk][l_node] = make_float2(-X.x, -X.x);
                    } else {
                        reinterpret_cast<float*>(sm.cola[kk])[l_node - FC_T] = X.x;
                        reinterpret_cast<float*>(sm.colb[kk])[l_node - FC_T] = X.y;
                    }
                }
            }
            __syncthreads();  // converted; the raw buffer is free again
            // start copying the next chunk (this bin's or the next's)
            if (ci + 1 < nchunk)
                issue_copy(f, k0 + csize);
            else if (f + 1 < fb)
                issue_copy(f + 1, 0);
            if (!vmask) continue;
            float2 pim[4], pab[4], psq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) pim[q] = pab[q] = psq[q] = make_float2(0.f, 0.f);
            auto chunk = [&](auto tiny_c) {
                constexpr bool TINY = decltype(tiny_c)::value;
#pragma unroll 4
                for (int kk = 0; kk < kn; ++kk) {
                    const float4 ca = sm.cola[kk][cg], cb = sm.colb[kk][cg];
                    const float2 aj[2] = {make_float2(ca.x, ca.y), make_float2(ca.z, ca.w)};
                    const float2 bj[2] = {make_float2(cb.x, cb.y), make_float2(cb.z, cb.w)};
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const float4 rv = sm.rowv[kk][li0 + r];
                        const float2 rn = sm.rown[kk][li0 + r];
                        const float2 ai = make_float2(rv.x, rv.y), bi = make_float2(rv.z, rv.w);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int q = 2 * r + h;
                            float2 im = kahan_im2(bi, ai, rn, aj[h], bj[h]);
                            if (TINY) {
                                int s0 = sign_of(im.x), s1 = sign_of(im.y);
                                if (tmask & ((1u << r) | (4u << (2 * h)))) im_sign_fp64(rv.x, rv.z, aj[h].x, bj[h].x, im.x, s0);
                                if (tmask & ((1u << r) | (8u << (2 * h)))) im_sign_fp64(rv.x, rv.z, aj[h].y, bj[h].y, im.y, s1);
                                pos[q] = add2(pos[q], make_float2(s0 > 0 ? 1.f : 0.f, s1 > 0 ? 1.f : 0.f));
                                neg[q] = add2(neg[q], make_float2(s0 < 0 ? 1.f : 0.f, s1 < 0 ? 1.f : 0.f));
                            } else {
                                pos[q] = add2(pos[q], make_float2(gt0(im.x), gt0(im.y)));
                                neg[q] = add2(neg[q], make_float2(lt0(im.x), lt0(im.y)));
                            }
                            if constexpr (ACC) {
                                // the streaming update's own terms, exactly: Im, |Im| and the
                                // exact two-product of Im^2 into the double-word window sums
                                acc2_f_lazy(imh[q], iml[q], im);
                                acc2_f_lazy(abh[q], abl[q], make_float2(fabsf(im.x), fabsf(im.y)));
                                float2 p2, e2;
                                two_prod(im.x, im.x, p2.x, e2.x);
                                two_prod(im.y, im.y, p2.y, e2.y);
                                acc2_d_lazy(sqh[q], sql[q], p2, e2);
                            } else {
                                pab[q] = make_float2(__fadd_rn(pab[q].x, fabsf(im.x)), __fadd_rn(pab[q].y, fabsf(im.y)));
                                pim[q] = add2(pim[q], im);
                                psq[q] = fma2(im, im, psq[q]);
                            }
                        }
                    }
                }
            };
            if (bin_tiny)
                chunk(std::true_type{});
            else
                chunk(std::false_type{});
            if constexpr (ACC) {
                // per-term lazy sums: renormalized every chunk (at most NK terms each)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    renorm2(imh[q], iml[q]);
                    renorm2(abh[q], abl[q]);
                    renorm2(sqh[q], sql[q]);
                }
            } else {
                // the chunk's partial sums into the double-word window sums (lazy:
                // renormalized once per bin)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc2_f_lazy(imh[q], iml[q], pim[q]);
                    acc2_f_lazy(abh[q], abl[q], pab[q]);
                    acc2_f_lazy(sqh[q], sql[q], psq[q]);
                }
            }
        }
        if (vmask) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                renorm2(imh[q], iml[q]);
                renorm2(abh[q], abl[q]);
                renorm2(sqh[q], sql[q]);
            }
            if constexpr (ACC) {
                // accumulator block of (tile pair, bin): planes 2k, 2k + 1 = hi, lo of field k
                // (1 sum Im, 4 sum |Im|, 5 sum Im^2), plane 12 the sign count
                float* blk = a.acc + ((size_t)(a.acc_by_pos ? (int)blockIdx.x : tp) * a.B + f) * FC_BLOCK_WORDS;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int w0 = (li0 + r) * FC_T + lj0, q0 = 2 * r, q1 = 2 * r + 1;
                    auto put = [&](int k, const float2* h, const float2* l) {
                        __stcs(reinterpret_cast<float4*>(blk + (2 * k) * FC_TT + w0),
                               make_float4(h[q0].x, h[q0].y, h[q1].x, h[q1].y));
                        __stcs(reinterpret_cast<float4*>(blk + (2 * k + 1) * FC_TT + w0),
                               make_float4(l[q0].x, l[q0].y, l[q1].x, l[q1].y));
                    };
                    put(1, imh, iml);
                    put(4, abh, abl);
                    put(5, sqh, sql);
                    __stcs(reinterpret_cast<int4*>(blk + 12 * FC_TT + w0),
                           make_int4((int)pos[q0].x - (int)neg[q0].x, (int)pos[q0].y - (int)neg[q0].y,
                                     (int)pos[q1].x - (int)neg[q1].x, (int)pos[q1].y - (int)neg[q1].y));
                }
            } else {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float4 acc[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) acc[m] = *reinterpret_cast<float4*>(&sm.band[m][li0 + r][lj0]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // two pairs (columns lj0 + 2h, + 1) per packed operation; every lane takes
                        // the same correctly rounded steps as the scalar finalize of a session
                        const int q = 2 * r + h;
                        const float2 m1 = make_float2(-1.f, -1.f);
                        const float2 nz = __fadd2_rn(pos[q], neg[q]);  // nonzero terms (exact)
                        float2 pli, uspli;
                        if (K <= 4096) {
                            // S = pos - neg and S^2 - K are exact in FP32 while |S| <= K <= 4096
                            const float2 sg = __ffma2_rn(neg[q], m1, pos[q]);
                            pli = make_float2(__fmul_rn(fabsf(sg.x), kc.inv_K), __fmul_rn(fabsf(sg.y), kc.inv_K));
                            uspli = __fmul2_rn(__ffma2_rn(sg, sg, f2(-(float)K)), f2(kc.inv_KK1));
                        } else {
                            float* pl = &pli.x;
                            float* us = &uspli.x;
#pragma unroll
                            for (int y = 0; y < 2; ++y) {
                                const int sg = (int)(y ? pos[q].y : pos[q].x) - (int)(y ? neg[q].y : neg[q].x);
                                const float usn = K <= 46340 ? (float)(sg * sg - K) : (float)((long long)sg * sg - K);
                                pl[y] = __fmul_rn((float)abs(sg), kc.inv_K);
                                us[y] = __fmul_rn(usn, kc.inv_KK1);
                            }
                        }
                        const float2 fsab = __fadd2_rn(abh[q], abl[q]);  // double words to float
                        const float2 fsim = __fadd2_rn(imh[q], iml[q]);
                        const float2 wpli = make_float2(fsab.x > 0.f ? __fdividef(fabsf(fsim.x), fsab.x) : 0.f,
                                                        fsab.y > 0.f ? __fdividef(fabsf(fsim.y), fsab.y) : 0.f);
                        // (sum Im)^2 - sum Im^2 and (sum |Im|)^2 - sum Im^2 from the double words
                        const float2 num = sq_minus2(imh[q], iml[q], sqh[q], sql[q]);
                        const float2 den = sq_minus2(abh[q], abl[q], sqh[q], sql[q]);
                        // two or more nonzero terms, else 0 (the definition's zero denominator)
                        const float2 dsw = make_float2(nz.x > 1.f && den.x != 0.f ? __fdividef(num.x, den.x) : 0.f,
                                                       nz.y > 1.f && den.y != 0.f ? __fdividef(num.y, den.y) : 0.f);
                        auto add_lanes = [&](float4& v, float2 t) {
                            if (h == 0) {
                                const float2 u = __fadd2_rn(make_float2(v.x, v.y), t);
                                v.x = u.x;
                                v.y = u.y;
                            } else {
                                const float2 u = __fadd2_rn(make_float2(v.z, v.w), t);
                                v.z = u.x;
                                v.w = u.y;
                            }
                        };
                        add_lanes(acc[0], pli);
                        add_lanes(acc[1], uspli);
                        add_lanes(acc[2], wpli);
                        add_lanes(acc[3], dsw);
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) *reinterpret_cast<float4*>(&sm.band[m][li0 + r][lj0]) = acc[m];
                }
            }
        }
    }
    if (ACC || !vmask) return;
    const float invB = 1.0f / (float)(a.fsel1 - a.fsel0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int mi = m + 3;  // PLI .. DSWPLI among the seven spectral planes
        if (!(a.mask & (1u << (mi + 2)))) continue;
        float* dst = a.groups == 1 ? a.net_spec + (size_t)mi * a.P : a.partial + ((size_t)g * 7 + mi) * a.P;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int gi = ta * FC_T + li0 + r;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!(vmask & (1u << (4 * r + q)))) continue;
                const float v = sm.band[m][li0 + r][lj0 + q];
                dst[packed_index(gi, tb * FC_T + lj0 + q, a.n)] = a.groups == 1 ? __fmul_rn(v, invB) : v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_nonlinear_sums(const PairArgs& a, cudaStream_t st) {
    const int smem = (int)sizeof(NlSmem);
    cudaError_t e = cudaFuncSetAttribute(k_nonlin<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(a.ntp, a.groups);
    k_nonlin<false><<<grid, NL_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nonlinear_acc(const PairArgs& a, cudaStream_t st) {
    if (a.tp_count <= 0) return cudaSuccess;
    PairArgs b = a;
    b.finalize = 0;
    b.write_acc = 1;
    const int smem = (int)sizeof(NlSmem);
    cudaError_t e = cudaFuncSetAttribute(k_nonlin<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(b.tp_count, b.groups);
    k_nonlin<true><<<grid, NL_THREADS, smem, st>>>(b);
    return cudaGetLastError();
}

int nonlinear_ctas_per_sm() { return 3; }
