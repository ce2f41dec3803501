// k_nonlin.cu - the non-linear pair sums of the mixed-precision full-window path.
//
// The phase-lag metrics need sums that are not contractions (Supplementary Information 1):
//   PLI = |sum sign(Im CSD)| / K, USPLI from the same integer,
//   WPLI = |sum Im| / sum |Im|,  DSWPLI = ((sum Im)^2 - sum Im^2) / ((sum |Im|)^2 - sum Im^2),
// with Im = Im(X_i X_j*). Here they run on the CUDA cores beside the tensor-core linear
// sums (k_herk_tc.cu), which produce COH, IMAGCOHY and PLV. Im and its exact sign use the
// same term code as the exact path (terms.cuh). The sums run in FP32 over chunks of 16
// trials and each chunk's partial sums (Im, |Im|, Im^2) are promoted to double-word
// accumulators, so the debiased cancellation (sum Im)^2 - sum Im^2 is evaluated from
// FP64-class sums; the sign count is an exact int32.
//
// CTA: one 32 x 32 tile pair x a group of bins; thread: 4 adjacent pairs of the tile.
#include "df32.cuh"
#include "fc_internal.h"
#include "pair_common.cuh"
#include "terms.cuh"

#include <type_traits>

namespace {

using namespace fcpair;

constexpr int NK = 16;  // trials per staged chunk (and per FP32 partial sum)

__global__ void __launch_bounds__(256, 3) k_nonlin(PairArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    if (K <= 0) return;
    const KConst kc = make_kconst(K);

    const int tp = blockIdx.x, g = blockIdx.y;
    const int f0 = g * a.group_bins, f1 = min(a.B, f0 + a.group_bins);
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x, li = tid >> 3, lj0 = (tid & 7) * 4;
    const unsigned vmask = pair_mask(ta, tb, li, lj0, a.n);
    const int gi = ta * FC_T + li, gj0 = tb * FC_T + lj0;

    // planar: [trial][node] real parts, imaginary parts, tiny flags (two adjacent column
    // nodes load as one packed operand)
    __shared__ __align__(16) float sa[NK][2 * FC_T];
    __shared__ __align__(16) float sb[NK][2 * FC_T];
    __shared__ unsigned char stiny[NK][2 * FC_T];

    float band[7][4];
#pragma unroll
    for (int m = 0; m < 7; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) band[m][q] = 0.f;

    for (int f = f0; f < f1; ++f) {
        df32 s_im[4], s_sq[4], s_abs[4];
        int s_sg[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s_im[q] = s_sq[q] = s_abs[q] = df_make(0.f, 0.f);
            s_sg[q] = 0;
        }
        for (int k0 = 0; k0 < K; k0 += NK) {
            const int kn = min(NK, K - k0);
            __syncthreads();
            bool any_tiny = false;
            for (int e = tid; e < kn * 2 * FC_T; e += 256) {
                const int kk = e / (2 * FC_T), l = e % (2 * FC_T);
                const int node = l < FC_T ? ta * FC_T + l : tb * FC_T + l - FC_T;
                const long long trial = start + k0 + kk;
                float2 X = make_float2(0.f, 0.f);
                if (node < a.n) X = a.ring[((size_t)(trial % a.slots) * a.B + f) * a.n + node];
                sa[kk][l] = X.x;
                sb[kk][l] = X.y;
                const bool tn = node_tiny(X);
                stiny[kk][l] = tn ? 1 : 0;
                any_tiny |= tn;
            }
            // chunks without a tiny node (the rule) run a loop with no FP64 branch at all
            const bool chunk_tiny = __syncthreads_or(any_tiny ? 1 : 0) != 0;
            if (!vmask) continue;
            // FP32 partial sums of this chunk, two column pairs per packed lane pair
            float2 p_im[2], p_sq[2], p_abs[2], p_sqe[2], p_pos[2], p_neg[2];
#pragma unroll
            for (int h = 0; h < 2; ++h)
                p_im[h] = p_sq[h] = p_abs[h] = p_sqe[h] = p_pos[h] = p_neg[h] = make_float2(0.f, 0.f);
            auto chunk = [&](auto tiny_c) {
                constexpr bool TINY = decltype(tiny_c)::value;
                for (int kk = 0; kk < kn; ++kk) {
                    const float ai = sa[kk][li], bi = sb[kk][li];
                    const float2 bi2 = f2(bi), ai2 = f2(ai), nai2 = f2(-ai);
                    const bool ti = TINY && stiny[kk][li] != 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = FC_T + lj0 + 2 * h;
                        const float2 aj = *reinterpret_cast<const float2*>(&sa[kk][j]);
                        const float2 bj = *reinterpret_cast<const float2*>(&sb[kk][j]);
                        // Im(X_i X_j*) and its exact sign, as in pair_terms2 (terms.cuh)
                        float2 im = kahan_im2(bi2, ai2, nai2, aj, bj);
                        if (TINY) {
                            int sg0 = sign_of(im.x), sg1 = sign_of(im.y);
                            if (ti || stiny[kk][j]) im_sign_fp64(ai, bi, aj.x, bj.x, im.x, sg0);
                            if (ti || stiny[kk][j + 1]) im_sign_fp64(ai, bi, aj.y, bj.y, im.y, sg1);
                            s_sg[2 * h] += sg0;
                            s_sg[2 * h + 1] += sg1;
                        } else {
                            // sign tallies as exact small FP32 counts (at most NK per chunk)
                            p_pos[h] = add2(p_pos[h], make_float2(im.x > 0.f ? 1.f : 0.f, im.y > 0.f ? 1.f : 0.f));
                            p_neg[h] = add2(p_neg[h], make_float2(im.x < 0.f ? 1.f : 0.f, im.y < 0.f ? 1.f : 0.f));
                        }
                        p_abs[h] = make_float2(__fadd_rn(p_abs[h].x, fabsf(im.x)), __fadd_rn(p_abs[h].y, fabsf(im.y)));
                        p_im[h] = add2(p_im[h], im);
                        // im^2 as an exact two-product (t + r), scalar: the products feed additions;
                        // a lone nonzero term then gives (sum |Im|)^2 - sum Im^2 = 0 exactly
                        float2 t, r;
                        two_prod(im.x, im.x, t.x, r.x);
                        two_prod(im.y, im.y, t.y, r.y);
                        p_sq[h] = make_float2(__fadd_rn(p_sq[h].x, t.x), __fadd_rn(p_sq[h].y, t.y));
                        p_sqe[h] = add2(p_sqe[h], r);
                    }
                }
            };
            if (chunk_tiny)
                chunk(std::true_type{});
            else
                chunk(std::false_type{});
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float pim = (q & 1) ? p_im[q >> 1].y : p_im[q >> 1].x;
                const float psq = (q & 1) ? p_sq[q >> 1].y : p_sq[q >> 1].x;
                const float pse = (q & 1) ? p_sqe[q >> 1].y : p_sqe[q >> 1].x;
                const float pab = (q & 1) ? p_abs[q >> 1].y : p_abs[q >> 1].x;
                const float pps = (q & 1) ? p_pos[q >> 1].y : p_pos[q >> 1].x;
                const float png = (q & 1) ? p_neg[q >> 1].y : p_neg[q >> 1].x;
                s_sg[q] += (int)pps - (int)png;
                s_im[q] = df_add_f(s_im[q], pim);
                s_sq[q] = df_add_f(df_add_f(s_sq[q], psq), pse);
                s_abs[q] = df_add_f(s_abs[q], pab);
            }
        }
        if (vmask && f >= a.fsel0 && f < a.fsel1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!(vmask & (1u << q))) continue;
                // PLI, USPLI, WPLI, DSWPLI (metric slots 3..6)
                band[3][q] = __fadd_rn(band[3][q], __fmul_rn((float)abs(s_sg[q]), kc.inv_K));
                const float usn = K <= 46340 ? (float)(s_sg[q] * s_sg[q] - K)
                                             : (float)((long long)s_sg[q] * s_sg[q] - K);
                band[4][q] = __fadd_rn(band[4][q], __fmul_rn(usn, kc.inv_KK1));
                const float sim = df_to_f(s_im[q]);
                const float sab = df_to_f(s_abs[q]);
                band[5][q] = __fadd_rn(band[5][q], sab > 0.f ? __fdividef(fabsf(sim), sab) : 0.f);
                const float num = df_sq_minus(s_im[q], s_sq[q]);
                const float den = df_sq_minus(s_abs[q], s_sq[q]);
                band[6][q] = __fadd_rn(band[6][q], den != 0.f ? __fdividef(num, den) : 0.f);
            }
        }
    }
    if (vmask) write_band(a, g, band, gi, gj0, vmask, f1 - f0);
}

}  // namespace

cudaError_t launch_nonlinear_sums(const PairArgs& a, cudaStream_t st) {
    dim3 grid(a.ntp, a.groups);
    k_nonlin<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}
