// k_pairs.cu - pair x bin x trial accumulation of the spectral sums and the metrics.
//
// Methods 2.4: per trial the CSD and PSD are formed and their sums over the trials are
// kept ("running average"); the metric is computed from the sums for one half of the
// edge weights (undirected). Supplementary Information 1 defines the metrics.
//
// (the streaming add/subtract update lives in k_stream.cu)
// k_window  (full-window sums): the same sums over all K trials of the window from the
//           stored spectra, in registers, with the finalize in the epilogue; optionally
//           stores the accumulators (re-sum that resets the drift of the streaming state).
// k_node    per-node PSD sums (FP64) and 1/sqrt(PSD).
#include "df32.cuh"
#include "fc_internal.h"
#include "terms.cuh"
#include "pair_common.cuh"

#include <type_traits>

namespace {

using namespace fcpair;

// ------------------------------------------------------------------------------- node
__device__ __forceinline__ void node_elem(const NodeArgs& a, int e) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    if (e >= a.B * a.n) return;
    const int f = e / a.n, i = e % a.n;
    double s;
    if (a.mode == 0) {
        const long long t = c->pushed;  // the new trial
        const float2 Xn = a.ring[((size_t)(t % a.slots) * a.B + f) * a.n + i];
        s = a.psd[e] + ((double)Xn.x * Xn.x + (double)Xn.y * Xn.y);
        if (a.W > 0 && t >= a.W) {
            const float2 Xo = a.ring[((size_t)((t - a.W) % a.slots) * a.B + f) * a.n + i];
            s -= ((double)Xo.x * Xo.x + (double)Xo.y * Xo.y);
        }
    } else {
        const long long end = c->pushed + a.count;
        const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
        const float sc = c->in_scale;  // 0 for sessions (their ring holds prescaled spectra)
        s = 0.0;
        bool tiny = false;
        for (long long k = start; k < end; ++k) {
            float2 X = a.ring[((size_t)(k % a.slots) * a.B + f) * a.n + i];
            if (sc != 0.f) X = make_float2(__fmul_rn(X.x, sc), __fmul_rn(X.y, sc));
            s += (double)X.x * X.x + (double)X.y * X.y;
            tiny |= node_tiny(X);
        }
        if (a.tiny) a.tiny[e] = tiny ? 1 : 0;
    }
    a.psd[e] = s;
    a.inv_psd[e] = (s > 0.0) ? (float)(1.0 / sqrt(s)) : 0.f;
}

__global__ void k_node(NodeArgs a) { node_elem(a, blockIdx.x * blockDim.x + threadIdx.x); }

// Several sessions: their node-bin elements follow each other (node_prefix).
__global__ void k_node_batch(PreBatch b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.nsess <= 0 || e >= b.node_prefix[b.nsess]) return;
    int s = 0;
    while (s + 1 < b.nsess && e >= b.node_prefix[s + 1]) ++s;
    node_elem(b.nd[s], e - b.node_prefix[s]);
}

// ---------------------------------------------------------------- full-window sums
constexpr int WK = 16;     // trials staged per chunk
constexpr int NODE_W = 5;  // staged words per node: a, b, Re u, Im u, tiny flag

// Thread: row node li of tile ta against columns lj0 .. lj0 + 3 of tile tb, as two packed
// column pairs (FP32x2 lanes), double-float running sums per lane: lazy TwoSum updates
// (acc2_f_lazy / acc2_d_lazy) renormalized after every chunk of WK trials, which keeps the
// error of a sum of K terms within about (WK + 1) K u^2 of their summed magnitudes.
__global__ void __launch_bounds__(256, 2) k_window(PairArgs a, int bins_metric, float* bins_out) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const WinFacts wf = window_facts(c, a.W, a.count);
    const int K = wf.K;
    const KConst kc = make_kconst(K);

    const int tp = a.tp0 + blockIdx.x;
    const int g = blockIdx.y;
    const int f0 = g * a.group_bins;
    const int f1 = min(a.B, f0 + a.group_bins);
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x;
    const int li = tid >> 3, lj0 = (tid & 7) * 4;
    const unsigned vmask = pair_mask(ta, tb, li, lj0, a.n);
    const int gi = ta * FC_T + li, gj0 = tb * FC_T + lj0;

    // [trial][side: 0 row tile, 1 column tile][word][node], planar so that two adjacent
    // column nodes load as one packed operand
    __shared__ __align__(16) float sn[WK][2][NODE_W][FC_T];
    __shared__ float sinv[2][FC_T];

    float band[7][4];
#pragma unroll
    for (int m = 0; m < 7; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) band[m][q] = 0.f;

    for (int f = f0; f < f1; ++f) {
        float2 vh[2][FC_NFIELD], vl[2][FC_NFIELD];
        int s[4] = {0, 0, 0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < FC_NFIELD; ++k) vh[h][k] = vl[h][k] = make_float2(0.f, 0.f);
        if (tid < 64) {
            const int w = tid >> 5, l = tid & 31;
            const int node = (w ? tb : ta) * FC_T + l;
            sinv[w][l] = node < a.n ? a.inv_psd[(size_t)f * a.n + node] : 0.f;
        }
        for (int k0 = 0; k0 < K; k0 += WK) {
            const int kn = min(WK, K - k0);
            __syncthreads();
            bool any_tiny = false;
            const float sc = c->in_scale;  // 0 for sessions (their ring holds prescaled spectra)
            for (int e = tid; e < WK * 2 * FC_T; e += 256) {
                const int kk = e / (2 * FC_T), side = (e / FC_T) & 1, l = e % FC_T;
                const int node = (side ? tb : ta) * FC_T + l;
                float2 X = make_float2(0.f, 0.f);
                if (kk < kn && node < a.n)
                    X = a.ring[((size_t)((wf.start + k0 + kk) % a.slots) * a.B + f) * a.n + node];
                if (sc != 0.f) X = make_float2(__fmul_rn(X.x, sc), __fmul_rn(X.y, sc));
                const float2 u = phasor_of(X);
                sn[kk][side][0][l] = X.x;
                sn[kk][side][1][l] = X.y;
                sn[kk][side][2][l] = u.x;
                sn[kk][side][3][l] = u.y;
                const bool tn = node_tiny(X);
                sn[kk][side][4][l] = tn ? 1.f : 0.f;
                any_tiny |= tn;
            }
            // chunks without a tiny node (the rule) run a loop with no FP64 branch at all
            const bool chunk_tiny = __syncthreads_or(any_tiny ? 1 : 0) != 0;
            auto chunk = [&](auto tiny_c) {
                constexpr bool TINY = decltype(tiny_c)::value;
                for (int kk = 0; kk < kn; ++kk) {
                    const float (*r)[FC_T] = sn[kk][0];
                    const float (*cl)[FC_T] = sn[kk][1];
                    const RowConst rc = row_const(r[0][li], r[1][li], r[2][li], r[3][li], r[4][li] != 0.f);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = lj0 + 2 * h;
                        const float2 tj = *reinterpret_cast<const float2*>(&cl[4][j]);
                        const PairTerms2 t = pair_terms2<TINY>(rc, *reinterpret_cast<const float2*>(&cl[0][j]),
                                                         *reinterpret_cast<const float2*>(&cl[1][j]),
                                                         *reinterpret_cast<const float2*>(&cl[2][j]),
                                                         *reinterpret_cast<const float2*>(&cl[3][j]), tj.x != 0.f,
                                                         tj.y != 0.f);
                        acc2_f_lazy(vh[h][0], vl[h][0], t.re);
                        acc2_f_lazy(vh[h][1], vl[h][1], t.im);
                        acc2_f_lazy(vh[h][2], vl[h][2], t.ure);
                        acc2_f_lazy(vh[h][3], vl[h][3], t.uim);
                        acc2_f_lazy(vh[h][4], vl[h][4], make_float2(fabsf(t.im.x), fabsf(t.im.y)));
                        // im^2 as an exact two-product, scalar: the product feeds additions
                        float2 p2, e2;
                        two_prod(t.im.x, t.im.x, p2.x, e2.x);
                        two_prod(t.im.y, t.im.y, p2.y, e2.y);
                        acc2_d_lazy(vh[h][5], vl[h][5], p2, e2);
                        s[2 * h] += t.s0;
                        s[2 * h + 1] += t.s1;
                    }
                }
                // back to normalized double words once per chunk of WK terms
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int k = 0; k < FC_NFIELD; ++k) renorm2(vh[h][k], vl[h][k]);
            };
            if (vmask) {
                if (chunk_tiny)
                    chunk(std::true_type{});
                else
                    chunk(std::false_type{});
            }
        }
        __syncthreads();  // sinv visible
        if (vmask) {
            df32 v[4][FC_NFIELD];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k)
                    v[q][k] = (q & 1) ? df_make(vh[q >> 1][k].y, vl[q >> 1][k].y)
                                      : df_make(vh[q >> 1][k].x, vl[q >> 1][k].x);
            if (a.write_acc) {
                float* blk = a.acc + ((size_t)tp * a.B + f) * FC_BLOCK_WORDS;
                const int w0 = li * FC_T + lj0;
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k) {
                    float4 hq = make_float4(v[0][k].hi, v[1][k].hi, v[2][k].hi, v[3][k].hi);
                    float4 lq = make_float4(v[0][k].lo, v[1][k].lo, v[2][k].lo, v[3][k].lo);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k) * FC_TT + w0), hq);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k + 1) * FC_TT + w0), lq);
                }
                __stcs(reinterpret_cast<int4*>(blk + 12 * FC_TT + w0), make_int4(s[0], s[1], s[2], s[3]));
            }
            if (a.finalize || bins_out) {
                const float inv_i = sinv[0][li];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!(vmask & (1u << q))) continue;
                    float m[7];
                    finalize_bin(v[q], s[q], inv_i, sinv[1][lj0 + q], kc, m);
                    if (bins_out) {
                        bins_out[(size_t)f * a.P + packed_index(gi, gj0 + q, a.n)] = m[bins_metric - 2];
                    } else if (f >= a.fsel0 && f < a.fsel1) {
#pragma unroll
                        for (int mm = 0; mm < 7; ++mm) band[mm][q] = __fadd_rn(band[mm][q], m[mm]);
                    }
                }
            }
        }
        __syncthreads();  // sinv of the next bin is staged over this one
    }
    if (a.finalize && !bins_out && vmask) write_band(a, g, band, gi, gj0, vmask, f1 - f0);
}

// --------------------------------------------------- per-bin metrics from accumulators
__global__ void __launch_bounds__(256) k_bins_from_acc(PairArgs a, int metric, float* out) {
    const FcCtrl* c = a.ctrl;
    const long long t = c->pushed;
    const int K = (a.W > 0 && t > a.W) ? a.W : (int)t;
    const KConst kc = make_kconst(K);
    const int tp = blockIdx.x, f = blockIdx.y;
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x, li = tid >> 3, lj0 = (tid & 7) * 4;
    const unsigned vmask = pair_mask(ta, tb, li, lj0, a.n);
    if (!vmask) return;
    const int gi = ta * FC_T + li, gj0 = tb * FC_T + lj0;
    const float* blk = a.acc + ((size_t)tp * a.B + f) * FC_BLOCK_WORDS;
    const int w0 = li * FC_T + lj0;
    const float inv_i = a.inv_psd[(size_t)f * a.n + gi];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!(vmask & (1u << q))) continue;
        df32 v[FC_NFIELD];
        for (int k = 0; k < FC_NFIELD; ++k)
            v[k] = df_make(blk[(2 * k) * FC_TT + w0 + q], blk[(2 * k + 1) * FC_TT + w0 + q]);
        const int s = reinterpret_cast<const int*>(blk + 12 * FC_TT)[w0 + q];
        float m[7];
        finalize_bin(v, s, inv_i, a.inv_psd[(size_t)f * a.n + gj0 + q], kc, m);
        out[(size_t)f * a.P + packed_index(gi, gj0 + q, a.n)] = m[metric - 2];
    }
}

// ------------------------------------------------------------------ band reduce
__global__ void k_band_reduce(PairArgs a) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    if (a.ctrl->bad) return;
    const float invB = 1.0f / (float)(a.fsel1 - a.fsel0);
    for (int m = 0; m < 7; ++m) {
        if (!(a.mask & (1u << (m + 2)))) continue;
        float s = 0.f;
        for (int g = 0; g < a.groups; ++g) s = __fadd_rn(s, a.partial[((size_t)g * 7 + m) * a.P + p]);
        a.net_spec[(size_t)m * a.P + p] = __fmul_rn(s, invB);
    }
}

// --------------------------------------------------------------- debug / layout
__global__ void k_acc_field(const float* acc, const unsigned short* ta_, const unsigned short* tb_,
                            int B, int n, int field, double* out, long long P) {
    const int tp = blockIdx.x, f = blockIdx.y;
    const int ta = ta_[tp], tb = tb_[tp];
    for (int w = threadIdx.x; w < FC_TT; w += blockDim.x) {
        const int li = w / FC_T, lj = w % FC_T;
        const int gi = ta * FC_T + li, gj = tb * FC_T + lj;
        if (gi >= n || gj >= n || (ta == tb && lj <= li)) continue;
        const float* blk = acc + ((size_t)tp * B + f) * FC_BLOCK_WORDS;
        double v;
        if (field == FC_ACC_SIGN)
            v = (double)reinterpret_cast<const int*>(blk + 12 * FC_TT)[w];
        else
            v = (double)blk[(2 * field) * FC_TT + w] + (double)blk[(2 * field + 1) * FC_TT + w];
        out[(size_t)f * P + packed_index(gi, gj, n)] = v;
    }
}

__global__ void k_expand_dense(const float* packed, float* dense, int n, int antisym) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n) return;
    float v = 0.f;
    if (i < j) v = packed[packed_index(i, j, n)];
    else if (i > j) v = antisym ? -packed[packed_index(j, i, n)] : packed[packed_index(j, i, n)];
    dense[(size_t)i * n + j] = v;
}

__global__ void k_df_planes(const float* acc2, long long P, double* out) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) out[p] = (double)acc2[p] + (double)acc2[P + p];
}

}  // namespace

cudaError_t launch_node(const NodeArgs& a, cudaStream_t st) {
    const int total = a.B * a.n;
    k_node<<<(total + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_node_batch(const PreBatch& b, cudaStream_t st) {
    const int total = b.nsess > 0 ? b.node_prefix[b.nsess] : 0;
    if (total <= 0) return cudaSuccess;
    k_node_batch<<<(total + 255) / 256, 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_window_sums(const PairArgs& a, cudaStream_t st) {
    if (a.tp0 < 0 || a.tp_count < 0 || a.tp0 + (a.tp_count ? a.tp_count : a.ntp) > a.ntp) return cudaErrorInvalidValue;
    dim3 grid(a.tp_count ? a.tp_count : a.ntp, a.groups);
    k_window<<<grid, 256, 0, st>>>(a, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_bins_window(const PairArgs& a, int metric_index, float* out, cudaStream_t st) {
    dim3 grid(a.ntp, a.groups);
    PairArgs b = a;
    b.finalize = 0;
    b.write_acc = 0;
    b.tp0 = 0;
    b.tp_count = 0;
    k_window<<<grid, 256, 0, st>>>(b, metric_index, out);
    return cudaGetLastError();
}

cudaError_t launch_bins_from_acc(const PairArgs& a, int metric_index, float* out, cudaStream_t st) {
    dim3 grid(a.ntp, a.B);
    k_bins_from_acc<<<grid, 256, 0, st>>>(a, metric_index, out);
    return cudaGetLastError();
}

cudaError_t launch_band_reduce(const PairArgs& a, cudaStream_t st) {
    const long long blocks = (a.P + 255) / 256;
    k_band_reduce<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_acc_field(const float* acc, const unsigned short* ta, const unsigned short* tb,
                             int ntp, int B, int n, int field, double* out, cudaStream_t st) {
    const long long P = (long long)n * (n - 1) / 2;
    dim3 grid(ntp, B);
    k_acc_field<<<grid, 256, 0, st>>>(acc, ta, tb, B, n, field, out, P);
    return cudaGetLastError();
}

cudaError_t launch_expand_dense(const float* packed, float* dense, int n, int antisym, cudaStream_t st) {
    dim3 grid((n + 127) / 128, n);
    k_expand_dense<<<grid, 128, 0, st>>>(packed, dense, n, antisym);
    return cudaGetLastError();
}

cudaError_t launch_df_planes_to_double(const float* acc2, long long P, double* out, cudaStream_t st) {
    k_df_planes<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(acc2, P, out);
    return cudaGetLastError();
}
