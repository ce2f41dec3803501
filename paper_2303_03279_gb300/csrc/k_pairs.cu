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

namespace {

using namespace fcpair;

// ------------------------------------------------------------------------------- node
__global__ void k_node(NodeArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
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
        s = 0.0;
        for (long long k = start; k < end; ++k) {
            const float2 X = a.ring[((size_t)(k % a.slots) * a.B + f) * a.n + i];
            s += (double)X.x * X.x + (double)X.y * X.y;
        }
    }
    a.psd[e] = s;
    a.inv_psd[e] = (s > 0.0) ? (float)(1.0 / sqrt(s)) : 0.f;
}

// ---------------------------------------------------------------- full-window sums
constexpr int WK = 16;  // trials staged per chunk

__global__ void __launch_bounds__(256, 2) k_window(PairArgs a, int bins_metric, float* bins_out) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const WinFacts wf = window_facts(c, a.W, a.count);
    const int K = wf.K;
    const KConst kc = make_kconst(K);

    const int tp = blockIdx.x;
    const int g = blockIdx.y;
    const int f0 = g * a.group_bins;
    const int f1 = min(a.B, f0 + a.group_bins);
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x;
    const int li = tid >> 3, lj0 = (tid & 7) * 4;
    const unsigned vmask = pair_mask(ta, tb, li, lj0, a.n);
    const int gi = ta * FC_T + li, gj0 = tb * FC_T + lj0;

    __shared__ float2 sx[WK][2 * FC_T];
    __shared__ float2 su[WK][2 * FC_T];
    __shared__ float sinv[2][FC_T];

    float band[7][4];
#pragma unroll
    for (int m = 0; m < 7; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) band[m][q] = 0.f;

    for (int f = f0; f < f1; ++f) {
        df32 v[4][FC_NFIELD];
        int s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s[q] = 0;
#pragma unroll
            for (int k = 0; k < FC_NFIELD; ++k) v[q][k] = df_make(0.f, 0.f);
        }
        if (tid < 64) {
            const int w = tid >> 5, l = tid & 31;
            const int node = (w ? tb : ta) * FC_T + l;
            sinv[w][l] = node < a.n ? a.inv_psd[(size_t)f * a.n + node] : 0.f;
        }
        for (int k0 = 0; k0 < K; k0 += WK) {
            const int kc = min(WK, K - k0);
            __syncthreads();
            for (int e = tid; e < kc * 2 * FC_T; e += 256) {
                const int kk = e / (2 * FC_T), l = e % (2 * FC_T);
                const int node = (l < FC_T ? ta * FC_T + l : tb * FC_T + l - FC_T);
                const long long trial = wf.start + k0 + kk;
                float2 X = make_float2(0.f, 0.f);
                if (node < a.n) X = a.ring[((size_t)(trial % a.slots) * a.B + f) * a.n + node];
                sx[kk][l] = X;
                su[kk][l] = phasor_of(X);
            }
            __syncthreads();
            if (vmask) {
                for (int kk = 0; kk < kc; ++kk) {
                    const float2 xi = sx[kk][li], ui = su[kk][li];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 xj = sx[kk][FC_T + lj0 + q];
                        const PairTerms tt = pair_terms(xi, xj, ui, su[kk][FC_T + lj0 + q],
                                                        node_tiny(xi) || node_tiny(xj));
                        v[q][0] = df_add_f(v[q][0], tt.re);
                        v[q][1] = df_add_f(v[q][1], tt.im);
                        v[q][2] = df_add_f(v[q][2], tt.ure);
                        v[q][3] = df_add_f(v[q][3], tt.uim);
                        v[q][4] = df_add_f(v[q][4], fabsf(tt.im));
                        v[q][5] = df_add_df(v[q][5], df_sqr_f(tt.im));
                        s[q] += tt.sgn;
                    }
                }
            }
        }
        __syncthreads();  // sinv visible
        if (vmask) {
            if (a.write_acc) {
                float* blk = a.acc + ((size_t)tp * a.B + f) * FC_BLOCK_WORDS;
                const int w0 = li * FC_T + lj0;
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k) {
                    float4 h = make_float4(v[0][k].hi, v[1][k].hi, v[2][k].hi, v[3][k].hi);
                    float4 l = make_float4(v[0][k].lo, v[1][k].lo, v[2][k].lo, v[3][k].lo);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k) * FC_TT + w0), h);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k + 1) * FC_TT + w0), l);
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
                    } else {
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
    const float invB = 1.0f / (float)a.B;
    for (int m = 0; m < 7; ++m) {
        if (!(a.mask & (1u << (m + 2)))) continue;
        float s = 0.f;
        for (int g = 0; g < a.groups; ++g) s = __fadd_rn(s, a.partial[((size_t)g * 7 + m) * a.P + p]);
        a.net[(size_t)(m + 2) * a.P + p] = __fmul_rn(s, invB);
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

cudaError_t launch_window_sums(const PairArgs& a, cudaStream_t st) {
    dim3 grid(a.ntp, a.groups);
    k_window<<<grid, 256, 0, st>>>(a, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_bins_window(const PairArgs& a, int metric_index, float* out, cudaStream_t st) {
    dim3 grid(a.ntp, a.groups);
    PairArgs b = a;
    b.finalize = 0;
    b.write_acc = 0;
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
