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
        // flags kept across pushes: a superset of the window's tiny nodes until mode 1 renews them
        if (a.tiny && node_tiny(Xn)) a.tiny[e] = 1;
        if (a.W > 0 && t >= a.W) {
            const float2 Xo = a.ring[((size_t)((t - a.W) % a.slots) * a.B + f) * a.n + i];
            s -= ((double)Xo.x * Xo.x + (double)Xo.y * Xo.y);
        }
    } else {
        const long long end = c->pushed + a.count;
        const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
        const float sc = c->in_scale;  // 0 for sessions (their ring holds prescaled spectra)
        // |X|^2 summed as a double word on the FP32 pipes: both squares are exact two-products
        // while every nonzero component is at least 2^-50 (no underflow); a node with a tiny
        // component takes the FP64 sum instead
        df32 acc = df_make(0.f, 0.f);
        bool tiny = false;
        for (long long k = start; k < end; ++k) {
            float2 X = a.ring[((size_t)(k % a.slots) * a.B + f) * a.n + i];
            if (sc != 0.f) X = make_float2(__fmul_rn(X.x, sc), __fmul_rn(X.y, sc));
            float p1, e1, p2, e2;
            two_prod(X.x, X.x, p1, e1);
            two_prod(X.y, X.y, p2, e2);
            acc = df_add_df(acc, df_add_df(df_make(p1, e1), df_make(p2, e2)));
            tiny |= node_tiny(X);
        }
        s = (double)acc.hi + (double)acc.lo;
        if (tiny) {
            s = 0.0;
            for (long long k = start; k < end; ++k) {
                float2 X = a.ring[((size_t)(k % a.slots) * a.B + f) * a.n + i];
                if (sc != 0.f) X = make_float2(__fmul_rn(X.x, sc), __fmul_rn(X.y, sc));
                s += (double)X.x * X.x + (double)X.y * X.y;
            }
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
constexpr int WK = 24;           // most trials per staged chunk (balanced chunks)
constexpr int WIN_THREADS = 256;

struct WinSmem {
    float2 raw[WK][2 * FC_T];    // the next chunk's spectra as copied (row tile, column tile)
    // row node i, pre-broadcast for the packed operands: (a, a, b, b), (-a, -a, ua, ua),
    // (ub, ub, -ua, -ua) with u = X / |X|
    float4 row[WK][FC_T][3];
    float4 ca[WK][FC_T / 4], cb[WK][FC_T / 4], cua[WK][FC_T / 4], cub[WK][FC_T / 4];  // column planes
    unsigned char tiny[WK][2 * FC_T];
    float sinv[2][2][FC_T];      // 1/sqrt(PSD) of the row and column tiles, by bin parity
};
struct WinBand {
    float band[7][FC_T][FC_T];   // band sums per pair (finalizing launches only)
};

__device__ __forceinline__ void win_cp_async8(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ float win_gt0(float x) {
    float r;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float win_lt0(float x) {
    float r;
    asm("set.lt.f32.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    return r;
}

// Thread: row node li of tile ta against columns lj0 .. lj0 + 3 of tile tb, as two packed
// column pairs (FP32x2 lanes). The terms are those of the streaming kernel (pair_terms2 on
// the same staged values), so a re-summed accumulator and the later streaming subtraction
// of a trial agree bit for bit. Double-float running sums per lane: lazy TwoSum updates
// (acc2_f_lazy / acc2_d_lazy) renormalized after every chunk of at most WK trials, which
// keeps the error of a sum of K terms within about (WK + 1) K u^2 of their summed
// magnitudes. Sign counts: exact FP32 tallies of positive and negative terms. The next
// chunk's spectra are copied by cp.async while the current chunk is summed.
__global__ void __launch_bounds__(WIN_THREADS, 2) k_window(PairArgs a, int bins_metric, float* bins_out) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const WinFacts wf = window_facts(c, a.W, a.count);
    const int K = wf.K;
    if (K <= 0) return;
    const KConst kc = make_kconst(K);
    extern __shared__ __align__(16) unsigned char win_smem_raw[];
    WinSmem& sm = *reinterpret_cast<WinSmem*>(win_smem_raw);
    WinBand& sb = *reinterpret_cast<WinBand*>(win_smem_raw + sizeof(WinSmem));
    const bool band_out = a.finalize && !bins_out;

    const int tp = a.tp0 + blockIdx.x;
    const int g = blockIdx.y;
    const int f0 = g * a.group_bins;
    const int f1 = min(a.B, f0 + a.group_bins);
    const int ta = a.tile_a[tp], tb = a.tile_b[tp];
    const int tid = threadIdx.x;
    const int li = tid >> 3, lj0 = (tid & 7) * 4, cg = tid & 7;
    const unsigned vmask = pair_mask(ta, tb, li, lj0, a.n);
    const int gi = ta * FC_T + li, gj0 = tb * FC_T + lj0;
    if (band_out)
        for (int e = tid; e < 7 * FC_TT; e += WIN_THREADS) (&sb.band[0][0][0])[e] = 0.f;
    const float sc = c->in_scale;  // 0 for sessions (their ring holds prescaled spectra)

    // chunk copies: thread tid copies and converts node l_node of the two tiles, trials
    // kk0 + 4 q of a chunk
    const int l_node = tid & 63, kk0 = tid >> 6;
    const int node = l_node < FC_T ? ta * FC_T + l_node : tb * FC_T + l_node - FC_T;
    const bool node_ok = node < a.n;
    const int nchunk = (K + WK - 1) / WK;
    const int csize = (K + nchunk - 1) / nchunk;
    const int slot_start = (int)(wf.start % a.slots);
    constexpr int PER = WK * 2 * FC_T / WIN_THREADS;
    auto issue_copy = [&](int f, int k0) {
        const int kn = min(csize, K - k0);
        int slot = slot_start + k0 + kk0;
        while (slot >= a.slots) slot -= a.slots;
        const float2* src = a.ring + (size_t)f * a.n + node;
        const size_t slot_stride = (size_t)a.B * a.n;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int kk = kk0 + 4 * q;
            if (kk < kn && node_ok) win_cp_async8(&sm.raw[kk][l_node], src + (size_t)slot * slot_stride);
            slot += 4;
            while (slot >= a.slots) slot -= a.slots;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (f0 < f1) issue_copy(f0, 0);

    for (int f = f0; f < f1; ++f) {
        float2 vh[2][FC_NFIELD], vl[2][FC_NFIELD], pos[2], neg[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            pos[h] = neg[h] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < FC_NFIELD; ++k) vh[h][k] = vl[h][k] = make_float2(0.f, 0.f);
        }
        // (parity: a slow thread may still read the previous bin's values in its finalize;
        // the chunk barriers below order this bin's reads after these writes)
        const int par = f & 1;
        if (tid < 64) {
            const int w = tid >> 5, l = tid & 31;
            const int nd = (w ? tb : ta) * FC_T + l;
            sm.sinv[par][w][l] = nd < a.n ? a.inv_psd[(size_t)f * a.n + nd] : 0.f;
        }
        for (int ci = 0; ci < nchunk; ++ci) {
            const int k0 = ci * csize;
            const int kn = min(csize, K - k0);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();  // the chunk has landed; every thread is done with the previous one
            bool any_tiny = false;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int kk = kk0 + 4 * q;
                float2 X = make_float2(0.f, 0.f);
                if (kk < kn && node_ok) X = sm.raw[kk][l_node];
                if (sc != 0.f) X = make_float2(__fmul_rn(X.x, sc), __fmul_rn(X.y, sc));
                const float2 u = phasor_of(X);
                if (l_node < FC_T) {
                    sm.row[kk][l_node][0] = make_float4(X.x, X.x, X.y, X.y);
                    sm.row[kk][l_node][1] = make_float4(-X.x, -X.x, u.x, u.x);
                    sm.row[kk][l_node][2] = make_float4(u.y, u.y, -u.x, -u.x);
                } else {
                    const int l = l_node - FC_T;
                    reinterpret_cast<float*>(sm.ca[kk])[l] = X.x;
                    reinterpret_cast<float*>(sm.cb[kk])[l] = X.y;
                    reinterpret_cast<float*>(sm.cua[kk])[l] = u.x;
                    reinterpret_cast<float*>(sm.cub[kk])[l] = u.y;
                }
                const bool tn = node_tiny(X);
                sm.tiny[kk][l_node] = tn ? 1 : 0;
                any_tiny |= tn;
            }
            // chunks without a tiny node (the rule) run a loop with no FP64 branch at all
            const bool chunk_tiny = __syncthreads_or(any_tiny ? 1 : 0) != 0;
            // the raw buffer is free again: copy the next chunk (this bin's or the next's)
            if (ci + 1 < nchunk)
                issue_copy(f, k0 + csize);
            else if (f + 1 < f1)
                issue_copy(f + 1, 0);
            if (!vmask) continue;
            auto chunk = [&](auto tiny_c) {
                constexpr bool TINY = decltype(tiny_c)::value;
#pragma unroll 2
                for (int kk = 0; kk < kn; ++kk) {
                    const float4 r0 = sm.row[kk][li][0], r1 = sm.row[kk][li][1], r2 = sm.row[kk][li][2];
                    RowConst rc;
                    rc.a = make_float2(r0.x, r0.y);
                    rc.b = make_float2(r0.z, r0.w);
                    rc.na = make_float2(r1.x, r1.y);
                    rc.ua = make_float2(r1.z, r1.w);
                    rc.ub = make_float2(r2.x, r2.y);
                    rc.nua = make_float2(r2.z, r2.w);
                    rc.as = r0.x;
                    rc.bs = r0.z;
                    rc.tiny = TINY && sm.tiny[kk][li] != 0;
                    const float4 xa = sm.ca[kk][cg], xb = sm.cb[kk][cg], xua = sm.cua[kk][cg], xub = sm.cub[kk][cg];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 aj = h ? make_float2(xa.z, xa.w) : make_float2(xa.x, xa.y);
                        const float2 bj = h ? make_float2(xb.z, xb.w) : make_float2(xb.x, xb.y);
                        const float2 uaj = h ? make_float2(xua.z, xua.w) : make_float2(xua.x, xua.y);
                        const float2 ubj = h ? make_float2(xub.z, xub.w) : make_float2(xub.x, xub.y);
                        const int j = FC_T + lj0 + 2 * h;
                        const PairTerms2 t = pair_terms2<TINY>(rc, aj, bj, uaj, ubj, TINY && sm.tiny[kk][j] != 0,
                                                               TINY && sm.tiny[kk][j + 1] != 0);
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
                        if (TINY) {
                            pos[h] = add2(pos[h], make_float2(t.s0 > 0 ? 1.f : 0.f, t.s1 > 0 ? 1.f : 0.f));
                            neg[h] = add2(neg[h], make_float2(t.s0 < 0 ? 1.f : 0.f, t.s1 < 0 ? 1.f : 0.f));
                        } else {
                            pos[h] = add2(pos[h], make_float2(win_gt0(t.im.x), win_gt0(t.im.y)));
                            neg[h] = add2(neg[h], make_float2(win_lt0(t.im.x), win_lt0(t.im.y)));
                        }
                    }
                }
                // back to normalized double words once per chunk
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int k = 0; k < FC_NFIELD; ++k) renorm2(vh[h][k], vl[h][k]);
            };
            if (chunk_tiny)
                chunk(std::true_type{});
            else
                chunk(std::false_type{});
        }
        if (vmask) {
            df32 v[4][FC_NFIELD];
            int sgn[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k)
                    v[q][k] = (q & 1) ? df_make(vh[q >> 1][k].y, vl[q >> 1][k].y)
                                      : df_make(vh[q >> 1][k].x, vl[q >> 1][k].x);
                sgn[q] = (q & 1) ? (int)pos[q >> 1].y - (int)neg[q >> 1].y : (int)pos[q >> 1].x - (int)neg[q >> 1].x;
            }
            if (a.write_acc) {
                float* blk = a.acc + ((size_t)(tp - a.acc_tp_base) * a.B + f) * FC_BLOCK_WORDS;
                const int w0 = li * FC_T + lj0;
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k) {
                    float4 hq = make_float4(v[0][k].hi, v[1][k].hi, v[2][k].hi, v[3][k].hi);
                    float4 lq = make_float4(v[0][k].lo, v[1][k].lo, v[2][k].lo, v[3][k].lo);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k) * FC_TT + w0), hq);
                    __stcs(reinterpret_cast<float4*>(blk + (2 * k + 1) * FC_TT + w0), lq);
                }
                __stcs(reinterpret_cast<int4*>(blk + 12 * FC_TT + w0), make_int4(sgn[0], sgn[1], sgn[2], sgn[3]));
            }
            if (a.finalize || bins_out) {
                const float inv_i = sm.sinv[par][0][li];
                const bool in_band = band_out && f >= a.fsel0 && f < a.fsel1;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float m[7];
                    finalize_bin(v[q], sgn[q], inv_i, sm.sinv[par][1][lj0 + q], kc, m);
                    if (bins_out && (vmask & (1u << q))) {
                        float val = m[0];
#pragma unroll
                        for (int mm = 1; mm < 7; ++mm) val = (mm == bins_metric - 2) ? m[mm] : val;
                        bins_out[(size_t)f * a.P + packed_index(gi, gj0 + q, a.n)] = val;
                    }
                    if (in_band) {
#pragma unroll
                        for (int mm = 0; mm < 7; ++mm) sb.band[mm][li][lj0 + q] = __fadd_rn(sb.band[mm][li][lj0 + q], m[mm]);
                    }
                }
            }
        }
    }
    if (band_out && vmask) {
        float band[7][4];
#pragma unroll
        for (int mm = 0; mm < 7; ++mm)
#pragma unroll
            for (int q = 0; q < 4; ++q) band[mm][q] = sb.band[mm][li][lj0 + q];
        write_band(a, g, band, gi, gj0, vmask, f1 - f0);
    }
}

size_t window_smem_bytes(bool band) { return sizeof(WinSmem) + (band ? sizeof(WinBand) : 0); }

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

static cudaError_t launch_window_kernel(const PairArgs& a, dim3 grid, int metric_index, float* out, cudaStream_t st) {
    const size_t smem = window_smem_bytes(a.finalize && !out);
    cudaError_t e = cudaFuncSetAttribute(k_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)window_smem_bytes(true));
    if (e != cudaSuccess) return e;
    k_window<<<grid, WIN_THREADS, smem, st>>>(a, metric_index, out);
    return cudaGetLastError();
}

namespace {
// Re-summed accumulator blocks from the scratch into the state, unless the push was
// rejected (then the window, and with it every block, stays as it was).
__global__ void k_copy_blocks(const float4* __restrict__ src, float4* __restrict__ dst, long long n4,
                              const FcCtrl* ctrl) {
    if (ctrl->bad) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        __stcs(dst + i, __ldcs(src + i));
}
}  // namespace

namespace {
// planes 2, 3 (sum Im), 8 .. 11 (sum |Im|, sum Im^2) and 12 (sign count) of a block
__global__ void k_gather_nonlinear(const float4* __restrict__ scratch, float4* __restrict__ acc,
                                   const int* __restrict__ list, long long n4, int B, const FcCtrl* ctrl) {
    if (ctrl->bad) return;
    constexpr int P4 = FC_TT / 4;  // float4 per plane
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e % P4);
        long long rest = e / P4;
        const int pi = (int)(rest % 7);
        rest /= 7;
        const int f = (int)(rest % B);
        const long long i = rest / B;
        const int plane = pi < 2 ? 2 + pi : 6 + pi;  // 2, 3, 8, 9, 10, 11, 12
        const size_t off = (size_t)plane * P4 + w;
        const float4 v = __ldcs(scratch + ((size_t)i * B + f) * (FC_BLOCK_WORDS / 4) + off);
        __stcs(acc + ((size_t)list[i] * B + f) * (FC_BLOCK_WORDS / 4) + off, v);
    }
}
}  // namespace

cudaError_t launch_gather_nonlinear(const float* scratch, float* acc, const int* list, int count, int B,
                                    const FcCtrl* ctrl, cudaStream_t st) {
    const long long n4 = (long long)count * B * 7 * (FC_TT / 4);
    if (n4 <= 0) return cudaSuccess;
    long long blocks = (n4 + 255) / 256;
    const long long cap = 4LL * fc_device_sms();
    if (blocks > cap) blocks = cap;
    k_gather_nonlinear<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(scratch),
                                                       reinterpret_cast<float4*>(acc), list, n4, B, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_copy_blocks(const float* src, float* dst, long long nfloats, const FcCtrl* ctrl, cudaStream_t st) {
    const long long n4 = nfloats / 4;
    if (n4 <= 0) return cudaSuccess;
    long long blocks = (n4 + 255) / 256;
    const long long cap = 4LL * fc_device_sms();
    if (blocks > cap) blocks = cap;
    k_copy_blocks<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst),
                                                  n4, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_window_sums(const PairArgs& a, cudaStream_t st) {
    if (a.tp0 < 0 || a.tp_count < 0 || a.tp0 + (a.tp_count ? a.tp_count : a.ntp) > a.ntp) return cudaErrorInvalidValue;
    dim3 grid(a.tp_count ? a.tp_count : a.ntp, a.groups);
    return launch_window_kernel(a, grid, 0, nullptr, st);
}

cudaError_t launch_bins_window(const PairArgs& a, int metric_index, float* out, cudaStream_t st) {
    dim3 grid(a.ntp, a.groups);
    PairArgs b = a;
    b.finalize = 0;
    b.write_acc = 0;
    b.tp0 = 0;
    b.tp_count = 0;
    return launch_window_kernel(b, grid, metric_index, out, st);
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
