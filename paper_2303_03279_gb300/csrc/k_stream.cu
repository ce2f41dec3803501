// k_stream.cu - streaming update of the spectral running sums (Methods 2.4 storage mode:
// "for every newly added trial only the evaluation of this single trial is necessary";
// Methods 2.5 / Results 3.2.3: each new trial is added to the network, the user sets the
// number of trials averaged), with the metric finalize and band average fused.
//
// For every (pair, bin): add the terms of the newest trial and subtract those of the trial
// leaving the window on the resident double-float accumulators (52 B per pair-bin), then
// evaluate the metrics from the updated sums and accumulate their band average.
// HBM-bound: 104 B move per pair-bin and push.
//
// GB300 mapping: a persistent grid (2 CTAs per SM) walks a static round-robin list of
// (tile pair, bin group) units. The state of one (tile pair, bin) is one contiguous
// 53,248-byte block; one thread streams the block two steps ahead into shared memory
// with cp.async.bulk (TMA bulk copy) completing on an mbarrier, double-buffered, so the
// HBM read stream never waits for the arithmetic. Each thread updates 4 adjacent pairs
// of the 32 x 32 tile (128-bit shared loads, conflict-free) and writes the new state
// straight back to HBM with 128-bit streaming stores. The spectra of the next bin are
// prefetched into registers during the current bin and staged after it, so one barrier
// per bin suffices. Every mbarrier wait is bounded; on expiry the kernel records
// FC_ERR_TIMEOUT in the control block and returns.
#include "df32.cuh"
#include "fc_internal.h"
#include "pair_common.cuh"
#include "terms.cuh"
#include "mbar.cuh"


namespace {

using namespace fcpair;
using namespace fcmbar;

constexpr uint32_t BLK_BYTES = FC_BLOCK_WORDS * 4;  // 53,248
// per stage: 4 node sets (new row, new col, old row, old col negated) x 32 nodes of
// re, im, phasor re, phasor im (float) and a tiny flag (int); then 1/sqrt(PSD) rows/cols
constexpr int SET_WORDS = 5 * FC_T;
constexpr int STAGE_WORDS = 4 * SET_WORDS + 2 * FC_T;
constexpr int OFF_MBAR = 2 * BLK_BYTES;
constexpr int OFF_STAGE = OFF_MBAR + 16;
constexpr int SMEM_BYTES = OFF_STAGE + 2 * STAGE_WORDS * 4;

struct Step {
    int u;   // unit index over the whole batch
    int f;   // bin
    int s;   // session of the unit
    int lu;  // unit index within its session: tile pair * groups + bin group
};

// Facts of one session's push, read from its control block: window position, ring slots
// of the trial added and of the trial leaving, window length.
struct SessFacts {
    bool skip;  // the push was rejected (non-finite trial) or the window is empty
    bool upd, sub;
    int slot_new, slot_old;
    KConst kc;
};
__device__ __forceinline__ SessFacts facts_of(const PairArgs& a) {
    SessFacts F;
    const FcCtrl* c = a.ctrl;
    // t = newest trial after this call (count 1: being added; 0: finalize only)
    const long long t = c->pushed + a.count - 1;
    F.upd = a.update != 0;
    F.slot_new = F.upd ? (int)(t % a.slots) : 0;
    F.sub = F.upd && (a.W > 0) && (t >= a.W);
    F.slot_old = F.sub ? (int)((t - a.W) % a.slots) : 0;
    const int K = (a.W > 0 && t + 1 > a.W) ? a.W : (int)(t + 1);
    F.skip = c->bad != 0 || K <= 0;
    F.kc = make_kconst(K > 0 ? K : 1);
    return F;
}

// One launch updates every session of the batch: the units of all sessions form one list
// (batch.unit_prefix), walked round-robin by the persistent CTAs. MULTI = false is the
// single-session instantiation: every parameter read has a constant offset.
template <bool MULTI>
__global__ void __launch_bounds__(256, 2) k_stream(const StreamBatch batch) {
    extern __shared__ __align__(128) unsigned char smem[];
    auto sess = [&](int s) -> const PairArgs& { return batch.a[MULTI ? s : 0]; };
    const int units = MULTI ? batch.unit_prefix[batch.nsess] : batch.unit_prefix[1];
    if ((int)blockIdx.x >= units) return;

    float* buf[2] = {reinterpret_cast<float*>(smem), reinterpret_cast<float*>(smem + BLK_BYTES)};
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + OFF_MBAR);
    float* stg = reinterpret_cast<float*>(smem + OFF_STAGE);  // [2][STAGE_WORDS]

    const int tid = threadIdx.x;
    const int li = tid >> 3, lj0 = (tid & 7) * 4;
    const int w0 = li * FC_T + lj0;

    auto make_step = [&](int u) -> Step {  // first bin of unit u
        Step r{u, 0, 0, 0};
        if (u >= units) return r;
        if (MULTI) {
            while (r.s + 1 < batch.nsess && u >= batch.unit_prefix[r.s + 1]) ++r.s;
            r.lu = u - batch.unit_prefix[r.s] + sess(r.s).u0;
        } else {
            r.lu = u + sess(0).u0;
        }
        const PairArgs& A = sess(r.s);
        r.f = A.groups == 1 ? 0 : (r.lu % A.groups) * A.group_bins;
        return r;
    };
    auto unit_tp = [&](const Step& s) {
        const PairArgs& A = sess(s.s);
        return A.groups == 1 ? s.lu : s.lu / A.groups;
    };
    auto next_step = [&](Step s) -> Step {
        const PairArgs& A = sess(s.s);
        const int end = A.groups == 1 ? A.B : min(A.B, (s.lu % A.groups) * A.group_bins + A.group_bins);
        if (s.f + 1 < end) {
            s.f += 1;
            return s;
        }
        return make_step(s.u + (int)gridDim.x);
    };
    auto block_ptr = [&](const Step& s) -> float* {
        const PairArgs& A = sess(s.s);
        return A.acc + ((size_t)unit_tp(s) * A.B + s.f) * FC_BLOCK_WORDS;
    };
    // spectra (threads 0..127: set w = tid/32, node l = tid%32) or 1/sqrt(PSD)
    // (threads 128..191) of step s
    auto fetch = [&](const Step& s, const SessFacts& F, float2& X, float& inv) {
        const PairArgs& A = sess(s.s);
        const int tp = unit_tp(s);
        const int ta = A.tile_a[tp], tb = A.tile_b[tp];
        if (tid < 128) {
            const int w = tid >> 5, l = tid & 31;
            const int node = ((w & 1) ? tb : ta) * FC_T + l;
            const bool old = w >= 2;
            X = make_float2(0.f, 0.f);
            if (F.upd && !F.skip && node < A.n && (!old || F.sub))
                X = A.ring[((size_t)(old ? F.slot_old : F.slot_new) * A.B + s.f) * A.n + node];
            if (w == 3) X = make_float2(-X.x, -X.y);  // leaving trial, column side: negated
        } else if (tid < 192) {
            const int w = (tid - 128) >> 5, l = tid & 31;
            const int node = (w ? tb : ta) * FC_T + l;
            inv = node < A.n ? A.inv_psd[(size_t)s.f * A.n + node] : 0.f;
        }
    };
    auto stage = [&](int st, float2 X, float inv) {
        float* g = stg + st * STAGE_WORDS;
        if (tid < 128) {
            const int w = tid >> 5, l = tid & 31;
            const float2 u = phasor_of(X);
            float* set = g + w * SET_WORDS;
            set[l] = X.x;
            set[FC_T + l] = X.y;
            set[2 * FC_T + l] = u.x;
            set[3 * FC_T + l] = u.y;
            reinterpret_cast<int*>(set)[4 * FC_T + l] = node_tiny(X) ? 1 : 0;
        } else if (tid < 192) {
            g[4 * SET_WORDS + (tid - 128)] = inv;
        }
    };

    Step cur = make_step((int)blockIdx.x);
    SessFacts Fc = facts_of(sess(cur.s));
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&mbar[0], BLK_BYTES);
        bulk_g2s(buf[0], block_ptr(cur), BLK_BYTES, &mbar[0]);
        const Step s1 = next_step(cur);
        if (s1.u < units) {
            mbar_expect_tx(&mbar[1], BLK_BYTES);
            bulk_g2s(buf[1], block_ptr(s1), BLK_BYTES, &mbar[1]);
        }
    }
    {
        float2 X = make_float2(0.f, 0.f);
        float inv = 0.f;
        fetch(cur, Fc, X, inv);
        stage(0, X, inv);
    }
    __syncthreads();

    float2 band[7][2];
#pragma unroll
    for (int m = 0; m < 7; ++m) band[m][0] = band[m][1] = make_float2(0.f, 0.f);

    int it = 0;
    while (cur.u < units) {
        const int st = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        const PairArgs& a = sess(cur.s);
        const bool upd = Fc.upd, sub = Fc.sub;
        const KConst& kc = Fc.kc;
        const Step nxt = next_step(cur);
        const SessFacts Fn = (nxt.u < units && nxt.s != cur.s) ? facts_of(sess(nxt.s)) : Fc;
        float2 pX = make_float2(0.f, 0.f);
        float pinv = 0.f;
        if (nxt.u < units) fetch(nxt, Fn, pX, pinv);  // latency hidden behind this bin's work

        const bool arrived = mbar_wait_bounded(&mbar[st], parity);
        const int tp = unit_tp(cur);
        const int ta = a.tile_a[tp], tb = a.tile_b[tp];
        const unsigned vmask = (arrived && !Fc.skip) ? pair_mask(ta, tb, li, lj0, a.n) : 0u;
        if (vmask) {
            const float* blk = buf[st];
            const float* g = stg + st * STAGE_WORDS;
            float4 hi[FC_NFIELD], lo[FC_NFIELD];
#pragma unroll
            for (int k = 0; k < FC_NFIELD; ++k) {
                hi[k] = *reinterpret_cast<const float4*>(blk + (2 * k) * FC_TT + w0);
                lo[k] = *reinterpret_cast<const float4*>(blk + (2 * k + 1) * FC_TT + w0);
            }
            int4 sg = *reinterpret_cast<const int4*>(blk + 12 * FC_TT + w0);
            const float* Sn_r = g;                  // new trial, row nodes
            const float* Sn_c = g + SET_WORDS;      // new trial, column nodes
            const float* So_r = g + 2 * SET_WORDS;  // leaving trial, row nodes
            const float* So_c = g + 3 * SET_WORDS;  // leaving trial, column nodes (negated)
            const RowConst rn = row_const(Sn_r[li], Sn_r[FC_T + li], Sn_r[2 * FC_T + li], Sn_r[3 * FC_T + li],
                                          reinterpret_cast<const int*>(Sn_r)[4 * FC_T + li] != 0);
            const RowConst ro = row_const(So_r[li], So_r[FC_T + li], So_r[2 * FC_T + li], So_r[3 * FC_T + li],
                                          reinterpret_cast<const int*>(So_r)[4 * FC_T + li] != 0);
            const float inv_i = g[4 * SET_WORDS + li];
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // pairs (lj0 + 2h, lj0 + 2h + 1)
                const int j = lj0 + 2 * h;
                float2 vh[FC_NFIELD], vl[FC_NFIELD];
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k) {
                    vh[k] = h ? make_float2(hi[k].z, hi[k].w) : make_float2(hi[k].x, hi[k].y);
                    vl[k] = h ? make_float2(lo[k].z, lo[k].w) : make_float2(lo[k].x, lo[k].y);
                }
                int s0 = h ? sg.z : sg.x, s1 = h ? sg.w : sg.y;
                if (upd) {
                    // leaving trial against its negated columns: exact negated terms
                    PairTerms2 o;
                    if (sub) {
                        const int* to = reinterpret_cast<const int*>(So_c) + 4 * FC_T;
                        o = pair_terms2(ro, *reinterpret_cast<const float2*>(So_c + j),
                                        *reinterpret_cast<const float2*>(So_c + FC_T + j),
                                        *reinterpret_cast<const float2*>(So_c + 2 * FC_T + j),
                                        *reinterpret_cast<const float2*>(So_c + 3 * FC_T + j), to[j] != 0,
                                        to[j + 1] != 0);
                    } else {
                        o.re = o.im = o.ure = o.uim = make_float2(0.f, 0.f);
                        o.s0 = o.s1 = 0;
                    }
                    const int* tn = reinterpret_cast<const int*>(Sn_c) + 4 * FC_T;
                    const PairTerms2 n = pair_terms2(rn, *reinterpret_cast<const float2*>(Sn_c + j),
                                                     *reinterpret_cast<const float2*>(Sn_c + FC_T + j),
                                                     *reinterpret_cast<const float2*>(Sn_c + 2 * FC_T + j),
                                                     *reinterpret_cast<const float2*>(Sn_c + 3 * FC_T + j),
                                                     tn[j] != 0, tn[j + 1] != 0);
                    acc2_ff(vh[0], vl[0], n.re, o.re);
                    acc2_ff(vh[1], vl[1], n.im, o.im);
                    acc2_ff(vh[2], vl[2], n.ure, o.ure);
                    acc2_ff(vh[3], vl[3], n.uim, o.uim);
                    const float2 an = make_float2(fabsf(n.im.x), fabsf(n.im.y));
                    const float2 ao = make_float2(-fabsf(o.im.x), -fabsf(o.im.y));
                    acc2_ff(vh[4], vl[4], an, ao);
                    // im^2 as exact two-products: (p, e) of the new trial, (-p, -e) of the
                    // leaving one; scalar, because the products feed additions (see terms.cuh)
                    float2 pn, en, npo, neo;
                    two_prod(n.im.x, n.im.x, pn.x, en.x);
                    two_prod(n.im.y, n.im.y, pn.y, en.y);
                    two_prod(o.im.x, -o.im.x, npo.x, neo.x);
                    two_prod(o.im.y, -o.im.y, npo.y, neo.y);
                    acc2_dd(vh[5], vl[5], pn, en, npo, neo);
                    s0 += n.s0 + o.s0;
                    s1 += n.s1 + o.s1;
#pragma unroll
                    for (int k = 0; k < FC_NFIELD; ++k) {
                        if (h) {
                            hi[k].z = vh[k].x; hi[k].w = vh[k].y; lo[k].z = vl[k].x; lo[k].w = vl[k].y;
                        } else {
                            hi[k].x = vh[k].x; hi[k].y = vh[k].y; lo[k].x = vl[k].x; lo[k].y = vl[k].y;
                        }
                    }
                    if (h) { sg.z = s0; sg.w = s1; } else { sg.x = s0; sg.y = s1; }
                }
                if (a.finalize && cur.f >= a.fsel0 && cur.f < a.fsel1) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (!(vmask & (1u << (2 * h + e)))) continue;
                        df32 v[FC_NFIELD];
#pragma unroll
                        for (int k = 0; k < FC_NFIELD; ++k)
                            v[k] = e ? df_make(vh[k].y, vl[k].y) : df_make(vh[k].x, vl[k].x);
                        float m[7];
                        finalize_bin(v, e ? s1 : s0, inv_i, g[4 * SET_WORDS + FC_T + j + e], kc, m);
#pragma unroll
                        for (int mm = 0; mm < 7; ++mm) {
                            if (e) band[mm][h].y = __fadd_rn(band[mm][h].y, m[mm]);
                            else band[mm][h].x = __fadd_rn(band[mm][h].x, m[mm]);
                        }
                    }
                }
            }
            if (upd) {
                float* gp = block_ptr(cur);
#pragma unroll
                for (int k = 0; k < FC_NFIELD; ++k) {
                    __stcs(reinterpret_cast<float4*>(gp + (2 * k) * FC_TT + w0), hi[k]);
                    __stcs(reinterpret_cast<float4*>(gp + (2 * k + 1) * FC_TT + w0), lo[k]);
                }
                __stcs(reinterpret_cast<int4*>(gp + 12 * FC_TT + w0), sg);
            }
        }
        // end of a unit: write its band average (or band-group partial)
        if (nxt.u != cur.u) {
            if (a.finalize && vmask) {
                float bq[7][4];
#pragma unroll
                for (int m = 0; m < 7; ++m) {
                    bq[m][0] = band[m][0].x; bq[m][1] = band[m][0].y;
                    bq[m][2] = band[m][1].x; bq[m][3] = band[m][1].y;
                }
                write_band(a, a.groups == 1 ? 0 : cur.lu % a.groups, bq, ta * FC_T + li, tb * FC_T + lj0, vmask, 0);
            }
#pragma unroll
            for (int m = 0; m < 7; ++m) band[m][0] = band[m][1] = make_float2(0.f, 0.f);
        }
        if (nxt.u < units) stage(st ^ 1, pX, pinv);
        const int timed_out = __syncthreads_or(arrived ? 0 : 1);
        if (timed_out) {
            if (tid == 0) atomicOr(&const_cast<FcCtrl*>(a.ctrl)->timeout, 1);
            // let both stages' copies land before leaving (bounded)
            mbar_wait_bounded(&mbar[st], parity);
            mbar_wait_bounded(&mbar[st ^ 1], ((it + 1) >> 1) & 1);
            return;
        }
        if (tid == 0) {
            const Step nn = next_step(nxt);
            if (nxt.u < units && nn.u < units) {
                fence_proxy_async();
                mbar_expect_tx(&mbar[st], BLK_BYTES);
                bulk_g2s(buf[st], block_ptr(nn), BLK_BYTES, &mbar[st]);
            }
        }
        cur = nxt;
        Fc = Fn;
        ++it;
    }
}

}  // namespace

cudaError_t launch_stream_batch(const StreamBatch& b, int grid_ctas, cudaStream_t st) {
    if (b.nsess < 1 || b.nsess > FC_MAX_BATCH) return cudaErrorInvalidValue;
    const bool multi = b.nsess > 1;
    cudaError_t e = multi ? cudaFuncSetAttribute(k_stream<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)
                          : cudaFuncSetAttribute(k_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int units = b.unit_prefix[b.nsess];
    if (units <= 0) return cudaSuccess;
    const int ctas = units < grid_ctas ? units : grid_ctas;
    if (multi)
        k_stream<true><<<ctas, 256, SMEM_BYTES, st>>>(b);
    else
        k_stream<false><<<ctas, 256, SMEM_BYTES, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_stream_update(const PairArgs& a, cudaStream_t st) {
    StreamBatch b;
    b.nsess = 1;
    b.unit_prefix[0] = 0;
    b.unit_prefix[1] = a.ntp * a.groups;
    b.a[0] = a;
    return launch_stream_batch(b, a.grid_ctas, st);
}
