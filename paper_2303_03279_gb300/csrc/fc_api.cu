// fc_api.cu - the C ABI (include/fc.h): sessions, device state, push sequencing.
//
// A push enqueues, on the session's stream and without waiting for the device:
//   validate  -> taper + band spectrum into the ring slot of the new trial
//   -> (first pushes) power-of-two calibration of the spectra
//   -> per-node PSD sums -> pair update (streaming add/subtract, or the full-window
//      recompute in FC_MODE_FULL) -> band reduction (small sessions)
//   -> (stream mode) re-sum of one slice of the accumulators from the stored spectra
//   -> COR / XCOR -> commit.
// The window position lives in a device control block, so a rejected (non-finite) trial
// is skipped by every kernel and the host never synchronizes inside a push.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "fc_internal.h"

namespace {

thread_local std::string g_err;

fc_status fail(fc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(FC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

const double kPi = 3.14159265358979323846;

int metric_index(uint32_t bit) {
    for (int i = 0; i < FC_NMETRIC; ++i)
        if (bit == (1u << i)) return i;
    return -1;
}

fc_status dev_alloc(fc_session* s, size_t bytes, void** out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (s->cfg.dev_alloc) {
        p = s->cfg.dev_alloc(bytes, s->cfg.alloc_ctx);
        if (!p) return fail(FC_ERR_OUT_OF_MEMORY, "device allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FC_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    s->allocations.push_back(p);
    s->device_bytes += bytes;
    *out = p;
    return FC_OK;
}

template <class T>
fc_status alloc_zero(fc_session* s, size_t count, T** out) {
    void* p;
    fc_status st = dev_alloc(s, count * sizeof(T), &p);
    if (st != FC_OK) return st;
    CK(cudaMemsetAsync(p, 0, count * sizeof(T), s->stream));
    s->state_bufs.emplace_back(p, count > 0 ? count * sizeof(T) : 16);
    *out = static_cast<T*>(p);
    return FC_OK;
}

void free_all(fc_session* s) {
    for (void* p : s->allocations) {
        if (s->cfg.dev_free)
            s->cfg.dev_free(p, s->cfg.alloc_ctx);
        else if (!s->cfg.dev_alloc)
            cudaFree(p);
    }
    s->allocations.clear();
}

// -------------------------------------------------------------- profiling wrapper
std::vector<cudaEvent_t>& event_pool() {
    static thread_local std::vector<cudaEvent_t> pool;
    return pool;
}

cudaEvent_t get_event() {
    auto& pool = event_pool();
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

template <class F>
fc_status launch(fc_session* s, int kid, F&& f, cudaStream_t on = nullptr) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!on) on = s->stream;
    if (s->profiling) {
        e0 = get_event();
        e1 = get_event();
        cudaEventRecord(e0, on);
    }
    cudaError_t e = f();
    s->launches++;
    if (s->profiling) {
        cudaEventRecord(e1, on);
        s->pending.push_back({kid, e0, e1});
    }
    if (e != cudaSuccess) return fail(FC_ERR_CUDA, "kernel %d launch failed: %s", kid, cudaGetErrorString(e));
    return FC_OK;
}

#define LAUNCH(kid, expr)                                              \
    do {                                                               \
        fc_status st_ = launch(s, (kid), [&]() { return (expr); });    \
        if (st_ != FC_OK) return st_;                                  \
    } while (0)
// the same, timed on another stream of the session
#define LAUNCH_ON(kid, strm, expr)                                             \
    do {                                                                       \
        fc_status st_ = launch(s, (kid), [&]() { return (expr); }, (strm));    \
        if (st_ != FC_OK) return st_;                                          \
    } while (0)

fc_status drain_timings(fc_session* s) {
    for (auto& p : s->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p.start, p.stop);
        if (e == cudaSuccess) {
            s->ktime[p.kernel].launches += 1;
            s->ktime[p.kernel].total_ms += ms;
        }
        event_pool().push_back(p.start);
        event_pool().push_back(p.stop);
    }
    s->pending.clear();
    return FC_OK;
}

// ------------------------------------------------------------------ argument packs
PairArgs pair_args(fc_session* s, bool stream_kernel, int count) {
    PairArgs a{};
    a.ring = s->ring;
    a.inv_psd = s->inv_psd;
    a.acc = s->acc;
    a.tile_a = s->tile_a;
    a.tile_b = s->tile_b;
    a.net_spec = s->net + (size_t)MI_COH * s->P;
    a.partial = s->partial;
    a.slots = s->slots;
    a.n = s->n;
    a.B = s->B;
    a.W = s->W;
    a.ntp = s->ntp;
    a.P = s->P;
    a.groups = stream_kernel ? s->stream_groups : s->groups;
    a.group_bins = stream_kernel ? s->stream_group_bins : s->group_bins;
    a.mask = s->mask;
    a.finalize = 1;
    a.update = 1;
    a.write_acc = 0;
    a.count = count;
    a.grid_ctas = 2 * s->num_sms;
    a.fsel0 = s->sel0;
    a.fsel1 = s->sel1;
    a.ctrl = s->ctrl;
    return a;
}

SpectrumArgs spectrum_args(fc_session* s, const float* x, int count, int write_from) {
    SpectrumArgs a{};
    a.x = x;
    a.count = count;
    a.write_from = write_from;
    a.twiddle = s->twiddle;
    a.fft = s->use_fft ? 1 : 0;
    a.nfft = s->nfft;
    a.first_bin = s->first_bin;
    a.taper = s->taper_tab;
    a.fft_tw = s->fft_tw;
    a.fft_stages = fc_fft_radices(s->nfft / 2, &a.fft_radices);
    a.ring = s->ring;
    a.slots = s->slots;
    a.n = s->n;
    a.N = s->N;
    a.B = s->B;
    a.ctrl = s->ctrl;
    return a;
}

CorArgs cor_args(fc_session* s, const float* x, int count, int write_from, int mode) {
    CorArgs a{};
    a.x = x;
    a.count = count;
    a.write_from = write_from;
    a.zring = s->zring;
    a.cor_acc = s->cor_acc;
    a.net = s->net + (size_t)MI_COR * s->P;
    a.slots = s->slots;
    a.n = s->n;
    a.N = s->N;
    a.W = s->W;
    a.P = s->P;
    a.mode = mode;
    a.finalize = (s->mask & FC_COR) ? 1 : 0;
    a.groups = 1;
    a.ctrl = s->ctrl;
    return a;
}

XcorArgs xcor_args(fc_session* s, const float* x, int count, int write_from, int mode) {
    XcorArgs a{};
    a.x = x;
    a.count = count;
    a.write_from = write_from;
    a.n = s->n;
    a.N = s->N;
    a.L = s->xcor_L;
    a.W = s->W;
    a.slots = s->slots;
    a.P = s->P;
    a.tw = s->xcor_tw;
    a.spec = s->xcor_spec;
    a.energy = s->xcor_energy;
    a.vals = s->xcor_vals;
    a.lag = s->xcor_lag;
    a.acc = s->xcor_acc;
    a.net = s->net + (size_t)MI_XCOR * s->P;
    a.mode = mode;
    a.finalize = (s->mask & FC_XCOR) ? 1 : 0;
    a.ctrl = s->ctrl;
    return a;
}

// ------------------------------------------------------------------ push stages
fc_status stage_spectra(fc_session* s, const float* x, int count, int write_from) {
    SpectrumArgs sa = spectrum_args(s, x, count, write_from);
    if (s->spec_project) {
        // x holds sensor trials: their band spectra, then the projection into the ring
        const int keep = count - write_from;
        if (s->sens_trials < keep) {
            if (s->sens_spec) cudaFree(s->sens_spec);
            s->sens_spec = nullptr;
            s->sens_trials = 0;
            CK(cudaMalloc(&s->sens_spec, (size_t)keep * s->B * s->proj_C * sizeof(float2)));
            s->sens_trials = keep;
        }
        SpectrumArgs ss = sa;
        ss.n = s->proj_C;
        ss.ring = s->sens_spec;
        ss.direct = 1;
        LAUNCH(FC_K_SPECTRUM, launch_spectrum(ss, s->stream));
        LAUNCH(FC_K_PROJECT, launch_project_spectra(s->proj, s->sens_spec, s->ring, s->n, s->proj_C, s->B, keep,
                                                    write_from, s->slots, s->ctrl, s->stream));
    } else {
        LAUNCH(FC_K_SPECTRUM, launch_spectrum(sa, s->stream));
    }
    if (!s->calibrated) {
        for (int ph = 0; ph < 3; ++ph) LAUNCH(FC_K_CALIBRATE, launch_calibrate(sa, s->stream, ph));
    }
    return FC_OK;
}

fc_status stage_time_metrics(fc_session* s, const float* x, int count, int write_from, int mode) {
    if (s->time_mask & FC_COR) {
        // normalized trials -> split-TF32 operand ring -> per-trial Gram products on the
        // tensor cores, added to (mode 0: and the leaving trial's subtracted from) the sums
        CorArgs ca = cor_args(s, x, count, write_from, mode);
        CorTcArgs ta{};
        ta.zring = s->zring;
        ta.ops = s->cor_ops;
        ta.n = s->n;
        ta.N = s->N;
        ta.nt = s->cor_nt;
        ta.ntp = s->cor_ntp;
        ta.nchunks = s->cor_nchunks;
        ta.slots = s->slots;
        ta.W = s->W;
        ta.P = s->P;
        ta.count = count;
        ta.write_from = write_from;
        ta.mode = mode;
        ta.groups = 1;
        ta.cor_acc = s->cor_acc;
        ta.net = ca.net;
        ta.finalize = ca.finalize;
        ta.grid_ctas = s->num_sms;
        ta.ctrl = s->ctrl;
        if (mode == 1) {
            // split the window's trials over G groups per tile pair, G minimizing the busiest
            // CTA's work: ceil(units / SMs) units of ceil(K / G) trials each (ties: fewer groups)
            const long long k_est = s->W > 0 ? std::min<long long>(s->W, s->enqueued + count) : s->enqueued + count;
            int G = 1;
            long long best = -1;
            for (int g = 1; g <= std::min<long long>(k_est, 64); ++g) {
                const long long rounds = ((long long)s->cor_ntp * g + s->num_sms - 1) / s->num_sms;
                const long long cost = rounds * ((k_est + g - 1) / g);
                if (best < 0 || cost < best) {
                    best = cost;
                    G = g;
                }
            }
            if (G > 1) {
                const size_t need = (size_t)G * 2 * s->P;
                if (s->cor_part_len < need) {
                    if (s->cor_part) cudaFree(s->cor_part);
                    s->cor_part = nullptr;
                    s->cor_part_len = 0;
                    CK(cudaMalloc(&s->cor_part, need * sizeof(float)));
                    s->cor_part_len = need;
                }
                ca.groups = ta.groups = G;
                ca.part = ta.part = s->cor_part;
            }
        }
        LAUNCH(FC_K_COR, launch_cor_normalize(ca, s->stream));
        LAUNCH(FC_K_COR, launch_cor_tc_pack(ta, s->stream));
        LAUNCH(FC_K_COR, launch_cor_tc(ta, s->stream));
        if (ta.groups > 1) LAUNCH(FC_K_COR, launch_cor_combine(ca, s->stream));
    }
    if (s->time_mask & FC_XCOR) {
        XcorArgs xa = xcor_args(s, x, count, write_from, mode);
        LAUNCH(FC_K_XCOR, launch_xcor_spectra(xa, s->stream));
        LAUNCH(FC_K_XCOR, launch_xcor_pairs(xa, s->stream));
        LAUNCH(FC_K_XCOR, launch_xcor_update(xa, s->stream));
    }
    return FC_OK;
}

// Bin groups of the tensor-core full window: units are (128-node tile pair, group of
// consecutive selected bins), one CTA walks a unit's bins in order. Chooses the number of
// groups g <= cap minimizing the busiest CTA's bins (ceil(units / SMs) rounds of a group's
// bins, ~17 us per tile pair and bin as measured on GB300) plus the band-sum planes' traffic
// (write-back and final sum: ~8 B per pair, metric and group at ~6 TB/s); every group holds
// at least one bin.
void herk_groups(long long ntp, int nsel, int sms, long long P, int cap, int& groups, int& group_bins) {
    groups = 1;
    group_bins = nsel;
    double best = 1e300;
    for (int g = 1; g <= std::min(nsel, std::max(1, cap)); ++g) {
        const int gb = (nsel + g - 1) / g;
        if ((nsel + gb - 1) / gb != g) continue;  // a group would be empty
        const long long rounds = (ntp * g + sms - 1) / sms;
        const double t = (double)rounds * gb * 17e-6 + (double)g * 3 * P * 8 / 6e12;
        if (t < best) {
            best = t;
            groups = g;
            group_bins = gb;
        }
    }
}

// Bin groups of the non-linear sums kernel (one CTA per 32-node tile pair and group of
// selected bins, nonlinear_ctas_per_sm() CTAs per SM): the count g <= cap minimizing the
// busiest slot's work (ceil(ntp g / slots) rounds of ceil(nsel / g) bins of K trials, about
// 0.1 us per bin and trial) plus, for g > 1, writing and reducing the g x 4 band planes
// (~5 TB/s); every group holds at least one bin.
void nonlin_groups(long long ntp, int nsel, long long P, int K, int sms, int cap, int& groups, int& group_bins) {
    groups = 1;
    group_bins = nsel;
    const long long slots = (long long)sms * nonlinear_ctas_per_sm();
    double best = -1.0;
    for (int g = 1; g <= std::min(nsel, std::max(1, cap)); ++g) {
        const int gb = (nsel + g - 1) / g;
        if ((nsel + gb - 1) / gb != g) continue;
        const long long rounds = (ntp * g + slots - 1) / slots;
        const double t = (double)rounds * gb * (K > 0 ? K : 1) * 0.1e-6 + (g > 1 ? g * 4.0 * (double)P * 8.0 / 5.0e12 : 0.0);
        if (best < 0.0 || t < best) {
            best = t;
            groups = g;
            group_bins = gb;
        }
    }
}

// Column tiles per resident-operand work item: longer segments reuse the row tile's operands
// more, but every CTA's band sums (a segment's tile pairs x 3 planes) must stay in L2 while
// its bins are added: 152 CTAs x 6 tile pairs x up to 192 KB exceeded the 129 MB L2 and sent
// the reductions to DRAM.
constexpr int kHerkSegTiles = 3;

// Bin groups of the resident-operand tensor-core form: work items are 2 phases x groups x
// nseg segments (a row tile and at most seg_max column tiles); the count g <= cap minimizing
// the busiest CTA's work (ceil(items / SMs) rounds of a group's bins, each bin ~1.2 us per
// column tile plus ~1.5 us to fill the resident operands) plus the band-sum planes' traffic
// (write-back and final sum: ~8 B per pair, metric and group at ~6 TB/s).
void herk_res_groups(int nseg, int seg_max, int nsel, int sms, long long P, int cap, int& groups, int& group_bins) {
    groups = 1;
    group_bins = nsel;
    double best = 1e300;
    for (int g = 1; g <= std::min(nsel, std::max(1, cap)); ++g) {
        const int gb = (nsel + g - 1) / g;
        if ((nsel + gb - 1) / gb != g) continue;
        const long long rounds = (2LL * nseg * g + sms - 1) / sms;
        const double t = (double)rounds * gb * (seg_max * 1.2e-6 + 1.5e-6) + (double)g * 3 * P * 8 / 6e12;
        if (t < best) {
            best = t;
            groups = g;
            group_bins = gb;
        }
    }
}

// Spectral pair sums over the whole window (bulk push, re-sum, full mode).
fc_status stage_window(fc_session* s, int count, bool write_acc) {
    NodeArgs na{s->ring, s->psd, s->inv_psd, s->slots, s->n, s->B, s->W, 1, s->ctrl, count};
    const bool mixed_full = s->ops && !s->mixed_stream && !write_acc;
    if (mixed_full || s->mixed_stream) na.tiny = s->tiny_flags;  // read by the non-linear sums
    LAUNCH(FC_K_NODE, launch_node(na, s->stream));
    if (mixed_full) {
        // mixed precision: linear sums (COH, IMAGCOHY, PLV) on the tensor cores, the
        // non-linear sums (PLI, USPLI, WPLI, DSWPLI) on the CUDA cores
        PackArgs pk{};
        pk.ring = s->ring;
        pk.ops = s->ops;
        pk.n = s->n;
        pk.B = s->B;
        pk.W = s->W;
        pk.slots = s->slots;
        pk.ntiles = s->nt128;
        pk.nchunks = s->nchunks;
        pk.count = count;
        pk.ab_format = s->ab_format;
        pk.ctrl = s->ctrl;
        pk.ring_order = 1;  // operands by ring slot: a single push rewrites one slot only
        pk.last_kc = s->last_kc;
        HerkArgs ha{};
        ha.ops = s->ops;
        ha.tile_a = s->tile_a128;
        ha.tile_b = s->tile_b128;
        ha.inv_psd = s->inv_psd;
        ha.part = s->herk_part;
        ha.net = s->net;
        ha.n = s->n;
        ha.B = s->B;
        ha.ntp = s->ntp128;
        ha.nchunks = s->nchunks;
        ha.W = s->W;
        ha.count = count;
        ha.ab_format = s->ab_format;
        ha.grid_ctas = s->num_sms;
        ha.P = s->P;
        ha.mask = s->mask;
        ha.fsel0 = s->sel0;
        ha.fsel1 = s->sel1;
        ha.ctrl = s->ctrl;
        ha.seg_a = s->seg_a;
        ha.seg_b0 = s->seg_b0;
        ha.seg_b1 = s->seg_b1;
        ha.nseg = s->nseg;
        ha.seg_max = s->seg_max;
        ha.last_kc = s->last_kc;
        if (s->mask & (FC_COH | FC_IMAGCOHY | FC_PLV)) {
            if (s->seg_a)
                herk_res_groups(s->nseg, s->seg_max, s->sel1 - s->sel0, s->num_sms, (long long)s->P, s->herk_gcap,
                                ha.groups, ha.group_bins);
            else
                herk_groups(s->ntp128, s->sel1 - s->sel0, s->num_sms, (long long)s->P, s->herk_gcap, ha.groups,
                            ha.group_bins);
            if (count == 1)  // the new trial's slot (it held the trial that left)
                LAUNCH(FC_K_HERK_TC, launch_pack_ring(pk, 2, s->stream));
            else if (count > 1)  // the whole window (a band change, count 0, keeps the operands)
                LAUNCH(FC_K_HERK_TC, launch_pack_operands(pk, s->stream));
            LAUNCH(FC_K_HERK_TC, launch_herk_tc(ha, s->stream));
            LAUNCH(FC_K_BAND_REDUCE, launch_herk_band(ha, s->stream));
        }
        PairArgs pn = pair_args(s, false, count);
        pn.mask = s->mask & (FC_PLI | FC_USPLI | FC_WPLI | FC_DSWPLI);
        pn.tiny = s->tiny_flags;
        const long long k_est = std::min<long long>(s->W, s->enqueued + count);
        nonlin_groups(s->ntp, s->sel1 - s->sel0, s->P, (int)k_est, s->num_sms, s->partial_groups, pn.groups,
                      pn.group_bins);
        if (pn.mask) {
            LAUNCH(FC_K_WINDOW, launch_nonlinear_sums(pn, s->stream));
            if (pn.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pn, s->stream));
        }
        return FC_OK;
    }
    PairArgs pa = pair_args(s, false, count);
    pa.write_acc = write_acc ? 1 : 0;
    pa.finalize = (s->mask & FC_SPECTRAL_METRICS) ? 1 : 0;
    LAUNCH(FC_K_WINDOW, launch_window_sums(pa, s->stream));
    if (pa.finalize && pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
    return FC_OK;
}

// Drift reset of the streaming sums, spread over the pushes: push r of every period of R
// pushes (R = resum_period, default W) re-sums the tile pairs [ntp r / R, ntp (r+1) / R)
// from the stored spectra of the window, after the streaming update of that push, so every
// accumulator block is recomputed exactly once per R pushes and no push carries a whole
// window's recompute. The per-node PSD sums are re-summed at r = 0.
bool resum_on(const fc_session* s) { return s->W > 0 && s->cfg.resum_period >= 0; }

int push_node_mode(const fc_session* s) { return (resum_on(s) && s->resum_phase == 0) ? 1 : 0; }

PackArgs ring_pack_args(fc_session* s, int count) {
    PackArgs pk{};
    pk.ring = s->ring;
    pk.ops = s->ops;
    pk.n = s->n;
    pk.B = s->B;
    pk.W = s->W;
    pk.slots = s->slots;
    pk.ntiles = s->nt128;
    pk.nchunks = s->nchunks;
    pk.count = count;
    pk.ab_format = s->ab_format;
    pk.ctrl = s->ctrl;
    pk.last_kc = s->last_kc;
    return pk;
}

// Mixed-precision streaming: push r of a period re-sums the 128-node tile pairs
// [ntp128 r / R, ntp128 (r + 1) / R): their linear sums (CSD re, phasor re and im) from the
// tensor cores over the operand ring, their non-linear sums (sum Im, sum |Im|, sum Im^2,
// signs) from the non-linear sums kernel on the 32-node tile pairs inside them. The ring
// takes this push's trial first (and drops the one leaving the window).
// The tensor-core part: linear sums of 128-node tile pairs p0 .. p1 - 1 into the state.
fc_status resum_mixed_linear(fc_session* s, int p0, int p1) {
    HerkArgs ha{};
    ha.ops = s->ops;
    ha.tile_a = s->tile_a128;
    ha.tile_b = s->tile_b128;
    ha.inv_psd = s->inv_psd;
    ha.n = s->n;
    ha.B = s->B;
    ha.ntp = p1 - p0;
    ha.tp0 = p0;
    ha.nchunks = s->nchunks;
    ha.W = s->W;
    ha.count = 1;
    ha.ab_format = s->ab_format;
    ha.grid_ctas = s->num_sms;
    ha.groups = s->B;  // one bin per unit: no band order to keep
    ha.group_bins = 1;
    ha.P = s->P;
    ha.mask = s->mask;
    ha.fsel0 = 0;      // every computed bin: these are the accumulators, not the band average
    ha.fsel1 = s->B;
    ha.ctrl = s->ctrl;
    ha.acc_out = s->acc;
    ha.nt32 = s->nt;
    ha.last_kc = s->last_kc;
    LAUNCH(FC_K_HERK_TC, launch_herk_tc(ha, s->stream));
    return FC_OK;
}

// The non-linear sums (sum Im, sum |Im|, sum Im^2, signs) of the 32-node tile pairs inside
// 128-node tile pairs p0 .. p1 - 1: into the state, or (scratch) into the session's scratch
// by list position, on stream st.
fc_status resum_mixed_nonlinear(fc_session* s, int p0, int p1, bool scratch, cudaStream_t st) {
    PairArgs pa = pair_args(s, false, 1);
    pa.tp_list = s->list32;
    pa.tp0 = s->list32_off[p0];
    pa.tp_count = s->list32_off[p1] - s->list32_off[p0];
    pa.tiny = s->tiny_flags;
    pa.fsel0 = 0;
    pa.fsel1 = s->B;
    // bins per CTA: as many as keep about eight waves of resident CTAs
    const long long waves = 8LL * s->num_sms * nonlinear_ctas_per_sm();
    pa.group_bins = (int)std::max(1LL, std::min<long long>(s->B, (long long)pa.tp_count * s->B / std::max(1LL, waves)));
    pa.groups = (s->B + pa.group_bins - 1) / pa.group_bins;
    if (scratch) {
        pa.acc = s->resum_scratch;
        pa.acc_by_pos = 1;
    }
    LAUNCH_ON(FC_K_WINDOW, st, launch_nonlinear_acc(pa, st));
    return FC_OK;
}

fc_status stage_resum_slice_mixed(fc_session* s, long long r, long long R) {
    PackArgs pk = ring_pack_args(s, 1);
    LAUNCH(FC_K_HERK_TC, launch_pack_ring(pk, 0, s->stream));
    const int p0 = (int)(s->ntp128 * r / R), p1 = (int)(s->ntp128 * (r + 1) / R);
    if (p1 <= p0) return FC_OK;
    fc_status st = resum_mixed_linear(s, p0, p1);
    if (st != FC_OK) return st;
    return resum_mixed_nonlinear(s, p0, p1, false, s->stream);
}

// The slice phase of this push (r of R), advancing the session's phase.
void next_resum_phase(fc_session* s, long long& r, long long& R) {
    R = s->cfg.resum_period > 0 ? s->cfg.resum_period : s->W;
    r = s->resum_phase % R;
    s->resum_phase = (r + 1) % R;
}

fc_status stage_resum_slice(fc_session* s) {
    if (!resum_on(s)) return FC_OK;
    long long r, R;
    next_resum_phase(s, r, R);
    if (s->mixed_stream) return stage_resum_slice_mixed(s, r, R);
    const int tp0 = (int)(s->ntp * r / R), tp1 = (int)(s->ntp * (r + 1) / R);
    if (tp1 <= tp0) return FC_OK;
    PairArgs pa = pair_args(s, false, 1);
    pa.write_acc = 1;
    pa.finalize = 0;
    pa.tp0 = tp0;
    pa.tp_count = tp1 - tp0;
    pa.groups = s->B;  // one CTA per (tile pair, bin): a slice still fills the GPU
    pa.group_bins = 1;
    LAUNCH(FC_K_WINDOW, launch_window_sums(pa, s->stream));
    return FC_OK;
}

// Streaming update of one trial with the exact re-sum slice of the push overlapped (FP32
// stream sessions). The update (k_stream, two persistent CTAs per SM: fewer leave HBM
// under-used, 11.2 instead of 9.6 ms per launch at 1.5 per SM) is launched first; the slice
// runs on the session's lowest-priority side stream, so its CTAs take the SMs that the
// update's CTAs leave as they finish their units, writing its blocks into the scratch,
// which then replaces the slice's blocks in the state (unless the push was rejected). The
// networks come from the streaming state and the state ends as the slice's sums: the same
// arithmetic and order of effects as the update followed by the slice.

// Marks the point of the session stream after which the slice may start (the push's
// spectra and per-node sums are in), creating the side stream on first use.
fc_status resum_fork_point(fc_session* s) {
    if (!s->side_stream) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&s->side_stream, cudaStreamNonBlocking, least));
        CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(s->ev_fork, s->stream));
    return FC_OK;
}

// This push's slice: 32-node tile pairs [t0, t1) of an FP32 session, 128-node tile pairs of
// a mixed-precision one (advances the session's re-sum phase); false when it is empty.
bool resum_range(fc_session* s, int& t0, int& t1) {
    long long r, R;
    next_resum_phase(s, r, R);
    const long long nt = s->mixed_stream ? s->ntp128 : s->ntp;
    t0 = (int)(nt * r / R);
    t1 = (int)(nt * (r + 1) / R);
    return t1 > t0;
}

// The slice [t0, t1) on the side stream, into the scratch: the whole exact re-sum of an FP32
// session; the operand-ring update and the non-linear sums of a mixed-precision one.
fc_status resum_fork(fc_session* s, int t0, int t1) {
    CK(cudaStreamWaitEvent(s->side_stream, s->ev_fork, 0));
    if (s->mixed_stream) {
        PackArgs pk = ring_pack_args(s, 1);
        LAUNCH_ON(FC_K_OTHER, s->side_stream, launch_pack_ring(pk, 0, s->side_stream));
        fc_status st = resum_mixed_nonlinear(s, t0, t1, true, s->side_stream);
        if (st != FC_OK) return st;
        CK(cudaEventRecord(s->ev_join, s->side_stream));
        return FC_OK;
    }
    const int tp0 = t0, tp1 = t1;
    PairArgs ps = pair_args(s, false, 1);
    ps.write_acc = 1;
    ps.finalize = 0;
    ps.tp0 = tp0;
    ps.tp_count = tp1 - tp0;
    ps.groups = s->B;  // one CTA per (tile pair, bin)
    ps.group_bins = 1;
    ps.acc = s->resum_scratch;
    ps.acc_tp_base = tp0;
    LAUNCH_ON(FC_K_WINDOW, s->side_stream, launch_window_sums(ps, s->side_stream));
    CK(cudaEventRecord(s->ev_join, s->side_stream));
    return FC_OK;
}

// After the update: the scratch over the slice's blocks (skipped for a rejected push); for a
// mixed-precision session first the tensor-core linear sums straight into the state, then
// the non-linear planes from the scratch.
fc_status resum_join(fc_session* s, int t0, int t1) {
    CK(cudaStreamWaitEvent(s->stream, s->ev_join, 0));
    if (s->mixed_stream) {
        fc_status st = resum_mixed_linear(s, t0, t1);
        if (st != FC_OK) return st;
        const int off = s->list32_off[t0], cnt = s->list32_off[t1] - off;
        LAUNCH(FC_K_OTHER, launch_gather_nonlinear(s->resum_scratch, s->acc, s->list32 + off, cnt, s->B, s->ctrl,
                                                   s->stream));
        return FC_OK;
    }
    const int tp0 = t0, tp1 = t1;
    const long long words = (long long)(tp1 - tp0) * s->B * FC_BLOCK_WORDS;
    LAUNCH(FC_K_OTHER, launch_copy_blocks(s->resum_scratch, s->acc + (size_t)tp0 * s->B * FC_BLOCK_WORDS, words,
                                          s->ctrl, s->stream));
    return FC_OK;
}

fc_status push_stream_overlapped(fc_session* s, PairArgs pa) {
    int t0, t1;
    const bool slice = resum_range(s, t0, t1);
    fc_status st;
    if (slice && (st = resum_fork_point(s)) != FC_OK) return st;
    LAUNCH(FC_K_STREAM, launch_stream_update(pa, s->stream));
    if (slice) {
        if ((st = resum_fork(s, t0, t1)) != FC_OK) return st;
        if ((st = resum_join(s, t0, t1)) != FC_OK) return st;
    } else if (s->mixed_stream) {  // the operand ring takes the trial every push
        PackArgs pk = ring_pack_args(s, 1);
        LAUNCH(FC_K_HERK_TC, launch_pack_ring(pk, 0, s->stream));
    }
    if (pa.finalize && pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
    return FC_OK;
}

// One trial through the streaming path: x points at one [n][N] trial on the device.
fc_status push_one_stream(fc_session* s, const float* x, bool finalize) {
    const long long nx = (long long)(s->spec_project ? s->proj_C : s->n) * s->N;
    LAUNCH(FC_K_OTHER, launch_validate(x, nx, s->ctrl, s->stream));
    fc_status st;
    if (s->spectral) {
        st = stage_spectra(s, x, 1, 0);
        if (st != FC_OK) return st;
        NodeArgs na{s->ring, s->psd, s->inv_psd, s->slots, s->n, s->B, s->W, push_node_mode(s), s->ctrl, 1};
        if (s->mixed_stream) na.tiny = s->tiny_flags;
        LAUNCH(FC_K_NODE, launch_node(na, s->stream));
        PairArgs pa = pair_args(s, true, 1);
        pa.finalize = (finalize && (s->mask & FC_SPECTRAL_METRICS)) ? 1 : 0;
        if (s->resum_scratch && resum_on(s)) {
            st = push_stream_overlapped(s, pa);
            if (st != FC_OK) return st;
        } else {
            LAUNCH(FC_K_STREAM, launch_stream_update(pa, s->stream));
            if (pa.finalize && pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
            st = stage_resum_slice(s);
            if (st != FC_OK) return st;
        }
    }
    st = stage_time_metrics(s, x, 1, 0, 0);
    if (st != FC_OK) return st;
    CommitArgs ca{s->ctrl, 1};
    LAUNCH(FC_K_OTHER, launch_commit(ca, s->stream));
    s->enqueued += 1;
    return FC_OK;
}

// Many trials at once, then one window computation (stream bulk or full mode).
fc_status push_bulk(fc_session* s, const float* x, int count, bool write_acc) {
    const long long nx = (long long)(s->spec_project ? s->proj_C : s->n) * s->N;
    LAUNCH(FC_K_OTHER, launch_validate(x, nx * count, s->ctrl, s->stream));
    const int keep = s->W > 0 ? std::min(count, s->W) : count;
    const int write_from = count - keep;
    fc_status st;
    if (s->spectral) {
        st = stage_spectra(s, x, count, write_from);
        if (st != FC_OK) return st;
        st = stage_window(s, count, write_acc);
        if (st != FC_OK) return st;
        if (s->mixed_stream) {  // the operand ring of the new window
            PackArgs pk = ring_pack_args(s, count);
            LAUNCH(FC_K_HERK_TC, launch_pack_ring(pk, 1, s->stream));
        }
    }
    st = stage_time_metrics(s, x, count, write_from, 1);
    if (st != FC_OK) return st;
    CommitArgs ca{s->ctrl, count};
    LAUNCH(FC_K_OTHER, launch_commit(ca, s->stream));
    s->enqueued += count;
    return FC_OK;
}

// Bin groups of the full-window kernels (one CTA per tile pair and group of bins, two CTAs
// per SM): the count minimizing an estimate of the time, the busiest slot's work
// (ceil(ntp g / (2 SMs)) rounds of ceil(B / g) bins, about 0.67 us per bin and trial of the
// window) plus, for g > 1, writing and reducing g x 7 band planes of P pairs (~5 TB/s).
void window_groups(long long ntp, int B, long long P, int K, int sms, int& groups, int& group_bins) {
    double best = -1.0;
    groups = 1;
    group_bins = B;
    const double us_per_bin = 0.67 * (K > 0 ? K : 100);
    for (int g = 1; g <= B; ++g) {
        const int gb = (B + g - 1) / g;
        if ((B + gb - 1) / gb != g) continue;  // g groups of gb bins cover B exactly
        const long long rounds = (ntp * g + 2LL * sms - 1) / (2LL * sms);
        const double t = (double)rounds * gb * us_per_bin + (g > 1 ? g * 7.0 * (double)P * 8.0 / 5.0e6 : 0.0);
        if (best < 0.0 || t < best) {
            best = t;
            groups = g;
            group_bins = gb;
        }
    }
}

// Streams and events of the pipelined host I/O, created on first use.
fc_status ensure_io(fc_session* s) {
    if (s->in_stream) return FC_OK;
    CK(cudaStreamCreateWithFlags(&s->in_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&s->out_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t* e : {&s->ev_in[b], &s->ev_used[b], &s->ev_snap[b], &s->ev_out[b]})
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return FC_OK;
}

// Host -> device copy ordered on the session stream, complete on return (the host buffer
// may be pageable and temporary).
fc_status upload(fc_session* s, void* dst, const void* src, size_t bytes) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return FC_OK;
}

fc_status ensure_stage(fc_session* s, int count) {
    if (count <= s->stage_trials) return FC_OK;
    void* p;
    fc_status st = dev_alloc(s, (size_t)count * s->n * s->N * sizeof(float), &p);
    if (st != FC_OK) return st;
    s->x_stage = static_cast<float*>(p);
    s->stage_trials = count;
    return FC_OK;
}

fc_status read_ctrl(fc_session* s, FcCtrl* h) {
    CK(cudaMemcpyAsync(h, s->ctrl, sizeof(FcCtrl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (h->scale != 0.f) s->calibrated = true;
    return FC_OK;
}

fc_status check_latched(fc_session* s, FcCtrl* h) {
    fc_status st = read_ctrl(s, h);
    if (st != FC_OK) return st;
    if (h->timeout)
        return fail(FC_ERR_TIMEOUT, "a bounded device-side wait ran out; the session state is unreliable");
    if (h->bad_latched) {
        CK(cudaMemsetAsync(&s->ctrl->bad_latched, 0, sizeof(int), s->stream));
        CK(cudaStreamSynchronize(s->stream));
        return fail(FC_ERR_NONFINITE, "a pushed trial held NaN or Inf and was rejected (%lld rejected so far)",
                    h->rejected);
    }
    return FC_OK;
}

}  // namespace

void fc_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }

int fc_device_sms(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    if (device >= 64) device = 63;
    std::lock_guard<std::mutex> lk(mu);
    if (cache[device] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v < 1) {
            cudaGetLastError();
            return 152;  // not cached: the next call asks again
        }
        cache[device] = v;
    }
    return cache[device];
}

// ------------------------------------------------- streaming push in pieces (serving)
bool fc_push_needs_single(fc_session* s) {
    return !s->calibrated || s->time_mask != 0 || s->cfg.mode != FC_MODE_STREAM;
}

fc_status fc_push_single(fc_session* s, const float* xdev) {
    if (s->cfg.mode == FC_MODE_FULL) return push_bulk(s, xdev, 1, false);
    return push_one_stream(s, xdev, true);
}

PairArgs fc_push_stream_args(fc_session* s) {
    PairArgs pa = pair_args(s, true, 1);
    pa.finalize = (s->mask & FC_SPECTRAL_METRICS) ? 1 : 0;
    return pa;
}

// The same stages for several sessions at once (one launch per stage for all of them);
// every session must be one fc_push_needs_single declines, all on the stream st.
fc_status fc_push_batch_pre(fc_session* const* ss, const float* const* x, int count, cudaStream_t st) {
    if (count <= 0) return FC_OK;
    if (count > FC_MAX_BATCH) return fail(FC_ERR_INVALID_ARG, "batch of %d sessions (at most %d)", count, FC_MAX_BATCH);
    PreBatch b;
    b.nsess = count;
    b.val_prefix[0] = 0;
    b.spec_prefix[0] = 0;
    b.node_prefix[0] = 0;
    for (int i = 0; i < count; ++i) {
        fc_session* s = ss[i];
        b.sp[i] = spectrum_args(s, x[i], 1, 0);
        b.nd[i] = NodeArgs{s->ring, s->psd, s->inv_psd, s->slots, s->n, s->B, s->W, push_node_mode(s), s->ctrl, 1};
        if (s->mixed_stream) b.nd[i].tiny = s->tiny_flags;
        b.val_prefix[i + 1] = b.val_prefix[i] + (long long)s->n * s->N;
        // (sessions on the FFT method are launched on their own: no CTA of the batched kernel)
        b.spec_prefix[i + 1] = b.spec_prefix[i] + (s->use_fft ? 0 : ((s->n + 31) / 32) * ((s->B + 31) / 32));
        b.node_prefix[i + 1] = b.node_prefix[i] + s->B * s->n;
    }
    fc_session* s = ss[0];  // launches are counted (and timed) on the first session
    LAUNCH(FC_K_OTHER, launch_validate_batch(b, st));
    LAUNCH(FC_K_SPECTRUM, launch_spectrum_batch(b, st));
    LAUNCH(FC_K_NODE, launch_node_batch(b, st));
    // drift re-sum slices (FP32 sessions: the exact re-sum; mixed-precision sessions: its
    // non-linear sums): set up here (their inputs are in), launched by fc_push_batch_fork
    // beside the update, put into the state by fc_push_batch_post
    for (int i = 0; i < count; ++i) {
        fc_session* si = ss[i];
        if (!si->resum_scratch || !resum_on(si) || si->resum_pending) continue;
        if (!resum_range(si, si->resum_tp0, si->resum_tp1)) {
            si->resum_tp0 = si->resum_tp1 = -1;  // empty phase (a mixed session's ring still takes the trial)
            continue;
        }
        fc_status fst = resum_fork_point(si);
        if (fst != FC_OK) return fst;
        si->resum_pending = true;
        si->resum_forked = false;
    }
    return FC_OK;
}

fc_status fc_push_batch_fork(fc_session* const* ss, int count) {
    for (int i = 0; i < count; ++i) {
        fc_session* s = ss[i];
        if (!s->resum_pending || s->resum_forked) continue;
        fc_status st = resum_fork(s, s->resum_tp0, s->resum_tp1);
        if (st != FC_OK) return st;
        s->resum_forked = true;
    }
    return FC_OK;
}

fc_status fc_push_batch_post(fc_session* const* ss, FcCtrl* const* snap, int count, cudaStream_t st) {
    if (count <= 0) return FC_OK;
    if (count > FC_MAX_BATCH) return fail(FC_ERR_INVALID_ARG, "batch of %d sessions (at most %d)", count, FC_MAX_BATCH);
    CommitBatch b;
    b.nsess = count;
    for (int i = 0; i < count; ++i) {
        fc_session* s = ss[i];
        PairArgs pa = fc_push_stream_args(s);
        if (pa.finalize && pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
        fc_status r;
        if (s->resum_pending) {  // the slice forked at the push's first share
            if (!s->resum_forked && (r = resum_fork(s, s->resum_tp0, s->resum_tp1)) != FC_OK) return r;
            if ((r = resum_join(s, s->resum_tp0, s->resum_tp1)) != FC_OK) return r;
            s->resum_pending = s->resum_forked = false;
        } else if (!s->resum_scratch) {
            if ((r = stage_resum_slice(s)) != FC_OK) return r;
        } else if (s->mixed_stream && resum_on(s)) {  // empty phase: the operand ring takes the trial
            PackArgs pk = ring_pack_args(s, 1);
            LAUNCH(FC_K_HERK_TC, launch_pack_ring(pk, 0, s->stream));
        }
        b.ctrl[i] = s->ctrl;
        b.snap[i] = snap ? snap[i] : nullptr;
    }
    fc_session* s = ss[0];
    LAUNCH(FC_K_OTHER, launch_commit_batch(b, st));
    for (int i = 0; i < count; ++i) ss[i]->enqueued += 1;
    return FC_OK;
}

void fc_count_launch(fc_session* s) { s->launches++; }

// Device bytes fc_session_create would allocate for these settings (mirrors its allocations).
int fc_fft_radices(int m, unsigned long long* packed) {
    unsigned long long p = 0;
    int n = 0;
    auto take = [&](int r) {
        while (m % r == 0 && n < 16) {
            p |= (unsigned long long)r << (4 * n++);
            m /= r;
        }
    };
    take(4);
    take(2);
    take(3);
    take(5);
    take(7);
    if (packed) *packed = p;
    return m == 1 ? n : -1;
}

bool fc_fft_size_ok(int nfft) {
    return nfft >= 16 && nfft <= 16384 && nfft % 2 == 0 && fc_fft_radices(nfft / 2, nullptr) >= 0;
}

// Spectrum method. Cost per (trial, node): the band DFT kernel does N x (B rounded up to its
// 32-bin tiles) complex multiply-adds; the warp FFT does per pass and point about one (radix
// 2, 4), two (radix 3), three (radix 5) or four (radix 7) such operations' worth of work,
// times kFftCost for its shared-memory round trips.
bool fc_spectrum_uses_fft(int N, int B, int nfft, fc_spectrum method) {
    if (method == FC_SPECTRUM_DFT || !fc_fft_size_ok(nfft)) return false;
    if (method == FC_SPECTRUM_FFT) return true;
    constexpr double kFftCost = 2.0;
    unsigned long long p = 0;
    const int ns = fc_fft_radices(nfft / 2, &p);
    double per_point = 0.0;
    for (int i = 0; i < ns; ++i) {
        const int r = (int)((p >> (4 * i)) & 15u);
        per_point += r == 7 ? 4.0 : (r == 5 ? 3.0 : (r == 3 ? 2.0 : 1.0));
    }
    const double dft = (double)N * ((B + 31) / 32 * 32);
    const double fft = kFftCost * (double)nfft * per_point;
    return fft < dft;
}

size_t fc_plan_session_bytes(int n, int N, int B, int W, uint32_t mask, fc_mode mode, fc_precision prec, int nfft) {
    const size_t nt = (n + FC_T - 1) / FC_T, ntp = nt * (nt + 1) / 2;
    const size_t P = (size_t)n * (n - 1) / 2;
    const size_t slots = mode == FC_MODE_FULL ? W : (W > 0 ? W + 1 : 1);
    size_t b = 256 + 9 * P * 4 + (size_t)n * N * 4;  // control block, network planes, trial staging
    if (mask & FC_SPECTRAL_METRICS) {
        // spectrum tables: DFT factors [N][B], or the FFT's taper [N] and twiddles [nfft/2]
        b += (nfft > 0 && fc_spectrum_uses_fft(N, B, nfft, FC_SPECTRUM_AUTO)) ? (size_t)N * 4 + (size_t)nfft / 2 * 8
                                                                               : (size_t)N * B * 8;
        b += slots * B * n * 8 + (size_t)B * n * 12 + ntp * 4;
        if (mode == FC_MODE_STREAM) b += ntp * B * FC_BLOCK_WORDS * 4;
        if (mode == FC_MODE_STREAM && prec == FC_PREC_FP32 && W > 0)  // re-sum scratch (period W)
            b += (ntp + W - 1) / W * B * FC_BLOCK_WORDS * 4;
        if (mode == FC_MODE_STREAM && prec != FC_PREC_FP32) {
            // operand ring, 128-node tile lists, the 32-in-128 tile-pair list, tiny-node flags
            const size_t nt128 = (n + 127) / 128, ntp128 = nt128 * (nt128 + 1) / 2;
            const size_t per_chunk = (prec == FC_PREC_TF32 || prec == FC_PREC_TF32X3) ? 32 : 64;
            const size_t nchunks = (2 * slots + per_chunk - 1) / per_chunk;
            const size_t kinds = prec == FC_PREC_TF32X3 ? 8 : 4;  // split TF32: high and low parts
            b += nt128 * B * kinds * nchunks * herk_chunk_bytes() + ntp128 * 4 + ntp * 4 + (size_t)B * n;
            // re-sum scratch: at most 16 32-node tile pairs per 128-node tile pair of a slice
            b += (ntp128 + W - 1) / W * 16 * B * FC_BLOCK_WORDS * 4;
        }
        int wg, wgb;
        const int sms = fc_device_sms();
        window_groups((long long)ntp, B, (long long)P, W, sms, wg, wgb);
        const int groups = std::max(wg, std::min(B, std::max(1, (int)((sms * 4 + ntp - 1) / ntp))));
        if (groups > 1) b += (size_t)groups * 7 * P * 4;
    }
    if (mask & FC_COR)
        b += slots * n * N * 4 + 2 * P * 4 + slots * ((n + 127) / 128) * ((N + 31) / 32) * 32768;
    if (mask & FC_XCOR) {
        size_t L = 1;
        while (L < (size_t)(2 * N - 1)) L *= 2;
        if (L < 64) L = 64;
        b += L / 2 * 8 + slots * n * (L / 2 + 1) * 8 + slots * n * 4 + slots * P * 4 + P * 4 + 2 * P * 4;
    }
    return b;
}

int fc_band_bins(double fs, fc_band band, int* first) {
    int f0 = -1, B = 0;
    for (int k = 0; k <= band.nfft / 2; ++k) {
        const double kf = (double)k * fs;
        if (kf >= band.f_lo * band.nfft && kf < band.f_hi * band.nfft) {
            if (f0 < 0) f0 = k;
            ++B;
        }
    }
    if (first) *first = f0;
    return B;
}

// ====================================================================== public API
extern "C" {

const char* fc_last_error(void) { return g_err.c_str(); }

fc_status fc_config_default(fc_config* cfg) {
    if (!cfg) return fail(FC_ERR_INVALID_ARG, "cfg is NULL");
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = FC_PREC_FP32;
    cfg->mode = FC_MODE_STREAM;
    cfg->resum_period = 0;
    return FC_OK;
}

fc_status fc_session_create(int n_nodes, int n_samples, double fs, fc_band band, fc_taper taper,
                            uint32_t metric_mask, int window, const fc_config* cfg_in,
                            fc_session** out) {
    if (!out) return fail(FC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    fc_config cfg;
    if (cfg_in) cfg = *cfg_in; else fc_config_default(&cfg);
    if (n_nodes < 2 || n_nodes > 65535 * FC_T) return fail(FC_ERR_INVALID_ARG, "n_nodes %d out of range", n_nodes);
    if (n_samples < 1) return fail(FC_ERR_INVALID_ARG, "n_samples %d < 1", n_samples);
    if (!(fs > 0.0) || !std::isfinite(fs)) return fail(FC_ERR_INVALID_ARG, "fs must be positive");
    if (band.nfft < n_samples) return fail(FC_ERR_INVALID_ARG, "nfft %d < n_samples %d", band.nfft, n_samples);
    if (!(band.f_lo < band.f_hi)) return fail(FC_ERR_INVALID_ARG, "band f_lo must be < f_hi");
    if (taper < FC_TAPER_NONE || taper > FC_TAPER_HANN_SYM) return fail(FC_ERR_INVALID_ARG, "bad taper");
    if (metric_mask == 0 || (metric_mask & ~(uint32_t)FC_ALL_METRICS))
        return fail(FC_ERR_INVALID_ARG, "bad metric mask 0x%x", metric_mask);
    if (window < 0) return fail(FC_ERR_INVALID_ARG, "window must be >= 0");
    if (cfg.mode != FC_MODE_STREAM && cfg.mode != FC_MODE_FULL) return fail(FC_ERR_INVALID_ARG, "bad mode");
    if (cfg.mode == FC_MODE_FULL && window < 1) return fail(FC_ERR_INVALID_ARG, "full mode needs window >= 1");
    if (cfg.precision < FC_PREC_FP32 || cfg.precision > FC_PREC_TF32X3) return fail(FC_ERR_INVALID_ARG, "bad precision");
    if (cfg.spectrum < FC_SPECTRUM_AUTO || cfg.spectrum > FC_SPECTRUM_FFT) return fail(FC_ERR_INVALID_ARG, "bad spectrum method");
    if (cfg.spectrum == FC_SPECTRUM_FFT && !fc_fft_size_ok(band.nfft))
        return fail(FC_ERR_UNSUPPORTED,
                    "the FFT spectrum needs an even nfft in 16 .. 16384 whose half has no prime factor above 7 "
                    "(nfft %d)", band.nfft);
    if (cfg.precision != FC_PREC_FP32 && cfg.mode == FC_MODE_STREAM && (window < 1 || cfg.resum_period < 0))
        return fail(FC_ERR_UNSUPPORTED,
                    "a tensor-core precision in stream mode applies to the drift re-sum of a sliding window "
                    "(window >= 1, resum_period >= 0)");
    if ((cfg.dev_alloc == nullptr) != (cfg.dev_free == nullptr))
        return fail(FC_ERR_INVALID_ARG, "dev_alloc and dev_free must be given together");
    // band bins: f_lo <= k fs / nfft < f_hi
    int first = -1, B = 0;
    for (int k = 0; k <= band.nfft / 2; ++k) {
        const double kf = (double)k * fs;
        if (kf >= band.f_lo * band.nfft && kf < band.f_hi * band.nfft) {
            if (first < 0) first = k;
            ++B;
        }
    }
    if (B == 0) return fail(FC_ERR_INVALID_ARG, "the band selects no bin");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(FC_ERR_CUDA, "no CUDA device: this library has no CPU path");
    }

    fc_session* s = new (std::nothrow) fc_session();
    if (!s) return fail(FC_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->n = n_nodes;
    s->N = n_samples;
    s->B = B;
    s->sel0 = 0;
    s->sel1 = B;
    s->first_bin = first;
    s->nfft = band.nfft;
    s->W = window;
    s->fs = fs;
    s->band = band;
    s->taper = taper;
    s->mask = metric_mask;
    s->time_mask = metric_mask & (FC_COR | FC_XCOR);
    s->spectral = (metric_mask & FC_SPECTRAL_METRICS) != 0;
    s->cfg = cfg;
    s->nt = (n_nodes + FC_T - 1) / FC_T;
    s->ntp = s->nt * (s->nt + 1) / 2;
    s->P = (long long)n_nodes * (n_nodes - 1) / 2;
    s->slots = cfg.mode == FC_MODE_FULL ? window : (window > 0 ? window + 1 : 1);
    s->use_fft = fc_spectrum_uses_fft(n_samples, B, band.nfft, cfg.spectrum);
    cudaGetDevice(&s->device);
    s->num_sms = fc_device_sms(s->device);

    auto cleanup = [&](fc_status st) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        free_all(s);
        if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return st;
    };

    if (cfg.stream) {
        s->stream = static_cast<cudaStream_t>(cfg.stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(fail(FC_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
        s->own_stream = true;
    }

    // work split: enough CTAs to fill every SM twice over (two CTAs per SM)
    const int target = s->num_sms * 4;
    s->stream_groups = std::min(B, std::max(1, (target + s->ntp - 1) / s->ntp));
    s->stream_group_bins = (B + s->stream_groups - 1) / s->stream_groups;
    s->stream_groups = (B + s->stream_group_bins - 1) / s->stream_group_bins;
    window_groups(s->ntp, B, s->P, window, s->num_sms, s->groups, s->group_bins);
    const int max_groups = std::max(s->groups, s->stream_groups);

    fc_status st;
#define TRY(x) do { st = (x); if (st != FC_OK) return cleanup(st); } while (0)
    TRY(alloc_zero(s, 1, &s->ctrl));
    // spectral state only when the session has spectral metrics (a COR / XCOR session holds none)
    if (s->spectral) {
        auto taper_at = [&](int t) {
            double w = 1.0;
            if (taper == FC_TAPER_HANN) w = 0.5 - 0.5 * std::cos(2.0 * kPi * t / n_samples);
            if (taper == FC_TAPER_HANN_SYM) w = n_samples > 1 ? 0.5 - 0.5 * std::cos(2.0 * kPi * t / (n_samples - 1)) : 1.0;
            return w;
        };
        if (s->use_fft) {
            // real FFT: the taper and the twiddles e^{-2 pi i k / nfft}, FP64 on the host
            std::vector<float> wt(n_samples);
            for (int t = 0; t < n_samples; ++t) wt[t] = (float)taper_at(t);
            std::vector<float2> ft(band.nfft / 2);
            for (int k = 0; k < band.nfft / 2; ++k) {
                const double ang = 2.0 * kPi * (double)k / band.nfft;
                ft[k] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
            }
            TRY(alloc_zero(s, wt.size(), &s->taper_tab));
            TRY(alloc_zero(s, ft.size(), &s->fft_tw));
            TRY(upload(s, s->taper_tab, wt.data(), wt.size() * sizeof(float)));
            TRY(upload(s, s->fft_tw, ft.data(), ft.size() * sizeof(float2)));
        } else {
            // taper-folded DFT factors, FP64 on the host with exact angle reduction
            std::vector<float2> tw((size_t)n_samples * B);
            for (int t = 0; t < n_samples; ++t) {
                const double w = taper_at(t);
                for (int b = 0; b < B; ++b) {
                    const long long m = ((long long)(first + b) * t) % band.nfft;
                    const double ang = 2.0 * kPi * (double)m / band.nfft;
                    tw[(size_t)t * B + b] = make_float2((float)(w * std::cos(ang)), (float)(-w * std::sin(ang)));
                }
            }
            TRY(alloc_zero(s, tw.size(), &s->twiddle));
            cudaError_t e = cudaMemcpyAsync(s->twiddle, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return cleanup(fail(FC_ERR_CUDA, "twiddle upload: %s", cudaGetErrorString(e)));
            cudaStreamSynchronize(s->stream);
        }
        TRY(alloc_zero(s, (size_t)s->slots * B * n_nodes, &s->ring));
        TRY(alloc_zero(s, (size_t)B * n_nodes, &s->psd));
        TRY(alloc_zero(s, (size_t)B * n_nodes, &s->inv_psd));
        {
            std::vector<unsigned short> ta, tb;
            for (int a = 0; a < s->nt; ++a)
                for (int b = a; b < s->nt; ++b) {
                    ta.push_back((unsigned short)a);
                    tb.push_back((unsigned short)b);
                }
            TRY(alloc_zero(s, ta.size(), &s->tile_a));
            TRY(alloc_zero(s, tb.size(), &s->tile_b));
            // on the session stream, after the zero fill of the same buffers (a copy on the legacy
            // stream is not ordered after work on a non-blocking stream)
            TRY(upload(s, s->tile_a, ta.data(), ta.size() * sizeof(unsigned short)));
            TRY(upload(s, s->tile_b, tb.data(), tb.size() * sizeof(unsigned short)));
        }
        if (cfg.mode == FC_MODE_STREAM) TRY(alloc_zero(s, (size_t)s->ntp * B * FC_BLOCK_WORDS, &s->acc));
        if (cfg.mode == FC_MODE_STREAM && cfg.precision == FC_PREC_FP32 && window > 0 && cfg.resum_period >= 0) {
            // the slice of one push: at most ceil(ntp / R) tile pairs, all bins
            const int R = cfg.resum_period > 0 ? cfg.resum_period : window;
            s->resum_scratch_tp = (s->ntp + R - 1) / R;
            TRY(alloc_zero(s, (size_t)s->resum_scratch_tp * B * FC_BLOCK_WORDS, &s->resum_scratch));
        }
        if (cfg.precision != FC_PREC_FP32 && cfg.mode == FC_MODE_STREAM) {
            // mixed-precision streaming: the drift re-sum takes the linear sums from the tensor
            // cores over an operand ring of the window (inner dimension 2 (W + 1): ring slots)
            s->mixed_stream = true;
            s->ab_format = cfg.precision == FC_PREC_BF16 ? 1
                           : cfg.precision == FC_PREC_FP16 ? 0
                           : cfg.precision == FC_PREC_TF32X3 ? 3 : 2;
            const int per_chunk = s->ab_format >= 2 ? 32 : 64;
            s->nchunks = (2 * s->slots + per_chunk - 1) / per_chunk;
            s->nt128 = (n_nodes + 127) / 128;
            s->ntp128 = s->nt128 * (s->nt128 + 1) / 2;
            std::vector<unsigned short> ta, tb;
            std::vector<int> l32;
            s->list32_off.assign(1, 0);
            for (int a = 0; a < s->nt128; ++a)
                for (int b = a; b < s->nt128; ++b) {
                    ta.push_back((unsigned short)a);
                    tb.push_back((unsigned short)b);
                    // the 32-node tile pairs inside this 128-node tile pair
                    for (int x = 4 * a; x < std::min(4 * a + 4, s->nt); ++x)
                        for (int y = std::max(x, 4 * b); y < std::min(4 * b + 4, s->nt); ++y)
                            l32.push_back(x * s->nt - x * (x - 1) / 2 + (y - x));
                    s->list32_off.push_back((int)l32.size());
                }
            TRY(alloc_zero(s, ta.size(), &s->tile_a128));
            TRY(alloc_zero(s, tb.size(), &s->tile_b128));
            TRY(upload(s, s->tile_a128, ta.data(), ta.size() * sizeof(unsigned short)));
            TRY(upload(s, s->tile_b128, tb.data(), tb.size() * sizeof(unsigned short)));
            TRY(alloc_zero(s, l32.size(), &s->list32));
            TRY(upload(s, s->list32, l32.data(), l32.size() * sizeof(int)));
            const size_t kinds = s->ab_format == 3 ? 8 : 4;  // split TF32: high and low parts
            TRY(alloc_zero(s, (size_t)s->nt128 * B * kinds * s->nchunks * herk_chunk_bytes(), &s->ops));
            TRY(alloc_zero(s, (size_t)B * n_nodes, &s->tiny_flags));
            // the non-linear re-sum of one push beside the update: its 32-node tile pairs (at
            // most those inside one slice of 128-node tile pairs), all bins
            const int R = cfg.resum_period > 0 ? cfg.resum_period : window;
            int most = 0;
            for (int r = 0; r < R; ++r) {
                const int p0 = (int)((long long)s->ntp128 * r / R), p1 = (int)((long long)s->ntp128 * (r + 1) / R);
                most = std::max(most, s->list32_off[p1] - s->list32_off[p0]);
            }
            s->resum_scratch_tp = std::max(1, most);
            TRY(alloc_zero(s, (size_t)s->resum_scratch_tp * B * FC_BLOCK_WORDS, &s->resum_scratch));
        }
        if (cfg.precision != FC_PREC_FP32 && cfg.mode == FC_MODE_FULL) {
            s->ab_format = cfg.precision == FC_PREC_BF16 ? 1
                           : cfg.precision == FC_PREC_FP16 ? 0
                           : cfg.precision == FC_PREC_TF32X3 ? 3 : 2;
            const int per_chunk = s->ab_format >= 2 ? 32 : 64;  // inner elements per 128-byte K-chunk
            s->nchunks = (2 * window + per_chunk - 1) / per_chunk;
            s->nt128 = (n_nodes + 127) / 128;
            s->ntp128 = s->nt128 * (s->nt128 + 1) / 2;
            std::vector<unsigned short> ta, tb;
            for (int a = 0; a < s->nt128; ++a)
                for (int b = a; b < s->nt128; ++b) {
                    ta.push_back((unsigned short)a);
                    tb.push_back((unsigned short)b);
                }
            TRY(alloc_zero(s, ta.size(), &s->tile_a128));
            TRY(alloc_zero(s, tb.size(), &s->tile_b128));
            TRY(upload(s, s->tile_a128, ta.data(), ta.size() * sizeof(unsigned short)));
            TRY(upload(s, s->tile_b128, tb.data(), tb.size() * sizeof(unsigned short)));
            const size_t kinds = s->ab_format == 3 ? 8 : 4;  // split TF32: high and low parts
            TRY(alloc_zero(s, (size_t)s->nt128 * B * kinds * s->nchunks * herk_chunk_bytes(), &s->ops));
            TRY(alloc_zero(s, (size_t)B * n_nodes, &s->tiny_flags));
            int gb;
            // (split TF32 takes the streaming-operand form: both parts of a row tile would not
            // stay resident)
            if (s->nchunks <= herk_resident_max_chunks() && s->ab_format != 3) {
                // resident-operand form: each row tile a with its column tiles b >= a in balanced
                // segments of at most kHerkSegTiles tiles. Its operands keep, in the last
                // K-chunk, only the 16-byte columns up to the last K-step that holds inner
                // positions (2 W of them; the rest would be zero padding)
                const int per16 = per_chunk / 8;
                const int units16 = (2 * window + per16 - 1) / per16;
                const int last = units16 - 8 * (s->nchunks - 1);
                s->last_kc = std::min(8, last + (last & 1));
                std::vector<unsigned short> sa, sb0, sb1;
                for (int ta = 0; ta < s->nt128; ++ta) {
                    const int len = s->nt128 - ta, parts = (len + kHerkSegTiles - 1) / kHerkSegTiles;
                    for (int q = 0; q < parts; ++q) {
                        sa.push_back((unsigned short)ta);
                        sb0.push_back((unsigned short)(ta + len * q / parts));
                        sb1.push_back((unsigned short)(ta + len * (q + 1) / parts));
                        s->seg_max = std::max(s->seg_max, (int)(sb1.back() - sb0.back()));
                    }
                }
                s->nseg = (int)sa.size();
                TRY(alloc_zero(s, sa.size(), &s->seg_a));
                TRY(alloc_zero(s, sa.size(), &s->seg_b0));
                TRY(alloc_zero(s, sa.size(), &s->seg_b1));
                TRY(upload(s, s->seg_a, sa.data(), sa.size() * sizeof(unsigned short)));
                TRY(upload(s, s->seg_b0, sb0.data(), sb0.size() * sizeof(unsigned short)));
                TRY(upload(s, s->seg_b1, sb1.data(), sb1.size() * sizeof(unsigned short)));
                herk_res_groups(s->nseg, s->seg_max, B, s->num_sms, (long long)s->P, B, s->herk_gcap, gb);
            } else {
                herk_groups(s->ntp128, B, s->num_sms, (long long)s->P, B, s->herk_gcap, gb);
            }
            TRY(alloc_zero(s, (size_t)s->herk_gcap * 3 * s->P, &s->herk_part));
        }
        if (max_groups > 1) TRY(alloc_zero(s, (size_t)max_groups * 7 * s->P, &s->partial));
        s->partial_groups = max_groups > 1 ? max_groups : 1;
    }  // spectral state
    TRY(alloc_zero(s, (size_t)FC_NMETRIC * s->P, &s->net));
    if (s->time_mask & FC_COR) {
        TRY(alloc_zero(s, (size_t)s->slots * n_nodes * n_samples, &s->zring));
        TRY(alloc_zero(s, (size_t)2 * s->P, &s->cor_acc));
        s->cor_nt = (n_nodes + 127) / 128;
        s->cor_ntp = s->cor_nt * (s->cor_nt + 1) / 2;
        s->cor_nchunks = (n_samples + 31) / 32;
        TRY(alloc_zero(s, (size_t)s->slots * s->cor_nt * s->cor_nchunks * cor_tc_pair_bytes(), &s->cor_ops));
    }
    if (s->time_mask & FC_XCOR) {
        int L = 1;
        while (L < 2 * n_samples - 1) L *= 2;
        if (L < 64) L = 64;
        s->xcor_L = L;
        if (L > 16384) return cleanup(fail(FC_ERR_UNSUPPORTED, "XCOR supports n_samples <= 8192"));
        const int M = L / 2;
        std::vector<float2> xt(M);
        for (int k = 0; k < M; ++k) {
            const double ang = 2.0 * kPi * k / L;
            xt[k] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
        }
        TRY(alloc_zero(s, (size_t)M, &s->xcor_tw));
        TRY(upload(s, s->xcor_tw, xt.data(), M * sizeof(float2)));
        TRY(alloc_zero(s, (size_t)s->slots * n_nodes * (M + 1), &s->xcor_spec));
        TRY(alloc_zero(s, (size_t)s->slots * n_nodes, &s->xcor_energy));
        TRY(alloc_zero(s, (size_t)s->slots * s->P, &s->xcor_vals));
        TRY(alloc_zero(s, (size_t)s->P, &s->xcor_lag));
        TRY(alloc_zero(s, (size_t)2 * s->P, &s->xcor_acc));
    }
    TRY(ensure_stage(s, 1));
#undef TRY
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cleanup(fail(FC_ERR_CUDA, "session init: %s", cudaGetErrorString(e)));
    *out = s;
    return FC_OK;
}

fc_status fc_session_destroy(fc_session* s) {
    if (!s) return FC_OK;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    if (s->in_stream) cudaStreamSynchronize(s->in_stream);
    if (s->out_stream) cudaStreamSynchronize(s->out_stream);
    if (s->side_stream) cudaStreamSynchronize(s->side_stream);  // a re-sum slice may still write the scratch
    drain_timings(s);
    free_all(s);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    if (s->side_stream) {
        cudaStreamDestroy(s->side_stream);
        cudaEventDestroy(s->ev_fork);
        cudaEventDestroy(s->ev_join);
    }
    if (s->dense_scratch) cudaFree(s->dense_scratch);
    if (s->post_scratch) cudaFree(s->post_scratch);
    if (s->proj) cudaFree(s->proj);
    if (s->proj_in) cudaFree(s->proj_in);
    if (s->sens_spec) cudaFree(s->sens_spec);
    if (s->cor_part) cudaFree(s->cor_part);
    for (int b = 0; b < 2; ++b) {
        if (s->x_in[b]) cudaFree(s->x_in[b]);
        if (s->snap[b]) cudaFree(s->snap[b]);
        for (cudaEvent_t e : {s->ev_in[b], s->ev_used[b], s->ev_snap[b], s->ev_out[b]})
            if (e) cudaEventDestroy(e);
    }
    if (s->in_stream) cudaStreamDestroy(s->in_stream);
    if (s->out_stream) cudaStreamDestroy(s->out_stream);
    delete s;
    return FC_OK;
}

fc_status fc_push_trials(fc_session* s, const float* x, int count, int x_on_device) {
    if (!s || !x) return fail(FC_ERR_INVALID_ARG, "NULL session or trial pointer");
    if (count < 1) return fail(FC_ERR_INVALID_ARG, "count must be >= 1");
    CK(cudaSetDevice(s->device));
    const float* xd = x;
    const size_t per = (size_t)s->n * s->N;
    if (s->proj) {
        // sensor trials [count][C][N] -> source trials [count][n][N] in the staging buffer
        const size_t per_in = (size_t)s->proj_C * s->N;
        if (count > 65535) return fail(FC_ERR_INVALID_ARG, "at most 65535 trials per call with a projection");
        const float* xin = x;
        if (!x_on_device) {
            if (s->proj_in_trials < count) {
                if (s->proj_in) cudaFree(s->proj_in);
                s->proj_in = nullptr;
                s->proj_in_trials = 0;
                CK(cudaMalloc(&s->proj_in, per_in * count * sizeof(float)));
                s->proj_in_trials = count;
            }
            CK(cudaMemcpyAsync(s->proj_in, x, per_in * count * sizeof(float), cudaMemcpyHostToDevice, s->stream));
            xin = s->proj_in;
        }
        if (!s->time_mask) {
            // spectral metrics only: the sensor trials go to the spectrum stage, which
            // projects their band spectra (M commutes with the taper and the DFT)
            s->spec_project = true;
            const int bulk_min = std::max(2, s->W / 4);
            fc_status st;
            if (s->cfg.mode == FC_MODE_FULL)
                st = push_bulk(s, xin, count, false);
            else if (s->W > 0 && count >= bulk_min)
                st = push_bulk(s, xin, count, true);
            else {
                st = FC_OK;
                for (int u = 0; u < count && st == FC_OK; ++u) st = push_one_stream(s, xin + per_in * u, u == count - 1);
            }
            s->spec_project = false;
            return st;
        }
        fc_status st = ensure_stage(s, count);
        if (st != FC_OK) return st;
        LAUNCH(FC_K_PROJECT, launch_project(s->proj, xin, s->x_stage, s->n, s->proj_C, s->N, count, s->stream));
        xd = s->x_stage;
    } else if (!x_on_device && count == 1) {
        // one host trial: copied on the input stream into the buffer the push before last
        // used, while the compute stream may still be busy with the previous push
        fc_status st = ensure_io(s);
        if (st != FC_OK) return st;
        const int b = s->in_flip;
        s->in_flip ^= 1;
        if (!s->x_in[b]) CK(cudaMalloc(&s->x_in[b], per * sizeof(float)));
        if (s->used_valid[b]) CK(cudaStreamWaitEvent(s->in_stream, s->ev_used[b], 0));
        CK(cudaMemcpyAsync(s->x_in[b], x, per * sizeof(float), cudaMemcpyHostToDevice, s->in_stream));
        CK(cudaEventRecord(s->ev_in[b], s->in_stream));
        CK(cudaStreamWaitEvent(s->stream, s->ev_in[b], 0));
        st = s->cfg.mode == FC_MODE_FULL ? push_bulk(s, s->x_in[b], 1, false) : push_one_stream(s, s->x_in[b], true);
        if (st != FC_OK) return st;
        CK(cudaEventRecord(s->ev_used[b], s->stream));
        s->used_valid[b] = true;
        return FC_OK;
    } else if (!x_on_device) {
        fc_status st = ensure_stage(s, count);
        if (st != FC_OK) return st;
        CK(cudaMemcpyAsync(s->x_stage, x, per * count * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        xd = s->x_stage;
    }
    if (s->cfg.mode == FC_MODE_FULL) return push_bulk(s, xd, count, false);
    const bool bulk = s->W > 0 && count >= std::max(2, s->W / 4);
    if (bulk) return push_bulk(s, xd, count, true);
    for (int u = 0; u < count; ++u) {
        fc_status st = push_one_stream(s, xd + per * u, u == count - 1);
        if (st != FC_OK) return st;
    }
    return FC_OK;
}

fc_status fc_push_trial(fc_session* s, const float* x, int x_on_device) {
    return fc_push_trials(s, x, 1, x_on_device);
}

fc_status fc_sync(fc_session* s) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    return check_latched(s, &h);
}

fc_status fc_get_network(fc_session* s, uint32_t metric, int packed_upper, float* out, size_t out_len,
                         int out_on_device, int* k_used) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL session or output");
    const int mi = metric_index(metric);
    if (mi < 0) return fail(FC_ERR_INVALID_ARG, "metric must be a single FC_* bit");
    if (!(s->mask & metric)) return fail(FC_ERR_INVALID_ARG, "metric 0x%x is not in the session mask", metric);
    const size_t need = packed_upper ? (size_t)s->P : (size_t)s->n * s->n;
    if (out_len < need) return fail(FC_ERR_INVALID_ARG, "out_len %zu < %zu", out_len, need);
    CK(cudaSetDevice(s->device));
    if (s->enqueued == 0) return fail(FC_ERR_NOT_READY, "no trial has been pushed");
    if (!out_on_device || k_used) {
        FcCtrl h;
        fc_status st = check_latched(s, &h);
        if (st != FC_OK) return st;
        if (h.pushed == 0) return fail(FC_ERR_NOT_READY, "no trial has been accepted");
        if (k_used) *k_used = (int)((s->W > 0 && h.pushed > s->W) ? s->W : h.pushed);
    }
    const float* src = s->net + (size_t)mi * s->P;
    if (packed_upper) {
        CK(cudaMemcpyAsync(out, src, need * sizeof(float),
                           out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    } else {
        float* dst = out;
        if (!out_on_device) {
            if (s->dense_scratch_len < need) {
                if (s->dense_scratch) cudaFree(s->dense_scratch);
                s->dense_scratch = nullptr;
                s->dense_scratch_len = 0;
                CK(cudaMalloc(&s->dense_scratch, need * sizeof(float)));
                s->dense_scratch_len = need;
            }
            dst = s->dense_scratch;
        }
        LAUNCH(FC_K_OTHER, launch_expand_dense(src, dst, s->n, mi == MI_IMAGCOHY, s->stream));
        if (!out_on_device) CK(cudaMemcpyAsync(out, dst, need * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    }
    if (!out_on_device) CK(cudaStreamSynchronize(s->stream));
    return FC_OK;
}

fc_status fc_get_network_async(fc_session* s, uint32_t metric, float* out, size_t out_len) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL session or output");
    const int mi = metric_index(metric);
    if (mi < 0) return fail(FC_ERR_INVALID_ARG, "metric must be a single FC_* bit");
    if (!(s->mask & metric)) return fail(FC_ERR_INVALID_ARG, "metric 0x%x is not in the session mask", metric);
    if (out_len < (size_t)s->P) return fail(FC_ERR_INVALID_ARG, "out_len %zu < %lld", out_len, (long long)s->P);
    CK(cudaSetDevice(s->device));
    if (s->enqueued == 0) return fail(FC_ERR_NOT_READY, "no trial has been pushed");
    fc_status st = ensure_io(s);
    if (st != FC_OK) return st;
    if (s->out_count == 2) {
        st = fc_network_wait(s);
        if (st != FC_OK) return st;
    }
    const int b = s->out_head;
    const size_t bytes = (size_t)s->P * sizeof(float);
    if (!s->snap[b]) CK(cudaMalloc(&s->snap[b], bytes));
    CK(cudaMemcpyAsync(s->snap[b], s->net + (size_t)mi * s->P, bytes, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaEventRecord(s->ev_snap[b], s->stream));
    CK(cudaStreamWaitEvent(s->out_stream, s->ev_snap[b], 0));
    CK(cudaMemcpyAsync(out, s->snap[b], bytes, cudaMemcpyDeviceToHost, s->out_stream));
    CK(cudaEventRecord(s->ev_out[b], s->out_stream));
    s->out_head ^= 1;
    s->out_count += 1;
    return FC_OK;
}

fc_status fc_network_wait(fc_session* s) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    if (s->out_count == 0) return FC_OK;
    CK(cudaSetDevice(s->device));
    const int oldest = (s->out_head + 2 - s->out_count) & 1;
    CK(cudaEventSynchronize(s->ev_out[oldest]));
    s->out_count -= 1;
    return FC_OK;
}

fc_status fc_get_network_top(fc_session* s, uint32_t metric, double percent, float* weights, int* degree,
                             float* strength, int out_on_device, fc_top_info* info) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    const int mi = metric_index(metric);
    if (mi < 0) return fail(FC_ERR_INVALID_ARG, "metric must be a single FC_* bit");
    if (!(s->mask & metric)) return fail(FC_ERR_INVALID_ARG, "metric 0x%x is not in the session mask", metric);
    if (!(percent >= 0.0 && percent <= 100.0)) return fail(FC_ERR_INVALID_ARG, "percent must be in [0, 100]");
    if ((degree == nullptr) != (strength == nullptr))
        return fail(FC_ERR_INVALID_ARG, "degree and strength are given together or not at all");
    CK(cudaSetDevice(s->device));
    if (s->enqueued == 0) return fail(FC_ERR_NOT_READY, "no trial has been pushed");
    FcCtrl h;
    fc_status st = check_latched(s, &h);
    if (st != FC_OK) return st;
    if (h.pushed == 0) return fail(FC_ERR_NOT_READY, "no trial has been accepted");
    const long long P = s->P;
    const long long k = std::min(P, std::max(0LL, (long long)std::ceil(percent * (double)P / 100.0)));
    // scratch: select state + ties + flags, then device outputs when the caller's are on the host
    const size_t base = (post_scratch_bytes(P) + 255) / 256 * 256;
    const size_t need = base + (size_t)P * sizeof(float) + (size_t)s->n * (sizeof(int) + sizeof(float)) + 256;
    if (s->post_scratch_len < need) {
        if (s->post_scratch) cudaFree(s->post_scratch);
        s->post_scratch = nullptr;
        s->post_scratch_len = 0;
        CK(cudaMalloc(&s->post_scratch, need));
        s->post_scratch_len = need;
    }
    char* sc = static_cast<char*>(s->post_scratch);
    float* d_w = (weights && out_on_device) ? weights : reinterpret_cast<float*>(sc + base);
    int* d_deg = nullptr;
    float* d_str = nullptr;
    if (degree) {
        d_deg = out_on_device ? degree : reinterpret_cast<int*>(sc + base + (size_t)P * sizeof(float));
        d_str = out_on_device ? strength : reinterpret_cast<float*>(sc + base + (size_t)P * sizeof(float) +
                                                                     (size_t)s->n * sizeof(int));
    }
    CK(launch_network_top(s->net + (size_t)mi * P, P, s->n, k, sc, d_w, d_deg, d_str, s->num_sms, s->stream));
    if (!out_on_device) {
        if (weights) CK(cudaMemcpy(weights, d_w, (size_t)P * sizeof(float), cudaMemcpyDeviceToHost));
        if (degree) {
            CK(cudaMemcpy(degree, d_deg, (size_t)s->n * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(strength, d_str, (size_t)s->n * sizeof(float), cudaMemcpyDeviceToHost));
        }
    }
    if (info) {
        PostState ps;
        CK(cudaMemcpy(&ps, s->post_scratch, sizeof(PostState), cudaMemcpyDeviceToHost));
        std::memcpy(&info->max_abs, &ps.max_key, sizeof(float));
        info->threshold = 0.f;
        if (k > 0) std::memcpy(&info->threshold, &ps.prefix, sizeof(float));
        info->kept = k;
    }
    return FC_OK;
}

fc_status fc_get_network_bins(fc_session* s, uint32_t metric, float* out, size_t out_len, int out_on_device) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL session or output");
    const int mi = metric_index(metric);
    if (mi < MI_COH) return fail(FC_ERR_INVALID_ARG, "per-bin values exist for spectral metrics only");
    if (s->ops) return fail(FC_ERR_UNSUPPORTED, "per-bin values are available with FC_PREC_FP32 sessions");
    const size_t need = (size_t)s->B * s->P;
    if (out_len < need) return fail(FC_ERR_INVALID_ARG, "out_len %zu < %zu", out_len, need);
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    fc_status st = check_latched(s, &h);
    if (st != FC_OK) return st;
    if (h.pushed == 0) return fail(FC_ERR_NOT_READY, "no trial has been accepted");
    float* dst = out;
    float* tmp = nullptr;
    if (!out_on_device) {
        CK(cudaMalloc(&tmp, need * sizeof(float)));
        dst = tmp;
    }
    if (s->cfg.mode == FC_MODE_STREAM) {
        PairArgs pa = pair_args(s, true, 0);
        LAUNCH(FC_K_OTHER, launch_bins_from_acc(pa, mi, dst, s->stream));
    } else {
        PairArgs pa = pair_args(s, false, 0);
        LAUNCH(FC_K_OTHER, launch_bins_window(pa, mi, dst, s->stream));
    }
    if (!out_on_device) {
        cudaError_t e = cudaMemcpyAsync(out, dst, need * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return fail(FC_ERR_CUDA, "per-bin copy: %s", cudaGetErrorString(e));
    }
    return FC_OK;
}

fc_status fc_get_xcor_lags(fc_session* s, int32_t* out, size_t out_len, int out_on_device) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL session or output");
    if (!(s->time_mask & FC_XCOR)) return fail(FC_ERR_INVALID_ARG, "XCOR is not in the session");
    if (out_len < (size_t)s->P) return fail(FC_ERR_INVALID_ARG, "out_len too small");
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    fc_status st = check_latched(s, &h);
    if (st != FC_OK) return st;
    if (h.pushed == 0) return fail(FC_ERR_NOT_READY, "no trial has been accepted");
    CK(cudaMemcpyAsync(out, s->xcor_lag, s->P * sizeof(int32_t),
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return FC_OK;
}

fc_status fc_set_metric_mask(fc_session* s, uint32_t metric_mask) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    if (metric_mask == 0 || (metric_mask & ~(uint32_t)FC_ALL_METRICS))
        return fail(FC_ERR_INVALID_ARG, "bad metric mask 0x%x", metric_mask);
    if ((metric_mask & (FC_COR | FC_XCOR)) & ~s->time_mask)
        return fail(FC_ERR_INVALID_ARG, "COR/XCOR can only be kept, not added after creation");
    if ((metric_mask & FC_SPECTRAL_METRICS) && !s->spectral)
        return fail(FC_ERR_INVALID_ARG, "the session was created without spectral metrics: none can be added");
    CK(cudaSetDevice(s->device));
    const uint32_t added = metric_mask & ~s->mask & FC_SPECTRAL_METRICS;
    s->mask = metric_mask;
    if (added && s->enqueued > 0) {
        // recompute the spectral networks from the shared sums (no trial is reprocessed)
        if (s->cfg.mode == FC_MODE_STREAM) {
            PairArgs pa = pair_args(s, true, 0);
            pa.finalize = 1;
            pa.update = 0;
            LAUNCH(FC_K_STREAM, launch_stream_update(pa, s->stream));
            if (pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
        } else {
            fc_status st = stage_window(s, 0, false);
            if (st != FC_OK) return st;
        }
    }
    return FC_OK;
}

fc_status fc_debug_wait_probe(fc_session* s, double limit_ms) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return fail(FC_ERR_INVALID_ARG, "limit_ms must be in (0, 1000]");
    CK(cudaSetDevice(s->device));
    LAUNCH(FC_K_OTHER, launch_wait_probe(s->ctrl, (unsigned long long)(limit_ms * 1e6), s->stream));
    FcCtrl h;
    return check_latched(s, &h);
}

fc_status fc_set_projection(fc_session* s, const float* op, int n_channels, int op_on_device) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    CK(cudaSetDevice(s->device));
    CK(cudaStreamSynchronize(s->stream));  // pushes in flight used the previous operator
    if (!op) {
        if (s->proj) cudaFree(s->proj);
        s->proj = nullptr;
        s->proj_C = 0;
        return FC_OK;
    }
    if (n_channels < 1) return fail(FC_ERR_INVALID_ARG, "n_channels must be >= 1");
    const size_t bytes = (size_t)s->n * n_channels * sizeof(float);
    if (s->proj && s->proj_C != n_channels) {
        cudaFree(s->proj);
        s->proj = nullptr;
    }
    // ordered after the pushes already enqueued (they may still read the previous operator)
    CK(cudaStreamSynchronize(s->stream));
    if (!s->proj) CK(cudaMalloc(&s->proj, bytes));
    s->proj_C = n_channels;
    CK(cudaMemcpyAsync(s->proj, op, bytes, op_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return FC_OK;
}

fc_status fc_set_band(fc_session* s, double f_lo, double f_hi) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    if (!s->spectral) return fail(FC_ERR_INVALID_ARG, "the session was created without spectral metrics");
    fc_band b = s->band;
    b.f_lo = f_lo;
    b.f_hi = f_hi;
    int first = -1;
    const int cnt = fc_band_bins(s->fs, b, &first);
    if (cnt <= 0) return fail(FC_ERR_INVALID_ARG, "the band [%g, %g) Hz selects no bin", f_lo, f_hi);
    if (first < s->first_bin || first + cnt > s->first_bin + s->B)
        return fail(FC_ERR_INVALID_ARG,
                    "the band [%g, %g) Hz reaches outside the computed bins %d..%d: create the session with "
                    "the wider band", f_lo, f_hi, s->first_bin, s->first_bin + s->B - 1);
    CK(cudaSetDevice(s->device));
    s->sel0 = first - s->first_bin;
    s->sel1 = s->sel0 + cnt;
    if (s->enqueued > 0 && (s->mask & FC_SPECTRAL_METRICS)) {
        // new band averages from the per-bin sums: no trial is reprocessed
        if (s->cfg.mode == FC_MODE_STREAM) {
            PairArgs pa = pair_args(s, true, 0);
            pa.finalize = 1;
            pa.update = 0;
            LAUNCH(FC_K_STREAM, launch_stream_update(pa, s->stream));
            if (pa.groups > 1) LAUNCH(FC_K_BAND_REDUCE, launch_band_reduce(pa, s->stream));
        } else {
            fc_status st = stage_window(s, 0, false);
            if (st != FC_OK) return st;
        }
    }
    return FC_OK;
}

// ------------------------------------------------------------ snapshot / restore
namespace {
struct SnapHeader {
    char magic[8];
    int n, N, B, first_bin, nfft, W, slots, mode, precision, taper;
    double fs, f_lo, f_hi;
    uint32_t mask, time_mask;
    int sel0, sel1, nbufs, calibrated;
    long long enqueued, resum_phase;
};
const char kSnapMagic[8] = {'F', 'C', 'S', 'N', 'A', 'P', '1', 0};

size_t snapshot_bytes(const fc_session* s) {
    size_t b = sizeof(SnapHeader) + s->state_bufs.size() * sizeof(unsigned long long);
    for (const auto& sb : s->state_bufs) b += sb.second;
    return b;
}
}  // namespace

fc_status fc_session_snapshot_size(fc_session* s, size_t* bytes) {
    if (!s || !bytes) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    *bytes = snapshot_bytes(s);
    return FC_OK;
}

fc_status fc_session_snapshot(fc_session* s, void* host_buf, size_t len) {
    if (!s || !host_buf) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    if (len < snapshot_bytes(s)) return fail(FC_ERR_INVALID_ARG, "buffer of %zu bytes < %zu", len, snapshot_bytes(s));
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    fc_status st = read_ctrl(s, &h);  // synchronizes: every enqueued push is in the state
    if (st != FC_OK) return st;
    SnapHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kSnapMagic, sizeof hd.magic);
    hd.n = s->n; hd.N = s->N; hd.B = s->B; hd.first_bin = s->first_bin; hd.nfft = s->nfft; hd.W = s->W;
    hd.slots = s->slots; hd.mode = (int)s->cfg.mode; hd.precision = (int)s->cfg.precision; hd.taper = (int)s->taper;
    hd.fs = s->fs; hd.f_lo = s->band.f_lo; hd.f_hi = s->band.f_hi;
    hd.mask = s->mask; hd.time_mask = s->time_mask; hd.sel0 = s->sel0; hd.sel1 = s->sel1;
    hd.nbufs = (int)s->state_bufs.size(); hd.calibrated = s->calibrated ? 1 : 0;
    hd.enqueued = s->enqueued; hd.resum_phase = s->resum_phase;
    char* out = static_cast<char*>(host_buf);
    std::memcpy(out, &hd, sizeof hd);
    size_t off = sizeof hd;
    for (const auto& sb : s->state_bufs) {
        const unsigned long long b = sb.second;
        std::memcpy(out + off, &b, sizeof b);
        off += sizeof b;
    }
    for (const auto& sb : s->state_bufs) {
        CK(cudaMemcpy(out + off, sb.first, sb.second, cudaMemcpyDeviceToHost));
        off += sb.second;
    }
    return FC_OK;
}

fc_status fc_session_restore(fc_session* s, const void* host_buf, size_t len) {
    if (!s || !host_buf) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    if (len < sizeof(SnapHeader)) return fail(FC_ERR_INVALID_ARG, "not a session snapshot (too short)");
    SnapHeader hd;
    std::memcpy(&hd, host_buf, sizeof hd);
    if (std::memcmp(hd.magic, kSnapMagic, sizeof hd.magic) != 0)
        return fail(FC_ERR_INVALID_ARG, "not a session snapshot (bad magic)");
    const bool same = hd.n == s->n && hd.N == s->N && hd.B == s->B && hd.first_bin == s->first_bin &&
                      hd.nfft == s->nfft && hd.W == s->W && hd.slots == s->slots && hd.mode == (int)s->cfg.mode &&
                      hd.precision == (int)s->cfg.precision && hd.taper == (int)s->taper && hd.fs == s->fs &&
                      hd.f_lo == s->band.f_lo && hd.f_hi == s->band.f_hi && hd.time_mask == s->time_mask &&
                      hd.nbufs == (int)s->state_bufs.size();
    if (!same) return fail(FC_ERR_INVALID_ARG, "the snapshot was taken from a session with other settings");
    if (len < snapshot_bytes(s)) return fail(FC_ERR_INVALID_ARG, "snapshot truncated");
    const char* in = static_cast<const char*>(host_buf);
    size_t off = sizeof hd;
    for (const auto& sb : s->state_bufs) {
        unsigned long long b;
        std::memcpy(&b, in + off, sizeof b);
        off += sizeof b;
        if (b != sb.second) return fail(FC_ERR_INVALID_ARG, "the snapshot's buffer sizes differ from this session's");
    }
    CK(cudaSetDevice(s->device));
    CK(cudaStreamSynchronize(s->stream));
    for (const auto& sb : s->state_bufs) {  // on the session stream: later pushes are ordered after
        CK(cudaMemcpyAsync(sb.first, in + off, sb.second, cudaMemcpyHostToDevice, s->stream));
        off += sb.second;
    }
    CK(cudaStreamSynchronize(s->stream));  // the caller may release host_buf on return
    s->mask = hd.mask;
    s->sel0 = hd.sel0;
    s->sel1 = hd.sel1;
    s->calibrated = hd.calibrated != 0;
    s->enqueued = hd.enqueued;
    s->resum_phase = hd.resum_phase;
    return FC_OK;
}

fc_status fc_session_info(fc_session* s, fc_info* info) {
    if (!s || !info) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    fc_status st = read_ctrl(s, &h);
    if (st != FC_OK) return st;
    memset(info, 0, sizeof *info);
    info->n_nodes = s->n;
    info->n_samples = s->N;
    info->n_bins = s->B;
    info->first_bin = s->first_bin;
    info->nfft = s->nfft;
    info->window = s->W;
    info->k_used = (int)((s->W > 0 && h.pushed > s->W) ? s->W : h.pushed);
    info->pushes = h.pushed;
    info->rejected = h.rejected;
    info->pairs = s->P;
    info->device_bytes = s->device_bytes;
    info->metric_mask = s->mask;
    info->mode = s->cfg.mode;
    info->precision = s->cfg.precision;
    info->spectrum = s->use_fft ? FC_SPECTRUM_FFT : FC_SPECTRUM_DFT;
    if (h.bad_latched) return check_latched(s, &h);
    return FC_OK;
}

fc_status fc_set_profiling(fc_session* s, int enable) {
    if (!s) return fail(FC_ERR_INVALID_ARG, "NULL session");
    s->profiling = enable != 0;
    return FC_OK;
}

fc_status fc_kernel_times(fc_session* s, fc_kernel_time* out, int reset) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(s->device));
    CK(cudaStreamSynchronize(s->stream));
    drain_timings(s);
    for (int k = 0; k < FC_K_COUNT; ++k) out[k] = s->ktime[k];
    if (reset)
        for (int k = 0; k < FC_K_COUNT; ++k) s->ktime[k] = fc_kernel_time{0, 0.0};
    return FC_OK;
}

long long fc_launch_count(const fc_session* s) { return s ? s->launches : 0; }

void* fc_session_stream(const fc_session* s) { return s ? (void*)s->stream : nullptr; }

fc_status fc_debug_get_spectra(fc_session* s, int age, float* out, size_t out_len) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    if (!s->spectral) return fail(FC_ERR_INVALID_ARG, "the session was created without spectral metrics");
    const size_t need = (size_t)2 * s->B * s->n;
    if (out_len < need) return fail(FC_ERR_INVALID_ARG, "out_len too small");
    CK(cudaSetDevice(s->device));
    FcCtrl h;
    fc_status st = read_ctrl(s, &h);
    if (st != FC_OK) return st;
    const long long kept = s->W > 0 ? std::min<long long>(h.pushed, s->W) : std::min<long long>(h.pushed, 1);
    if (age < 0 || age >= kept) return fail(FC_ERR_INVALID_ARG, "no stored trial of age %d", age);
    const long long g = h.pushed - 1 - age;
    CK(cudaMemcpy(out, s->ring + (size_t)(g % s->slots) * s->B * s->n, need * sizeof(float), cudaMemcpyDeviceToHost));
    return FC_OK;
}

fc_status fc_debug_get_scale(fc_session* s, float* scale) {
    if (!s || !scale) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    FcCtrl h;
    fc_status st = read_ctrl(s, &h);
    if (st != FC_OK) return st;
    *scale = h.scale == 0.f ? 1.f : h.scale;
    return FC_OK;
}

fc_status fc_debug_get_accumulators(fc_session* s, fc_acc_field field, double* out, size_t out_len) {
    if (!s || !out) return fail(FC_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(s->device));
    CK(cudaStreamSynchronize(s->stream));
    if (field != FC_ACC_COR && field != FC_ACC_XCOR && !s->spectral)
        return fail(FC_ERR_INVALID_ARG, "the session was created without spectral metrics");
    size_t need;
    if (field == FC_ACC_PSD) need = (size_t)s->B * s->n;
    else if (field == FC_ACC_COR || field == FC_ACC_XCOR) need = (size_t)s->P;
    else if (field >= FC_ACC_CSD_RE && field <= FC_ACC_SIGN) need = (size_t)s->B * s->P;
    else return fail(FC_ERR_INVALID_ARG, "bad field");
    if (out_len < need) return fail(FC_ERR_INVALID_ARG, "out_len too small");
    if (field == FC_ACC_PSD) {
        CK(cudaMemcpy(out, s->psd, need * sizeof(double), cudaMemcpyDeviceToHost));
        return FC_OK;
    }
    const float* planes = nullptr;
    if (field == FC_ACC_COR) planes = s->cor_acc;
    if (field == FC_ACC_XCOR) planes = s->xcor_acc;
    if ((field == FC_ACC_COR || field == FC_ACC_XCOR) && !planes)
        return fail(FC_ERR_INVALID_ARG, "metric not in the session");
    if (field <= FC_ACC_SIGN && !s->acc) return fail(FC_ERR_INVALID_ARG, "no accumulators in full mode");
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, need * sizeof(double)));
    cudaError_t e;
    if (planes)
        e = launch_df_planes_to_double(planes, s->P, tmp, s->stream);
    else
        e = launch_acc_field(s->acc, s->tile_a, s->tile_b, s->ntp, s->B, s->n, (int)field, tmp, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, need * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(FC_ERR_CUDA, "accumulator read: %s", cudaGetErrorString(e));
    return FC_OK;
}

}  // extern "C"
