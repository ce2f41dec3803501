// fc_server.cu - serving many concurrent sessions with continuous batching.
//
// The paper's online pipeline adds every newly arriving trial to the network as it comes
// (Methods 2.5; Results 3.2.3) and must keep up with the acquisition (Results 3.2.3: a
// 500-sample block at 1,792 Hz leaves 280 ms). Here many sessions share one GPU: each
// arriving trial of any session is a request. A worker thread runs ticks; every tick is
// ONE launch of the persistent streaming kernel over a share of the state of up to 32
// sessions, with each session's small kernels (validation, spectrum, per-node sums before
// its first share of a trial; re-sum slice and commit after its last) around it on the
// same stream.
//
// A launch carries at most `launch_blocks` state blocks (one tile pair x one bin, 106 KB
// of HBM traffic each). A trial whose push is larger is split over several launches (its
// units are walked in order; the window position only advances at the commit after the
// last share), so a 5,000-node session's ~10 ms push does not hold back the trials of
// small sessions that arrive meanwhile: the oldest unfinished push gets at least a quarter
// of the budget, then pushes that fit the remaining budget go in whole, shortest first, and
// what is left goes to the remaining pushes, oldest first. Trials that arrive while a
// launch runs join the next tick; two launches may be in flight, so the host staging of
// one overlaps the device work of the other. Session state stays resident; sessions are
// admitted against a device-memory budget.
//
// In plain mode (the comparison baseline) every trial is handled alone, in arrival order,
// as a full-window FP32 recompute (FC_MODE_FULL), with no batching and no streaming sums.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fc_internal.h"

namespace {

constexpr long long kDefaultLaunchBlocks = 65536;  // ~7 GB of state traffic, ~1.2 ms on GB300

double now_ms() {
    using namespace std::chrono;
    static const steady_clock::time_point t0 = steady_clock::now();
    return duration<double, std::milli>(steady_clock::now() - t0).count();
}

struct PendingTrial {
    std::vector<float> x;
    double arrival = 0.0;
    long long seq = 0;
};

struct SrvSession {
    int id = 0;
    fc_session* s = nullptr;
    size_t bytes = 0;
    long long pair_bins = 0;
    size_t trial_floats = 0;
    long long units = 0;  // streaming-kernel units of one push (tile pairs, all bins each)
    std::deque<PendingTrial> queue;
    long long submitted = 0, completed = 0;
    long long in_flight = 0;  // trials taken from the queue and not yet retired
    // the push in progress, whose units may span several launches (worker only)
    bool active = false;
    PendingTrial cur;
    long long next_unit = 0;  // first unit not yet planned
    // units of the push in progress already enqueued; nonzero: the device state holds a
    // partly applied push (guarded by dev_mu)
    long long partial = 0;
    float* pinned[2] = {nullptr, nullptr};  // trial staging, by tick parity
    FcCtrl* pinned_ctrl = nullptr;          // [2] control-block read-back, by tick parity
    FcCtrl* pinned_ctrl_dev = nullptr;      // the same memory as the device addresses it
    long long rejected_seen = 0;
    bool closing = false;
};

struct Part {  // one session's share of a tick
    SrvSession* ss;
    long long u0, nu;
    bool start, finish, single;
};

struct Done {  // a trial whose last share is in this tick
    SrvSession* ss;
    long long seq;
    double arrival;
    int launch_sessions;
};

struct InFlight {
    cudaEvent_t ev = nullptr;
    int slot = 0;
    std::vector<Done> done;
};

}  // namespace

struct fc_server {
    fc_server_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 152;
    // lock order: dev_mu before mu
    std::mutex mu;      // sessions, queues, plans, results, stats
    std::mutex dev_mu;  // device work on sessions (worker enqueue / retire vs API calls)
    std::condition_variable cv_work, cv_done;
    std::map<int, SrvSession*> sessions;
    int next_id = 1;
    std::deque<fc_result> results;
    std::deque<InFlight> inflight;  // owned by the worker
    std::vector<cudaEvent_t> event_pool;
    std::thread worker;
    bool stop = false;
    int parity = 0;
    size_t used = 0;
    fc_server_stats stats{};
    std::string worker_error;
};

namespace {

fc_status sfail(fc_status st, const char* msg) {
    fc_internal_set_error(msg);
    return st;
}

// Choose this tick's shares (worker, mu held). Starts the next queued trial of every idle
// session, then fills the launch's block budget.
std::vector<Part> plan_tick(fc_server* sv) {
    std::vector<Part> plan;
    std::vector<SrvSession*> cand;
    for (auto& kv : sv->sessions) {
        SrvSession* ss = kv.second;
        if (!ss->active && !ss->queue.empty()) {
            ss->cur = std::move(ss->queue.front());
            ss->queue.pop_front();
            ss->active = true;
            ss->next_unit = 0;
            ss->in_flight++;
        }
        if (ss->active && ss->next_unit < ss->units) cand.push_back(ss);
    }
    if (cand.empty()) return plan;
    auto oldest_first = [](SrvSession* a, SrvSession* b) { return a->cur.arrival < b->cur.arrival; };
    std::sort(cand.begin(), cand.end(), oldest_first);
    if (sv->cfg.plain) {  // one trial, in arrival order, as a full-window recompute
        SrvSession* ss = cand.front();
        plan.push_back(Part{ss, 0, ss->units, true, true, true});
        ss->next_unit = ss->units;
        return plan;
    }
    const int max_batch = sv->cfg.max_batch > 0 ? std::min(sv->cfg.max_batch, FC_MAX_BATCH) : FC_MAX_BATCH;
    const long long budget = sv->cfg.launch_blocks < 0
                                 ? (1LL << 60)
                                 : (sv->cfg.launch_blocks > 0 ? sv->cfg.launch_blocks : kDefaultLaunchBlocks);
    long long left = budget;
    auto rem_units = [](const SrvSession* ss) { return ss->units - ss->next_unit; };
    auto take = [&](SrvSession* ss, long long nu) {
        const bool single = ss->next_unit == 0 && fc_push_needs_single(ss->s);
        if (single) nu = ss->units;  // first pushes (calibration) and the like run whole
        plan.push_back(Part{ss, ss->next_unit, nu, ss->next_unit == 0, ss->next_unit + nu == ss->units, single});
        ss->next_unit += nu;
        left -= nu * ss->s->B;
    };
    // 1. the oldest unfinished push: at least a quarter of the budget (no starvation)
    SrvSession* oldest = cand.front();
    take(oldest, std::min(rem_units(oldest), std::max(1LL, (budget / 4) / oldest->s->B)));
    // 2. whole pushes that fit, shortest first
    std::vector<SrvSession*> by_size(cand.begin() + 1, cand.end());
    std::stable_sort(by_size.begin(), by_size.end(), [&](const SrvSession* a, const SrvSession* b) {
        return rem_units(a) * a->s->B < rem_units(b) * b->s->B;
    });
    for (SrvSession* ss : by_size) {
        if ((int)plan.size() >= max_batch) break;
        if (rem_units(ss) * ss->s->B <= left) take(ss, rem_units(ss));
    }
    // 3. the rest of the budget, oldest first (extending a share already planned)
    for (SrvSession* ss : cand) {
        const long long can = std::min(rem_units(ss), left / ss->s->B);
        if (can <= 0) continue;
        Part* mine = nullptr;
        for (Part& p : plan)
            if (p.ss == ss) mine = &p;
        if (mine) {
            if (mine->single) continue;
            mine->nu += can;
            ss->next_unit += can;
            mine->finish = ss->next_unit == ss->units;
            left -= can * ss->s->B;
        } else if ((int)plan.size() < max_batch && !(ss->next_unit == 0 && fc_push_needs_single(ss->s))) {
            take(ss, can);
        }
    }
    // whole waves: the persistent update grid takes units round-robin, so a share whose units
    // are not a multiple of its CTAs leaves the launch as long as the CTAs with one unit more.
    // The largest share that does not finish in this launch is trimmed to a multiple (its rest
    // goes next tick); any contiguous run of such a length gives every CTA as many of its units.
    const long long grid = 2LL * sv->num_sms;
    Part* big = nullptr;
    for (Part& p : plan)
        if (!p.single && !p.finish && (!big || p.nu > big->nu)) big = &p;
    if (big && big->nu > grid) {
        const long long extra = big->nu % grid;
        big->nu -= extra;
        big->ss->next_unit -= extra;
    }
    return plan;
}

// Enqueue one tick on the server stream (worker, dev_mu held).
fc_status enqueue_tick(fc_server* sv, const std::vector<Part>& plan, InFlight& fl) {
    const int slot = sv->parity;
    sv->parity ^= 1;
    fl.slot = slot;
    for (const Part& p : plan) {
        if (!p.start) continue;
        SrvSession* ss = p.ss;
        std::memcpy(ss->pinned[slot], ss->cur.x.data(), ss->trial_floats * sizeof(float));
        cudaError_t e = cudaMemcpyAsync(ss->s->x_stage, ss->pinned[slot], ss->trial_floats * sizeof(float),
                                        cudaMemcpyHostToDevice, sv->stream);
        if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
    }
    // singles (calibrating first pushes and the like) run whole, each on its own
    for (const Part& p : plan) {
        if (!p.single) continue;
        fc_status st = fc_push_single(p.ss->s, p.ss->s->x_stage);
        if (st != FC_OK) return st;
    }
    // validation, spectra and per-node sums of every push that starts: one launch each
    fc_session* pre_s[FC_MAX_BATCH];
    const float* pre_x[FC_MAX_BATCH];
    int npre = 0;
    for (const Part& p : plan) {
        if (p.single || !p.start) continue;
        pre_s[npre] = p.ss->s;
        pre_x[npre] = p.ss->s->x_stage;
        ++npre;
    }
    fc_status pst = fc_push_batch_pre(pre_s, pre_x, npre, sv->stream);
    if (pst != FC_OK) return pst;
    StreamBatch b;
    b.nsess = 0;
    b.unit_prefix[0] = 0;
    for (const Part& p : plan) {
        fc_session* s = p.ss->s;
        if (p.single) continue;
        PairArgs pa = fc_push_stream_args(s);
        pa.u0 = (int)p.u0;
        b.a[b.nsess] = pa;
        b.unit_prefix[b.nsess + 1] = b.unit_prefix[b.nsess] + (int)p.nu;
        ++b.nsess;
    }
    if (b.nsess > 0) {
        cudaError_t e = launch_stream_batch(b, 2 * sv->num_sms, sv->stream);
        if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
    }
    // the drift re-sum slices of the pushes that started in this tick, beside the update
    pst = fc_push_batch_fork(pre_s, npre);
    if (pst != FC_OK) return pst;
    // drift re-sum slices, then one commit of every push that finishes; the commit also
    // writes each control block (prescale, rejection count) to the session's pinned slot
    fc_session* post_s[FC_MAX_BATCH];
    FcCtrl* post_snap[FC_MAX_BATCH];
    int npost = 0;
    for (const Part& p : plan) {
        SrvSession* ss = p.ss;
        if (p.single) {
            cudaError_t e = cudaMemcpyAsync(&ss->pinned_ctrl[slot], ss->s->ctrl, sizeof(FcCtrl),
                                            cudaMemcpyDeviceToHost, sv->stream);
            if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
            continue;
        }
        fc_count_launch(ss->s);
        ss->partial = p.finish ? 0 : p.u0 + p.nu;
        if (p.finish) {
            post_s[npost] = ss->s;
            post_snap[npost] = ss->pinned_ctrl_dev + slot;
            ++npost;
        }
    }
    pst = fc_push_batch_post(post_s, post_snap, npost, sv->stream);
    if (pst != FC_OK) return pst;
    if (!sv->event_pool.empty()) {
        fl.ev = sv->event_pool.back();
        sv->event_pool.pop_back();
    } else if (cudaEventCreateWithFlags(&fl.ev, cudaEventDisableTiming) != cudaSuccess) {
        fl.ev = nullptr;
        return sfail(FC_ERR_CUDA, "event creation failed");
    }
    cudaEventRecord(fl.ev, sv->stream);
    return FC_OK;
}

void retire(fc_server* sv, InFlight& fl) {
    cudaEventSynchronize(fl.ev);
    const double done = now_ms();
    std::lock_guard<std::mutex> dk(sv->dev_mu);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->event_pool.push_back(fl.ev);
    for (const Done& d : fl.done) {
        SrvSession* ss = d.ss;
        const FcCtrl& c = ss->pinned_ctrl[fl.slot];
        // a session whose prescale is known joins the batched launches from its next trial
        if (!ss->s->calibrated && c.scale != 0.f) ss->s->calibrated = true;
        fc_result r;
        r.session = ss->id;
        r.seq = d.seq;
        r.status = FC_OK;
        if (c.rejected > ss->rejected_seen) r.status = FC_ERR_NONFINITE;
        if (c.timeout) r.status = FC_ERR_TIMEOUT;
        ss->rejected_seen = c.rejected;
        r.arrival_ms = d.arrival;
        r.done_ms = done;
        r.batch = d.launch_sessions;
        sv->results.push_back(r);
        ss->completed++;
        ss->in_flight--;
        sv->stats.completed++;
        if (r.status == FC_OK) sv->stats.pair_bin_updates += ss->pair_bins;
    }
    sv->cv_done.notify_all();
}

void worker_main(fc_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<Part> plan;
        InFlight fl;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            auto has_work = [&]() {
                for (auto& kv : sv->sessions) {
                    const SrvSession* ss = kv.second;
                    if (!ss->queue.empty() || (ss->active && ss->next_unit < ss->units)) return true;
                }
                return false;
            };
            if (sv->inflight.empty())
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&]() { return sv->stop || has_work(); });
            if (sv->stop && !has_work() && sv->inflight.empty()) break;
            plan = plan_tick(sv);
            int batched = 0;
            for (const Part& p : plan) batched += p.single ? 0 : 1;
            for (const Part& p : plan) {
                if (!p.finish) continue;
                fl.done.push_back(Done{p.ss, p.ss->cur.seq, p.ss->cur.arrival, p.single ? 1 : batched});
                p.ss->active = false;  // its next trial may start next tick (ordered on the stream)
            }
        }
        if (!plan.empty()) {
            fc_status st;
            {
                std::lock_guard<std::mutex> dk(sv->dev_mu);
                st = enqueue_tick(sv, plan, fl);
            }
            if (st != FC_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->worker_error = fc_last_error();
                for (const Done& d : fl.done) d.ss->in_flight--;
                if (fl.ev) sv->event_pool.push_back(fl.ev);
                sv->cv_done.notify_all();
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->stats.launches++;
                sv->stats.batched_trials += (long long)plan.size();
            }
            sv->inflight.push_back(std::move(fl));
        }
        // keep at most two launches in flight; retire the oldest when idle or full
        while (!sv->inflight.empty() && (sv->inflight.size() >= 2 || plan.empty())) {
            retire(sv, sv->inflight.front());
            sv->inflight.pop_front();
            if (!plan.empty()) break;
        }
    }
}

SrvSession* find_session(fc_server* sv, int id) {
    auto it = sv->sessions.find(id);
    return it == sv->sessions.end() ? nullptr : it->second;
}

void free_pinned(SrvSession* ss) {
    for (int k = 0; k < 2; ++k)
        if (ss->pinned[k]) cudaFreeHost(ss->pinned[k]);
    if (ss->pinned_ctrl) cudaFreeHost(ss->pinned_ctrl);
    ss->pinned[0] = ss->pinned[1] = nullptr;
    ss->pinned_ctrl = nullptr;
    ss->pinned_ctrl_dev = nullptr;
}

}  // namespace

extern "C" {

double fc_server_now_ms(void) { return now_ms(); }

fc_status fc_server_session_bytes(int n_nodes, int n_samples, double fs, fc_band band, uint32_t metric_mask,
                                  int window, int plain, size_t* bytes) {
    if (!bytes || n_nodes < 2 || n_samples < 1 || window < 1) return sfail(FC_ERR_INVALID_ARG, "bad session settings");
    const int B = fc_band_bins(fs, band, nullptr);
    if (B <= 0) return sfail(FC_ERR_INVALID_ARG, "the band selects no bin");
    *bytes = fc_plan_session_bytes(n_nodes, n_samples, B, window, metric_mask, plain ? FC_MODE_FULL : FC_MODE_STREAM,
                                    FC_PREC_FP32, band.nfft);
    return FC_OK;
}

fc_status fc_server_create(const fc_server_config* cfg, fc_server** out) {
    if (!out) return sfail(FC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return sfail(FC_ERR_CUDA, "no CUDA device: this library has no CPU path");
    }
    fc_server* sv = new fc_server();
    if (cfg) sv->cfg = *cfg;
    if (sv->cfg.max_batch < 0 || sv->cfg.max_batch > FC_MAX_BATCH) {
        delete sv;
        return sfail(FC_ERR_INVALID_ARG, "max_batch must be 0..32");
    }
    if (sv->cfg.precision < FC_PREC_FP32 || sv->cfg.precision > FC_PREC_TF32X3) {
        delete sv;
        return sfail(FC_ERR_INVALID_ARG, "bad precision");
    }
    cudaGetDevice(&sv->device);
    sv->num_sms = fc_device_sms(sv->device);
    if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return sfail(FC_ERR_CUDA, "stream creation failed");
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return FC_OK;
}

fc_status fc_server_open(fc_server* sv, int n_nodes, int n_samples, double fs, fc_band band, fc_taper taper,
                         uint32_t metric_mask, int window, int* session_id) {
    if (!sv || !session_id) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    if (window < 1) return sfail(FC_ERR_INVALID_ARG, "served sessions need a window >= 1");
    size_t need = 0;
    fc_status st = fc_server_session_bytes(n_nodes, n_samples, fs, band, metric_mask, window, sv->cfg.plain, &need);
    if (st != FC_OK) return st;
    if (!sv->cfg.plain && sv->cfg.precision != FC_PREC_FP32) {  // the operand ring of a mixed-precision session
        const int B = fc_band_bins(fs, band, nullptr);
        need = fc_plan_session_bytes(n_nodes, n_samples, B, window, metric_mask, FC_MODE_STREAM, sv->cfg.precision,
                                      band.nfft);
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->cfg.hbm_budget && sv->used + need > sv->cfg.hbm_budget)
            return sfail(FC_ERR_ADMISSION, "device-memory budget exhausted: session not admitted");
        sv->used += need;  // reserve
    }
    fc_config cfg;
    fc_config_default(&cfg);
    cfg.stream = sv->stream;
    cfg.mode = sv->cfg.plain ? FC_MODE_FULL : FC_MODE_STREAM;
    if (!sv->cfg.plain) cfg.precision = sv->cfg.precision;
    fc_session* s = nullptr;
    {
        std::lock_guard<std::mutex> dk(sv->dev_mu);
        st = fc_session_create(n_nodes, n_samples, fs, band, taper, metric_mask, window, &cfg, &s);
    }
    if (st != FC_OK) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= need;
        return st;
    }
    if (!sv->cfg.plain) {
        // one bin group per tile pair: the batch kernel then finalizes every session in place
        s->stream_groups = 1;
        s->stream_group_bins = s->B;
    }
    SrvSession* ss = new SrvSession();
    ss->s = s;
    ss->bytes = need;
    ss->pair_bins = s->P * s->B;
    ss->trial_floats = (size_t)n_nodes * n_samples;
    ss->units = sv->cfg.plain ? 1 : (long long)s->ntp * s->stream_groups;
    bool pinned_ok = cudaHostAlloc(&ss->pinned_ctrl, 2 * sizeof(FcCtrl), cudaHostAllocMapped) == cudaSuccess &&
                     cudaHostGetDevicePointer(&ss->pinned_ctrl_dev, ss->pinned_ctrl, 0) == cudaSuccess;
    for (int k = 0; k < 2 && pinned_ok; ++k)
        pinned_ok = cudaMallocHost(&ss->pinned[k], ss->trial_floats * sizeof(float)) == cudaSuccess;
    if (!pinned_ok) {
        free_pinned(ss);
        {
            std::lock_guard<std::mutex> dk(sv->dev_mu);
            fc_session_destroy(s);
        }
        delete ss;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= need;
        return sfail(FC_ERR_OUT_OF_MEMORY, "pinned staging allocation failed");
    }
    std::memset(ss->pinned_ctrl, 0, 2 * sizeof(FcCtrl));
    std::lock_guard<std::mutex> lk(sv->mu);
    ss->id = sv->next_id++;
    sv->sessions[ss->id] = ss;
    *session_id = ss->id;
    return FC_OK;
}

fc_status fc_server_submit(fc_server* sv, int session_id, const float* x, double arrival_ms) {
    if (!sv || !x) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    size_t nf = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        SrvSession* ss = find_session(sv, session_id);
        if (!ss || ss->closing) return sfail(FC_ERR_INVALID_ARG, "unknown or closing session");
        nf = ss->trial_floats;
    }
    PendingTrial t;
    t.x.assign(x, x + nf);  // copied outside the lock
    t.arrival = arrival_ms;
    std::lock_guard<std::mutex> lk(sv->mu);
    SrvSession* ss = find_session(sv, session_id);
    if (!ss || ss->closing) return sfail(FC_ERR_INVALID_ARG, "unknown or closing session");
    t.seq = ss->submitted++;
    ss->queue.push_back(std::move(t));
    sv->stats.submitted++;
    sv->cv_work.notify_one();
    return FC_OK;
}

fc_status fc_server_poll(fc_server* sv, fc_result* out, int max, int* n_out, int wait_ms) {
    if (!sv || !n_out || (max > 0 && !out)) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->results.empty() && wait_ms > 0)
        sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&]() { return !sv->results.empty(); });
    int n = 0;
    while (n < max && !sv->results.empty()) {
        out[n++] = sv->results.front();
        sv->results.pop_front();
    }
    *n_out = n;
    if (!sv->worker_error.empty()) {
        std::string e = sv->worker_error;
        sv->worker_error.clear();
        return sfail(FC_ERR_CUDA, e.c_str());
    }
    return FC_OK;
}

fc_status fc_server_drain(fc_server* sv, int timeout_ms) {
    if (!sv) return sfail(FC_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto idle = [&]() {
        for (auto& kv : sv->sessions)
            if (!kv.second->queue.empty() || kv.second->in_flight > 0) return false;
        return true;
    };
    sv->cv_work.notify_one();
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        return sfail(FC_ERR_TIMEOUT, "trials still pending");
    return FC_OK;
}

fc_status fc_server_get_network(fc_server* sv, int session_id, uint32_t metric, float* out, size_t out_len) {
    if (!sv || !out) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    // the network after the last trial whose push is fully enqueued: wait while the device
    // state holds a partly applied push (its remaining shares follow within a few ticks)
    const double t_end = now_ms() + 60000.0;
    for (;;) {
        {
            std::lock_guard<std::mutex> dk(sv->dev_mu);
            fc_session* s = nullptr;
            bool partial = false;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                SrvSession* ss = find_session(sv, session_id);
                if (!ss) return sfail(FC_ERR_INVALID_ARG, "unknown session");
                s = ss->s;
                partial = ss->partial != 0;
            }
            if (!partial) {
                fc_status st = fc_get_network(s, metric, 1, out, out_len, 0, nullptr);
                // a rejected trial was already reported through its fc_result; the session's
                // one-time latch is consumed here and the network read again
                if (st == FC_ERR_NONFINITE) st = fc_get_network(s, metric, 1, out, out_len, 0, nullptr);
                return st;
            }
        }
        if (now_ms() > t_end) return sfail(FC_ERR_TIMEOUT, "the session stayed in the middle of a push");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

fc_status fc_server_close(fc_server* sv, int session_id) {
    if (!sv) return sfail(FC_ERR_INVALID_ARG, "NULL server");
    SrvSession* ss = nullptr;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        ss = find_session(sv, session_id);
        if (!ss) return sfail(FC_ERR_INVALID_ARG, "unknown session");
        ss->closing = true;
        sv->cv_work.notify_one();
        sv->cv_done.wait(lk, [&]() { return ss->queue.empty() && ss->in_flight == 0; });
        sv->sessions.erase(session_id);
    }
    {
        std::lock_guard<std::mutex> dk(sv->dev_mu);
        fc_session_destroy(ss->s);
    }
    free_pinned(ss);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->used -= ss->bytes;
    delete ss;
    return FC_OK;
}

fc_status fc_server_stats_get(fc_server* sv, fc_server_stats* st) {
    if (!sv || !st) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *st = sv->stats;
    st->hbm_used = sv->used;
    st->sessions = (int)sv->sessions.size();
    return FC_OK;
}

fc_status fc_server_destroy(fc_server* sv) {
    if (!sv) return FC_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& kv : sv->sessions) {
        fc_session_destroy(kv.second->s);
        free_pinned(kv.second);
        delete kv.second;
    }
    for (cudaEvent_t e : sv->event_pool) cudaEventDestroy(e);
    cudaStreamDestroy(sv->stream);
    delete sv;
    return FC_OK;
}

}  // extern "C"
