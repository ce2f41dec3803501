// fc_server.cu - serving many concurrent sessions with continuous batching.
//
// The paper's online pipeline adds every newly arriving trial to the network as it comes
// (Methods 2.5; Results 3.2.3) and must keep up with the acquisition (Results 3.2.3: a
// 500-sample block at 1,792 Hz leaves 280 ms). Here many sessions share one GPU: each
// arriving trial of any session is a request; a worker thread takes, at every tick, the
// oldest pending trial of each session that has one (oldest arrivals first across
// sessions, at most max_batch sessions) and runs them through ONE launch of the
// persistent streaming kernel (their small per-session kernels - validation, spectrum,
// per-node sums, commit - around it). Trials that arrive while a launch runs join the
// next tick; two launches may be in flight, so the host staging of the next batch
// overlaps the device work of the current one. Session state stays resident; sessions
// are admitted against a device-memory budget.
//
// In plain mode (the comparison baseline) every trial is handled alone, in arrival
// order, as a full-window FP32 recompute (FC_MODE_FULL), with no batching and no
// streaming sums.
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

double now_ms() {
    using namespace std::chrono;
    static const steady_clock::time_point t0 = steady_clock::now();
    return duration<double, std::milli>(steady_clock::now() - t0).count();
}

struct PendingTrial {
    std::vector<float> x;
    double arrival;
    long long seq;
};

struct SrvSession {
    int id = 0;
    fc_session* s = nullptr;
    size_t bytes = 0;
    long long pair_bins = 0;
    size_t trial_floats = 0;
    std::deque<PendingTrial> queue;
    long long submitted = 0, completed = 0, in_flight = 0;
    float* pinned[2] = {nullptr, nullptr};
    float* pinned_scale = nullptr;  // the session's prescale, read back after its first pushes
    bool closing = false;
};

struct Item {
    SrvSession* ss;
    PendingTrial t;
    int launch_sessions = 1;  // sessions that shared this trial's streaming-kernel launch
};

struct InFlight {
    cudaEvent_t ev = nullptr;
    std::vector<Item> items;
};

}  // namespace

struct fc_server {
    fc_server_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 152;
    std::mutex mu;                  // sessions, queues, results, stats
    std::mutex dev_mu;              // device work on sessions (worker enqueue vs API calls)
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

// Enqueue one batch on the server stream (called by the worker with dev_mu held).
fc_status enqueue_batch(fc_server* sv, std::vector<Item>& items, InFlight& fl) {
    const int slot = sv->parity;
    sv->parity ^= 1;
    for (Item& it : items) {
        SrvSession* ss = it.ss;
        std::memcpy(ss->pinned[slot], it.t.x.data(), ss->trial_floats * sizeof(float));
        cudaError_t e = cudaMemcpyAsync(ss->s->x_stage, ss->pinned[slot], ss->trial_floats * sizeof(float),
                                        cudaMemcpyHostToDevice, sv->stream);
        if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (sv->cfg.plain) {
        for (Item& it : items) {
            fc_status st = fc_push_single(it.ss->s, it.ss->s->x_stage);
            if (st != FC_OK) return st;
        }
    } else {
        StreamBatch b;
        b.nsess = 0;
        b.unit_prefix[0] = 0;
        std::vector<fc_session*> batched;
        for (Item& it : items) {
            fc_session* s = it.ss->s;
            if (fc_push_needs_single(s)) {
                fc_status st = fc_push_single(s, s->x_stage);
                if (st != FC_OK) return st;
                if (!s->calibrated) {
                    // the push set the prescale on the device; read it back with the batch
                    cudaError_t e = cudaMemcpyAsync(it.ss->pinned_scale, &s->ctrl->scale, sizeof(float),
                                                    cudaMemcpyDeviceToHost, sv->stream);
                    if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
                }
                continue;
            }
            fc_status st = fc_push_stage_pre(s, s->x_stage);
            if (st != FC_OK) return st;
            const PairArgs pa = fc_push_stream_args(s);
            b.a[b.nsess] = pa;
            b.unit_prefix[b.nsess + 1] = b.unit_prefix[b.nsess] + pa.ntp * pa.groups;
            ++b.nsess;
            batched.push_back(s);
        }
        for (Item& it : items)
            if (std::find(batched.begin(), batched.end(), it.ss->s) != batched.end()) it.launch_sessions = b.nsess;
        if (b.nsess > 0) {
            cudaError_t e = launch_stream_batch(b, 2 * sv->num_sms, sv->stream);
            if (e != cudaSuccess) return sfail(FC_ERR_CUDA, cudaGetErrorString(e));
            fc_count_launch(batched[0]);
            for (fc_session* s : batched) {
                fc_status st = fc_push_stage_post(s);
                if (st != FC_OK) return st;
            }
        }
    }
    if (!sv->event_pool.empty()) {
        fl.ev = sv->event_pool.back();
        sv->event_pool.pop_back();
    } else {
        cudaEventCreateWithFlags(&fl.ev, cudaEventDisableTiming);
    }
    cudaEventRecord(fl.ev, sv->stream);
    fl.items = std::move(items);
    return FC_OK;
}

void retire(fc_server* sv, InFlight& fl) {
    cudaEventSynchronize(fl.ev);
    const double done = now_ms();
    {
        // a session whose prescale is now known joins the batched launches from its next trial
        std::lock_guard<std::mutex> dk(sv->dev_mu);
        for (Item& it : fl.items)
            if (!it.ss->s->calibrated && *it.ss->pinned_scale != 0.f) it.ss->s->calibrated = true;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->event_pool.push_back(fl.ev);
    for (Item& it : fl.items) {
        fc_result r;
        r.session = it.ss->id;
        r.seq = it.t.seq;
        r.status = FC_OK;
        r.arrival_ms = it.t.arrival;
        r.done_ms = done;
        r.batch = it.launch_sessions;
        sv->results.push_back(r);
        it.ss->completed++;
        it.ss->in_flight--;
        sv->stats.completed++;
        sv->stats.pair_bin_updates += it.ss->pair_bins;
    }
    sv->cv_done.notify_all();
}

void worker_main(fc_server* sv) {
    cudaSetDevice(sv->device);
    const int max_batch = sv->cfg.plain ? 1 : (sv->cfg.max_batch > 0 ? std::min(sv->cfg.max_batch, FC_MAX_BATCH)
                                                                       : FC_MAX_BATCH);
    for (;;) {
        std::vector<Item> items;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            auto has_work = [&]() {
                for (auto& kv : sv->sessions)
                    if (!kv.second->queue.empty()) return true;
                return false;
            };
            if (sv->inflight.empty())
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&]() { return sv->stop || has_work(); });
            if (sv->stop && !has_work() && sv->inflight.empty()) break;
            // oldest arrival first across sessions, one trial per session per launch
            std::vector<SrvSession*> cand;
            for (auto& kv : sv->sessions)
                if (!kv.second->queue.empty()) cand.push_back(kv.second);
            std::sort(cand.begin(), cand.end(), [](SrvSession* a, SrvSession* b) {
                return a->queue.front().arrival < b->queue.front().arrival;
            });
            if ((int)cand.size() > max_batch) cand.resize(max_batch);
            for (SrvSession* ss : cand) {
                items.push_back(Item{ss, std::move(ss->queue.front())});
                ss->queue.pop_front();
                ss->in_flight++;
            }
        }
        if (!items.empty()) {
            InFlight fl;
            const int n_items = (int)items.size();
            fc_status st;
            {
                std::lock_guard<std::mutex> dk(sv->dev_mu);
                st = enqueue_batch(sv, items, fl);
            }
            if (st != FC_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->worker_error = fc_last_error();
                for (Item& it : items) it.ss->in_flight--;
                sv->cv_done.notify_all();
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->stats.launches++;
                sv->stats.batched_trials += n_items;
            }
            sv->inflight.push_back(std::move(fl));
        }
        // keep at most two launches in flight; retire the oldest when idle or full
        while (!sv->inflight.empty() && (sv->inflight.size() >= 2 || items.empty())) {
            retire(sv, sv->inflight.front());
            sv->inflight.pop_front();
            if (!items.empty()) break;
        }
    }
}

void free_pinned(SrvSession* ss) {
    for (int k = 0; k < 2; ++k)
        if (ss->pinned[k]) cudaFreeHost(ss->pinned[k]);
    if (ss->pinned_scale) cudaFreeHost(ss->pinned_scale);
    ss->pinned[0] = ss->pinned[1] = ss->pinned_scale = nullptr;
}

SrvSession* find_session(fc_server* sv, int id) {
    auto it = sv->sessions.find(id);
    return it == sv->sessions.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

double fc_server_now_ms(void) { return now_ms(); }

fc_status fc_server_session_bytes(int n_nodes, int n_samples, double fs, fc_band band, uint32_t metric_mask,
                                  int window, int plain, size_t* bytes) {
    if (!bytes || n_nodes < 2 || n_samples < 1 || window < 1) return sfail(FC_ERR_INVALID_ARG, "bad session settings");
    const int B = fc_band_bins(fs, band, nullptr);
    if (B <= 0) return sfail(FC_ERR_INVALID_ARG, "the band selects no bin");
    *bytes = fc_plan_session_bytes(n_nodes, n_samples, B, window, metric_mask, plain ? FC_MODE_FULL : FC_MODE_STREAM);
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
    cudaGetDevice(&sv->device);
    cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device);
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
    bool pinned_ok = cudaMallocHost(&ss->pinned_scale, sizeof(float)) == cudaSuccess;
    for (int k = 0; k < 2 && pinned_ok; ++k)
        pinned_ok = cudaMallocHost(&ss->pinned[k], ss->trial_floats * sizeof(float)) == cudaSuccess;
    if (!pinned_ok) {
        free_pinned(ss);
        fc_session_destroy(s);
        delete ss;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= need;
        return sfail(FC_ERR_OUT_OF_MEMORY, "pinned staging allocation failed");
    }
    *ss->pinned_scale = 0.f;
    std::lock_guard<std::mutex> lk(sv->mu);
    ss->id = sv->next_id++;
    sv->sessions[ss->id] = ss;
    *session_id = ss->id;
    return FC_OK;
}

fc_status fc_server_submit(fc_server* sv, int session_id, const float* x, double arrival_ms) {
    if (!sv || !x) return sfail(FC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    SrvSession* ss = find_session(sv, session_id);
    if (!ss || ss->closing) return sfail(FC_ERR_INVALID_ARG, "unknown or closing session");
    PendingTrial t;
    t.x.assign(x, x + ss->trial_floats);
    t.arrival = arrival_ms;
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
    fc_session* s = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        SrvSession* ss = find_session(sv, session_id);
        if (!ss) return sfail(FC_ERR_INVALID_ARG, "unknown session");
        s = ss->s;
    }
    std::lock_guard<std::mutex> dk(sv->dev_mu);
    return fc_get_network(s, metric, 1, out, out_len, 0, nullptr);
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
