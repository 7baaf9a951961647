// Serving runtime: a request loop over daq_process_fills.
//
// Requests (one fill each) enter a FIFO.  A worker thread admits the oldest
// request whose arrival time has come as soon as a slot is free: it gives the
// fill a slot (outputs + workspace carved from one allocation made at
// creation within the memory budget), enqueues its work on the next of
// several streams between two timing events, and copies the fill's counts to
// page-locked host memory behind it.  Fills on different streams overlap on
// the GPU.  The worker retires fills whose completion event has fired, turns
// their events into server-clock times and, with auto-release, frees the slot
// at once.  Every fill adds its Q bins to one resident histogram; integer sums
// make that result independent of order and overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "daq.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxStreams = 16;
constexpr int kMaxSlots = 64;

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

struct Slot {
    int16_t *input = nullptr;  // DAQ_SERVER_HOST_INPUT only
    daq_island *hdr = nullptr;
    int16_t *pool = nullptr;
    int32_t *ped = nullptr;
    int64_t *counts = nullptr;
    void *ws = nullptr;
    int32_t *len = nullptr;    // device fill length
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_copied = nullptr;  // DAQ_SERVER_HOST_INPUT: the fill's samples are on the device
    int64_t ticket = 0;        // 0 = free
    int stream = 0;
};

struct Fill {
    daq_fill_record rec{};
    int state = DAQ_FILL_QUEUED;
    const int16_t *samples = nullptr;
    bool on_host = false;
    int32_t len = 0;
};

}  // namespace

struct daq_server {
    daq_server_config cfg{};
    int device = 0;
    size_t slot_bytes = 0, ws_bytes = 0;
    int64_t hdr_cap = 0, pool_cap = 0;
    unsigned char *arena = nullptr;
    int64_t *q = nullptr;
    bool own_q = false;
    int64_t q_values = 0;
    std::vector<Slot> slots;
    int64_t *counts_host = nullptr;  // [n_slots][4], page-locked
    int32_t *len_host = nullptr;     // [n_slots], page-locked
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    // DAQ_SERVER_HOST_INPUT: host-to-device copies of fills, one at a time in
    // admission order, so that each fill's copy ends as early as the link
    // allows (copies spread over the processing streams would share the link
    // and all end late)
    cudaStream_t copy_stream = nullptr;

    Clock::time_point t0;
    cudaEvent_t ref_ev = nullptr;
    double ref_us = 0.0;  // server-clock time of ref_ev
    double last_anchor_us = 0.0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Fill> fills;
    std::vector<daq_fill_record> done_records;
    int64_t next_ticket = 1;
    daq_server_stats st{};
    bool stop = false;
    std::thread worker;

    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }
};

namespace {

// Re-anchor the event clock: with nothing in flight, record an event, wait for
// it and take the host time (the GPU reaches an idle event within
// microseconds).
void anchor_clock(daq_server *s)
{
    if (cudaEventRecord(s->ref_ev, s->streams[0]) != cudaSuccess) return;
    cudaEventSynchronize(s->ref_ev);
    s->ref_us = s->now_us();
    s->last_anchor_us = s->ref_us;
}

double event_us(daq_server *s, cudaEvent_t e)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ref_ev, e) != cudaSuccess) return -1.0;
    return s->ref_us + 1e3 * (double)ms;
}

// Enqueue one fill on a free slot (worker thread, lock held).
void admit(daq_server *s, int si, Fill &f)
{
    Slot &sl = s->slots[si];
    const daq_server_config &c = s->cfg;
    sl.ticket = f.rec.ticket;
    sl.stream = s->next_stream;
    s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
    cudaStream_t st = s->streams[sl.stream];
    f.rec.slot = si;
    f.rec.t_admit = s->now_us();
    f.state = DAQ_FILL_RUNNING;

    const int64_t X = c.n_xtal, N = c.n_samples;
    daq_params p = c.params;
    p.stream = st;
    p.workspace = sl.ws;
    p.workspace_bytes = s->ws_bytes;
    p.events = nullptr;
    p.trace = nullptr;
    p.flags &= ~DAQ_SYNC;
    s->len_host[si] = f.len;
    p.fill_len = sl.len;
    daq_islands isl{sl.hdr, s->hdr_cap, sl.pool, s->pool_cap, sl.ped, sl.counts};
    const int16_t *in = f.samples;
    int rc = DAQ_OK;
    // the fill's work starts with its copy (host input) or its processing
    if (cudaEventRecord(sl.ev_start, f.on_host ? s->copy_stream : st) != cudaSuccess) rc = DAQ_ECUDA;
    if (rc == DAQ_OK &&
        cudaMemcpyAsync(sl.len, &s->len_host[si], sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = DAQ_ECUDA;
    if (rc == DAQ_OK && f.on_host) {
        if (cudaMemcpyAsync(sl.input, f.samples, (size_t)c.n_calo * X * N * sizeof(int16_t), cudaMemcpyHostToDevice,
                            s->copy_stream) != cudaSuccess ||
            cudaEventRecord(sl.ev_copied, s->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(st, sl.ev_copied, 0) != cudaSuccess)
            rc = DAQ_ECUDA;
        in = sl.input;
    }
    if (rc == DAQ_OK) rc = daq_process_fills(in, c.n_calo, c.n_xtal, N, 1, &p, &isl, s->q);
    if (rc == DAQ_OK && cudaMemcpyAsync(&s->counts_host[4 * si], sl.counts, 4 * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = DAQ_ECUDA;
    if (cudaEventRecord(sl.ev_done, st) != cudaSuccess && rc == DAQ_OK) rc = DAQ_ECUDA;
    f.rec.status = rc;  // an enqueue failure; the device status is read at retirement otherwise
    ++s->st.admitted;
    ++s->st.running;
    s->st.max_running = std::max(s->st.max_running, s->st.running);
}

// Retire a running fill whose completion event has fired (lock held).
void retire(daq_server *s, int si)
{
    Slot &sl = s->slots[si];
    Fill &f = s->fills[sl.ticket];
    const int64_t *ch = &s->counts_host[4 * si];
    if (f.rec.status == DAQ_OK) {
        f.rec.status = daq_status_from_counts(ch);
        f.rec.n_islands = ch[0];
        f.rec.n_rows = ch[1];
    }
    f.rec.t_start = event_us(s, sl.ev_start);
    f.rec.t_done = event_us(s, sl.ev_done);
    if (f.rec.t_done < 0) f.rec.t_done = s->now_us();
    if (f.rec.t_start < 0) f.rec.t_start = f.rec.t_admit;
    f.state = DAQ_FILL_DONE;
    --s->st.running;
    ++s->st.completed;
    if (f.rec.status != DAQ_OK) ++s->st.failed;
    s->done_records.push_back(f.rec);
    if (s->cfg.flags & DAQ_SERVER_AUTO_RELEASE) {
        f.state = DAQ_FILL_RELEASED;
        ++s->st.released;
        sl.ticket = 0;
        s->fills.erase(f.rec.ticket);
    }
}

void worker_main(daq_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        // retire
        for (int i = 0; i < (int)s->slots.size(); ++i) {
            Slot &sl = s->slots[i];
            if (!sl.ticket) continue;
            auto it = s->fills.find(sl.ticket);
            if (it == s->fills.end() || it->second.state != DAQ_FILL_RUNNING) continue;
            const cudaError_t q = cudaEventQuery(sl.ev_done);
            if (q == cudaErrorNotReady) continue;
            retire(s, i);
            progressed = true;
        }
        // admit, in arrival order
        const double now = s->now_us();
        double next_arrival = -1.0;
        while (!s->queue.empty()) {
            Fill &f = s->fills[s->queue.front()];
            if (f.rec.t_arrival > now) {
                next_arrival = f.rec.t_arrival;
                break;
            }
            int free_slot = -1;
            for (int i = 0; i < (int)s->slots.size(); ++i)
                if (!s->slots[i].ticket) {
                    free_slot = i;
                    break;
                }
            if (free_slot < 0) break;
            s->queue.pop_front();
            --s->st.queued;
            admit(s, free_slot, f);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        if (s->stop && s->queue.empty() && s->st.running == 0) break;
        if (s->st.running == 0 && s->now_us() - s->last_anchor_us > 50e3) anchor_clock(s);
        if (s->st.running > 0 || (next_arrival >= 0 && next_arrival - s->now_us() < 2000.0)) {
            // fills in flight or an arrival due within 2 ms: poll without sleeping
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else if (next_arrival >= 0) {
            s->cv_work.wait_for(lk, std::chrono::microseconds((int64_t)(next_arrival - s->now_us() - 1500.0)));
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

void free_server(daq_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.ev_start) cudaEventDestroy(sl.ev_start);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        if (sl.ev_copied) cudaEventDestroy(sl.ev_copied);
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->ref_ev) cudaEventDestroy(s->ref_ev);
    if (s->arena) cudaFree(s->arena);
    if (s->own_q && s->q) cudaFree(s->q);
    if (s->counts_host) cudaFreeHost(s->counts_host);
    if (s->len_host) cudaFreeHost(s->len_host);
    delete s;
}

double percentile(std::vector<double> v, double q)
{
    std::sort(v.begin(), v.end());
    const double pos = q / 100.0 * (double)(v.size() - 1);
    const size_t i = (size_t)std::floor(pos);
    const double fr = pos - (double)i;
    if (i + 1 >= v.size()) return v.back();
    return v[i] + fr * (v[i + 1] - v[i]);
}

}  // namespace

extern "C" {

int daq_server_create(const daq_server_config *cfg, daq_server **out)
{
    if (!out) return DAQ_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->n_calo < 1 || cfg->n_xtal < 1 || cfg->n_samples < 1 || cfg->mem_budget_bytes == 0 ||
        cfg->max_slots < 0 || cfg->n_streams < 0 || cfg->n_streams > kMaxStreams || cfg->hdr_cap < 0 ||
        cfg->pool_row_cap < 0 || (cfg->flags & ~(DAQ_SERVER_HOST_INPUT | DAQ_SERVER_AUTO_RELEASE)))
        return DAQ_EINVAL;
    daq_params p = cfg->params;
    p.fill_len = nullptr;
    size_t ws = 0;
    int rc = daq_workspace_size(cfg->n_calo, cfg->n_xtal, cfg->n_samples, 1, &p, &ws);
    if (rc != DAQ_OK) return rc;
    int64_t nq = 0;
    for (int d = 0; d < p.n_decim; ++d) nq += (int64_t)cfg->n_calo * daq_q_bins(cfg->n_samples, p.decim[d]);

    const int64_t C = cfg->n_calo, X = cfg->n_xtal, N = cfg->n_samples;
    const int64_t pool_cap = cfg->pool_row_cap ? cfg->pool_row_cap : C * N;
    const int64_t hdr_cap = cfg->hdr_cap ? cfg->hdr_cap : C * N / 2 + C + 1;
    size_t slot = 0;
    if (cfg->flags & DAQ_SERVER_HOST_INPUT) slot += up256((size_t)(C * X * N) * 2);
    slot += up256((size_t)hdr_cap * sizeof(daq_island));
    slot += up256((size_t)pool_cap * (size_t)X * 2);
    slot += up256((size_t)(C * X) * 4);
    slot += up256(4 * sizeof(int64_t));
    slot += up256(ws);
    slot += up256(sizeof(int32_t));
    const int cap_slots = cfg->max_slots ? std::min(cfg->max_slots, kMaxSlots) : kMaxSlots;
    const int n_slots = (int)std::min<size_t>((size_t)cap_slots, cfg->mem_budget_bytes / slot);
    if (n_slots < 1) return DAQ_EINVAL;  // the budget does not hold one fill

    daq_server *s = new daq_server();
    s->cfg = *cfg;
    s->cfg.params.fill_len = nullptr;
    s->slot_bytes = slot;
    s->ws_bytes = ws;
    s->hdr_cap = hdr_cap;
    s->pool_cap = pool_cap;
    s->q_values = nq;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    auto fail = [&](int code) {
        free_server(s);
        return code;
    };
    if (cudaMalloc(&s->arena, slot * (size_t)n_slots) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cudaMallocHost(&s->counts_host, sizeof(int64_t) * 4 * n_slots) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cudaMallocHost(&s->len_host, sizeof(int32_t) * n_slots) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cfg->qhist) {
        s->q = cfg->qhist;
    } else if (nq > 0) {
        if (cudaMalloc(&s->q, (size_t)nq * 8) != cudaSuccess) return fail(DAQ_ECUDA);
        s->own_q = true;
        if (cudaMemset(s->q, 0, (size_t)nq * 8) != cudaSuccess) return fail(DAQ_ECUDA);
    }
    s->slots.resize(n_slots);
    for (int i = 0; i < n_slots; ++i) {
        unsigned char *b = s->arena + (size_t)i * slot;
        Slot &sl = s->slots[i];
        if (cfg->flags & DAQ_SERVER_HOST_INPUT) {
            sl.input = reinterpret_cast<int16_t *>(b);
            b += up256((size_t)(C * X * N) * 2);
        }
        sl.hdr = reinterpret_cast<daq_island *>(b);
        b += up256((size_t)hdr_cap * sizeof(daq_island));
        sl.pool = reinterpret_cast<int16_t *>(b);
        b += up256((size_t)pool_cap * (size_t)X * 2);
        sl.ped = reinterpret_cast<int32_t *>(b);
        b += up256((size_t)(C * X) * 4);
        sl.counts = reinterpret_cast<int64_t *>(b);
        b += up256(4 * sizeof(int64_t));
        sl.ws = b;
        b += up256(ws);
        sl.len = reinterpret_cast<int32_t *>(b);
        if (cudaEventCreate(&sl.ev_start) != cudaSuccess || cudaEventCreate(&sl.ev_done) != cudaSuccess)
            return fail(DAQ_ECUDA);
        if ((cfg->flags & DAQ_SERVER_HOST_INPUT) &&
            cudaEventCreateWithFlags(&sl.ev_copied, cudaEventDisableTiming) != cudaSuccess)
            return fail(DAQ_ECUDA);
    }
    if ((cfg->flags & DAQ_SERVER_HOST_INPUT) &&
        cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(DAQ_ECUDA);
    const int n_streams = cfg->n_streams ? cfg->n_streams : 4;
    s->streams.resize(n_streams, nullptr);
    for (int i = 0; i < n_streams; ++i)
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cudaEventCreate(&s->ref_ev) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(DAQ_ECUDA);
    anchor_clock(s);
    s->st.n_slots = n_slots;
    s->st.n_streams = n_streams;
    s->st.slot_bytes = slot;
    s->st.mem_bytes = slot * (size_t)n_slots;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DAQ_OK;
}

int daq_server_submit(daq_server *s, const int16_t *samples, int on_host, int32_t fill_len, double arrival_us,
                      int64_t *ticket)
{
    if (!s || !samples || !ticket) return DAQ_EINVAL;
    if (on_host && !(s->cfg.flags & DAQ_SERVER_HOST_INPUT)) return DAQ_EINVAL;
    if (fill_len < 0) fill_len = (int32_t)std::min<int64_t>(s->cfg.n_samples, INT32_MAX);
    if ((int64_t)fill_len > s->cfg.n_samples) return DAQ_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    Fill f;
    f.rec.ticket = s->next_ticket++;
    f.rec.t_arrival = arrival_us < 0 ? s->now_us() : arrival_us;
    f.rec.raw_bytes = (int64_t)s->cfg.n_calo * s->cfg.n_xtal * fill_len * 2;
    f.rec.slot = -1;
    f.samples = samples;
    f.on_host = on_host != 0;
    f.len = fill_len;
    *ticket = f.rec.ticket;
    s->fills.emplace(f.rec.ticket, f);
    s->queue.push_back(f.rec.ticket);
    ++s->st.submitted;
    ++s->st.queued;
    s->cv_work.notify_one();
    return DAQ_OK;
}

static void fill_result(daq_server *s, const Fill &f, daq_fill_result *out)
{
    std::memset(out, 0, sizeof(*out));
    out->rec = f.rec;
    out->state = f.state;
    if (f.state == DAQ_FILL_DONE && f.rec.slot >= 0) {
        const Slot &sl = s->slots[f.rec.slot];
        out->hdr = sl.hdr;
        out->pool = sl.pool;
        out->pedestal = sl.ped;
    }
}

int daq_server_poll(daq_server *s, int64_t ticket, daq_fill_result *out)
{
    if (!s || !out) return DAQ_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->fills.find(ticket);
    if (it == s->fills.end()) {
        for (const daq_fill_record &r : s->done_records)  // auto-released: record only
            if (r.ticket == ticket) {
                std::memset(out, 0, sizeof(*out));
                out->rec = r;
                out->state = DAQ_FILL_RELEASED;
                return DAQ_OK;
            }
        return DAQ_EINVAL;
    }
    fill_result(s, it->second, out);
    return DAQ_OK;
}

int daq_server_wait(daq_server *s, int64_t ticket, double timeout_s, daq_fill_result *out)
{
    if (!s) return DAQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    while (true) {
        auto it = s->fills.find(ticket);
        if (it == s->fills.end()) {
            lk.unlock();
            return out ? daq_server_poll(s, ticket, out) : DAQ_OK;
        }
        if (it->second.state >= DAQ_FILL_DONE) {
            if (out) fill_result(s, it->second, out);
            return DAQ_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return DAQ_ETIMEOUT;
    }
}

int daq_server_fetch(daq_server *s, int64_t ticket, daq_island *hdr_host, int64_t hdr_cap, int16_t *pool_host,
                     int64_t pool_cap, int32_t *ped_host)
{
    if (!s || hdr_cap < 0 || pool_cap < 0 || (hdr_cap > 0 && !hdr_host) || (pool_cap > 0 && !pool_host))
        return DAQ_EINVAL;
    const daq_island *hdr = nullptr;
    const int16_t *pool = nullptr;
    const int32_t *ped = nullptr;
    int64_t n_isl = 0, n_rows = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->fills.find(ticket);
        if (it == s->fills.end() || it->second.state != DAQ_FILL_DONE || it->second.rec.slot < 0) return DAQ_EINVAL;
        const Slot &sl = s->slots[it->second.rec.slot];
        hdr = sl.hdr;
        pool = sl.pool;
        ped = sl.ped;
        n_isl = std::min(it->second.rec.n_islands, s->hdr_cap);
        n_rows = std::min(it->second.rec.n_rows, s->pool_cap);
    }
    // The slot stays with this fill until the caller releases it, so the copy
    // runs without the lock (the fill's work has completed).
    n_isl = std::min(n_isl, hdr_cap);
    n_rows = std::min(n_rows, pool_cap);
    if (n_isl > 0 && cudaMemcpy(hdr_host, hdr, (size_t)n_isl * sizeof(daq_island), cudaMemcpyDeviceToHost) !=
                         cudaSuccess)
        return DAQ_ECUDA;
    if (n_rows > 0 && cudaMemcpy(pool_host, pool, (size_t)n_rows * s->cfg.n_xtal * sizeof(int16_t),
                                 cudaMemcpyDeviceToHost) != cudaSuccess)
        return DAQ_ECUDA;
    if (ped_host && cudaMemcpy(ped_host, ped, (size_t)s->cfg.n_calo * s->cfg.n_xtal * sizeof(int32_t),
                               cudaMemcpyDeviceToHost) != cudaSuccess)
        return DAQ_ECUDA;
    return DAQ_OK;
}

int daq_server_release(daq_server *s, int64_t ticket)
{
    if (!s) return DAQ_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->fills.find(ticket);
    if (it == s->fills.end() || it->second.state != DAQ_FILL_DONE) return DAQ_EINVAL;
    if (it->second.rec.slot >= 0) s->slots[it->second.rec.slot].ticket = 0;
    ++s->st.released;
    s->fills.erase(it);
    s->cv_work.notify_one();
    return DAQ_OK;
}

int daq_server_drain(daq_server *s, double timeout_s)
{
    if (!s) return DAQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    while (s->st.queued > 0 || s->st.running > 0) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return DAQ_ETIMEOUT;
    }
    return DAQ_OK;
}

int daq_server_get_stats(daq_server *s, daq_server_stats *out)
{
    if (!s || !out) return DAQ_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    return DAQ_OK;
}

int daq_server_records(daq_server *s, daq_fill_record *out, int64_t cap, int64_t *n, int clear)
{
    if (!s || !n || cap < 0 || (cap > 0 && !out)) return DAQ_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *n = (int64_t)s->done_records.size();
    const int64_t k = std::min<int64_t>(cap, *n);
    if (k > 0) std::memcpy(out, s->done_records.data(), (size_t)k * sizeof(daq_fill_record));
    if (clear) s->done_records.clear();
    return DAQ_OK;
}

int64_t *daq_server_qhist(daq_server *s) { return s ? s->q : nullptr; }

double daq_server_now_us(daq_server *s) { return s ? s->now_us() : -1.0; }

int daq_server_destroy(daq_server *s)
{
    if (!s) return DAQ_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        // requests not yet admitted are dropped
        s->st.queued = 0;
        for (int64_t t : s->queue) s->fills.erase(t);
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    free_server(s);
    return DAQ_OK;
}

int daq_serving_summarize(const daq_fill_record *recs, int64_t n, daq_serving_summary *out)
{
    if (!out || n < 0 || (n > 0 && !recs)) return DAQ_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->n = n;
    if (n == 0) return DAQ_OK;
    std::vector<const daq_fill_record *> v(n);
    for (int64_t i = 0; i < n; ++i) v[i] = &recs[i];
    std::stable_sort(v.begin(), v.end(), [](const daq_fill_record *a, const daq_fill_record *b) {
        return a->t_arrival < b->t_arrival;
    });
    std::vector<double> lat(n);
    double bytes = 0.0, t_first = v[0]->t_arrival, t_last = v[0]->t_done;
    for (int64_t i = 0; i < n; ++i) {
        lat[i] = v[i]->t_done - v[i]->t_arrival;
        bytes += (double)v[i]->raw_bytes;
        t_last = std::max(t_last, v[i]->t_done);
    }
    out->latency_p50_us = percentile(lat, 50.0);
    out->latency_p99_us = percentile(lat, 99.0);
    out->latency_max_us = *std::max_element(lat.begin(), lat.end());
    int64_t dead = 0;
    for (int64_t i = 0; i + 1 < n; ++i)
        if (v[i]->t_done > v[i + 1]->t_arrival) ++dead;
    out->deadtime = n > 1 ? (double)dead / (double)(n - 1) : 0.0;
    out->span_us = t_last - t_first;
    out->gbs = out->span_us > 0 ? bytes / out->span_us / 1e3 : 0.0;
    return DAQ_OK;
}

}  // extern "C"
