// Serving loop: requests of one read each are admitted continuously and
// aligned in micro-batches, several of them in flight at once.
//
// The thesis aligns files batch by batch (Sec. "Data array serialisation"
// packs a batch, one launch per batch); a server cannot wait for a full
// batch.  Here a worker thread closes a micro-batch when it holds
// max_batch_reads requests or max_wait_us after its oldest request arrived
// (short reads and longer ones queue and batch apart; see run()),
// takes the first internal context whose previous micro-batch has finished,
// packs the requests into that context's page-locked staging and enqueues
// the whole path (copies in, pre-kernel, core kernel, copies out) on the
// context's stream without waiting.  A host function enqueued behind the
// copies out (cudaLaunchHostFunc; it calls no CUDA API) moves each result to
// its request, stamps the completion time and frees the context.  While a
// micro-batch with long reads is running, later requests run on the other
// contexts, and one context is always left for short requests.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "abea_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class State { Free, Queued, Running, Done };

struct Request {
    int64_t ticket = -1;
    State state = State::Free;
    std::vector<char> seq;
    std::vector<float> ev;
    abea_scalings sc{};
    int64_t pair_cap = 0;        // n_e + n_k - 1: every path fits
    size_t bytes = 0;            // device bytes in a micro-batch
    abea_result res{};
    std::vector<int32_t> pairs;
    int err = ABEA_OK;
    Clock::time_point t_submit, t_done;
};

// A page-locked host array that only grows (never while its context runs).
template <typename T>
struct Pinned {
    T *p = nullptr;
    size_t cap = 0;
    int reserve(size_t n)
    {
        n = std::max<size_t>(n, 1);
        if (n <= cap) return ABEA_OK;
        const size_t want = std::max(n, cap + cap / 2);
        release();
        if (cudaHostAlloc((void **)&p, want * sizeof(T), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return ABEA_ERR_NOMEM;
        }
        cap = want;
        return ABEA_OK;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

struct Slot {
    abea_server *srv = nullptr;
    abea_ctx *ctx = nullptr;
    bool busy = false;
    std::vector<int32_t> reqs;   // request indices of the running micro-batch
    std::vector<int64_t> seq_off, ev_off, pair_off;
    std::vector<abea_scalings> sc;
    Pinned<char> seq;
    Pinned<float> ev;
    Pinned<abea_result> out;
    Pinned<int32_t> pairs;
};

}  // namespace

struct abea_server {
    abea_server_cfg cfg{};
    int device = 0;
    int k = 0;
    size_t budget = 0;                 // per internal context
    std::vector<Request> table;        // max_requests entries; index = ticket % max_requests
    std::vector<int32_t> free_idx;
    std::deque<int32_t> fifo[2];       // queued requests, oldest first: [0] short reads, [1] the others
    std::vector<Slot> slots;
    std::mutex m;
    std::condition_variable cv_work;   // the worker: a request was queued, a micro-batch finished, or stop
    std::condition_variable cv_done;   // pollers: a micro-batch finished
    std::thread worker;
    bool stopping = false;
    int64_t serial = 0;
};

namespace {

bool all_free(const abea_server *s)
{
    for (const Slot &x : s->slots)
        if (x.busy) return false;
    return true;
}

// Host function behind a micro-batch's copies out.
void CUDART_CB batch_done(void *arg)
{
    Slot *slot = static_cast<Slot *>(arg);
    abea_server *s = slot->srv;
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->m);
        for (size_t t = 0; t < slot->reqs.size(); t++) {
            Request &r = s->table[slot->reqs[t]];
            r.res = slot->out.p[t];
            const int64_t cnt = (r.res.status == ABEA_READ_OK) ? std::min<int64_t>(r.res.n_pairs, r.pair_cap) : 0;
            const int32_t *src = slot->pairs.p + 2 * slot->pair_off[t];
            r.pairs.assign(src, src + 2 * cnt);
            r.state = State::Done;
            r.t_done = now;
        }
        slot->busy = false;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
}

// Pack the slot's requests and enqueue their micro-batch (no lock held; the
// requests' inputs do not change while they run).
int launch(abea_server *s, Slot &slot)
{
    const int32_t n = (int32_t)slot.reqs.size();
    slot.seq_off.assign(n + 1, 0);
    slot.ev_off.assign(n + 1, 0);
    slot.pair_off.assign(n + 1, 0);
    slot.sc.resize(n);
    for (int32_t t = 0; t < n; t++) {
        const Request &r = s->table[slot.reqs[t]];
        slot.seq_off[t + 1] = slot.seq_off[t] + (int64_t)r.seq.size();
        slot.ev_off[t + 1] = slot.ev_off[t] + (int64_t)r.ev.size();
        slot.pair_off[t + 1] = slot.pair_off[t] + r.pair_cap;
        slot.sc[t] = r.sc;
    }
    int rc;
    if ((rc = slot.seq.reserve((size_t)slot.seq_off[n])) || (rc = slot.ev.reserve((size_t)slot.ev_off[n])) ||
        (rc = slot.out.reserve((size_t)n)) || (rc = slot.pairs.reserve(2 * (size_t)slot.pair_off[n])))
        return rc;
    for (int32_t t = 0; t < n; t++) {
        const Request &r = s->table[slot.reqs[t]];
        if (!r.seq.empty()) std::memcpy(slot.seq.p + slot.seq_off[t], r.seq.data(), r.seq.size());
        if (!r.ev.empty()) std::memcpy(slot.ev.p + slot.ev_off[t], r.ev.data(), 4 * r.ev.size());
    }
    rc = abea::align_packed_async(slot.ctx, n, s->cfg.W, slot.seq.p, slot.seq_off.data(), slot.ev.p,
                                  slot.ev_off.data(), slot.sc.data(), slot.out.p, slot.pairs.p, slot.pair_off.data());
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)abea::context_stream(slot.ctx);
    if (cudaLaunchHostFunc(st, batch_done, &slot) != cudaSuccess) {
        cudaGetLastError();
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return ABEA_ERR_CUDA;
        }
        batch_done(&slot);
    }
    return ABEA_OK;
}

int free_slots(const abea_server *s)
{
    int f = 0;
    for (const Slot &x : s->slots) f += x.busy ? 0 : 1;
    return f;
}

// The worker.  Short reads (at most short_bases bases) and the others queue
// apart and form their own micro-batches; a queue's micro-batch closes when it
// holds max_batch_reads requests or max_wait_us after its oldest request.
// Short micro-batches go first and may take any free context; the others
// leave one context free for them (unless there is only one), so a short
// request never waits behind a context full of long reads.
void run(abea_server *s)
{
    cudaSetDevice(s->device);
    const std::chrono::microseconds wait(s->cfg.max_wait_us);
    std::unique_lock<std::mutex> lk(s->m);
    for (;;) {
        if (s->fifo[0].empty() && s->fifo[1].empty()) {
            if (s->stopping) break;
            s->cv_work.wait(lk);
            continue;
        }
        const Clock::time_point now = Clock::now();
        Clock::time_point next = Clock::time_point::max();
        int cls = -1;
        for (int c = 0; c < 2 && cls < 0; c++) {
            if (s->fifo[c].empty()) continue;
            const Clock::time_point close_at = s->table[s->fifo[c].front()].t_submit + wait;
            const bool ready = s->stopping || (int32_t)s->fifo[c].size() >= s->cfg.max_batch_reads || now >= close_at;
            const int need = (c == 1 && s->cfg.short_bases >= 0 && (int)s->slots.size() > 1) ? 2 : 1;
            if (ready && free_slots(s) >= need) cls = c;
            else if (!ready) next = std::min(next, close_at);
        }
        if (cls < 0) {                                    // nothing to start: wait for a close time, a request or a context
            if (next == Clock::time_point::max()) s->cv_work.wait(lk);
            else s->cv_work.wait_until(lk, next);
            continue;
        }
        Slot *slot = nullptr;
        for (Slot &x : s->slots)
            if (!x.busy) {
                slot = &x;
                break;
            }
        std::deque<int32_t> &q = s->fifo[cls];
        slot->reqs.clear();
        size_t bytes = 0;
        while (!q.empty() && (int32_t)slot->reqs.size() < s->cfg.max_batch_reads) {
            Request &r = s->table[q.front()];
            if (!slot->reqs.empty() && bytes + r.bytes > s->budget) break;
            bytes += r.bytes;
            r.state = State::Running;
            slot->reqs.push_back(q.front());
            q.pop_front();
        }
        slot->busy = true;
        lk.unlock();
        const int rc = launch(s, *slot);
        lk.lock();
        if (rc != ABEA_OK) {                              // the micro-batch never ran
            for (int32_t idx : slot->reqs) {
                Request &r = s->table[idx];
                r.err = rc;
                r.state = State::Done;
                r.t_done = Clock::now();
            }
            slot->busy = false;
            s->cv_done.notify_all();
        }
    }
    while (!all_free(s)) s->cv_work.wait(lk);
}

void retire(abea_server *s, int32_t idx)
{
    Request &r = s->table[idx];
    r.state = State::Free;
    r.ticket = -1;
    std::vector<char>().swap(r.seq);
    std::vector<float>().swap(r.ev);
    std::vector<int32_t>().swap(r.pairs);
    s->free_idx.push_back(idx);
}

}  // namespace

extern "C" {

int abea_server_start(abea_ctx *ctx, const abea_server_cfg *cfg, abea_server **out)
{
    if (!ctx || !cfg || !out) return ABEA_ERR_ARG;
    *out = nullptr;
    int k = 0;
    const float *mean = nullptr, *stdv = nullptr;
    if (abea::context_model(ctx, &k, &mean, &stdv) != ABEA_OK) return ABEA_ERR_NO_MODEL;
    abea_server_cfg c = *cfg;
    if (c.max_batch_reads == 0) c.max_batch_reads = 256;
    if (c.max_wait_us == 0) c.max_wait_us = 200;
    if (c.batches_in_flight == 0) c.batches_in_flight = 3;
    if (c.max_requests == 0) c.max_requests = 65536;
    if (c.short_bases == 0) c.short_bases = 1000;
    if (c.W < 2 || c.W > 256 || c.max_batch_reads < 1 || c.max_batch_reads > (1 << 20) || c.max_wait_us < 0 ||
        c.batches_in_flight < 1 || c.batches_in_flight > 16 || c.max_requests < 1 || c.max_requests > (1 << 24) ||
        std::isnan(c.block_theta))
        return ABEA_ERR_ARG;
    abea_server *s = new (std::nothrow) abea_server();
    if (!s) return ABEA_ERR_NOMEM;
    s->cfg = c;
    s->device = abea::context_device(ctx);
    s->k = k;
    s->budget = abea::context_budget(ctx) / (size_t)c.batches_in_flight;
    s->table.resize((size_t)c.max_requests);
    s->free_idx.reserve((size_t)c.max_requests);
    for (int32_t i = c.max_requests - 1; i >= 0; i--) s->free_idx.push_back(i);
    s->slots.resize((size_t)c.batches_in_flight);
    int rc = ABEA_OK;
    for (Slot &x : s->slots) {
        x.srv = s;
        if ((rc = abea_create(&x.ctx, s->device, s->budget)) || (rc = abea_set_model(x.ctx, k, mean, stdv)) ||
            (rc = abea_set_block_mode(x.ctx, c.block_theta)))
            break;
        // page-locked staging for typical micro-batches up front: growing it later costs a free of
        // page-locked memory while other micro-batches run
        if ((rc = x.seq.reserve(size_t(4) << 20)) || (rc = x.ev.reserve(size_t(2) << 20)) ||
            (rc = x.out.reserve(4096)) || (rc = x.pairs.reserve(size_t(4) << 20)))
            break;
    }
    if (rc != ABEA_OK) {
        for (Slot &x : s->slots)
            if (x.ctx) abea_destroy(x.ctx);
        delete s;
        return rc;
    }
    try {
        s->worker = std::thread(run, s);
    } catch (...) {
        for (Slot &x : s->slots) abea_destroy(x.ctx);
        delete s;
        return ABEA_ERR_NOMEM;
    }
    *out = s;
    return ABEA_OK;
}

int abea_server_submit(abea_server *s, const abea_read *rd, int64_t *ticket)
{
    if (!s || !rd || !ticket || rd->n_events < 0 || rd->seq_len < 0 || (rd->n_events > 0 && !rd->ev_mean) ||
        (rd->seq_len > 0 && !rd->seq))
        return ABEA_ERR_ARG;
    const int64_t n_k = (int64_t)rd->seq_len - s->k + 1;
    const int64_t cap = std::max<int64_t>((int64_t)rd->n_events + std::max<int64_t>(n_k, 1) - 1, 1);
    const size_t bytes = abea::request_bytes(s->slots[0].ctx, s->cfg.W, rd->n_events, rd->seq_len, cap);
    if (bytes > s->budget) return ABEA_ERR_NOMEM;
    std::vector<char> seq(rd->seq, rd->seq + rd->seq_len);
    std::vector<float> ev(rd->ev_mean, rd->ev_mean + rd->n_events);
    {
        std::lock_guard<std::mutex> lk(s->m);
        if (s->stopping) return ABEA_ERR_ARG;
        if (s->free_idx.empty()) return ABEA_ERR_CAPACITY;
        const int32_t idx = s->free_idx.back();
        s->free_idx.pop_back();
        Request &r = s->table[idx];
        r.ticket = s->serial++ * (int64_t)s->cfg.max_requests + idx;
        r.state = State::Queued;
        r.seq.swap(seq);
        r.ev.swap(ev);
        r.sc = rd->sc;
        r.pair_cap = cap;
        r.bytes = bytes;
        r.err = ABEA_OK;
        r.pairs.clear();
        r.t_submit = Clock::now();
        s->fifo[(s->cfg.short_bases >= 0 && rd->seq_len <= s->cfg.short_bases) ? 0 : 1].push_back(idx);
        *ticket = r.ticket;
    }
    s->cv_work.notify_one();
    return ABEA_OK;
}

int abea_server_poll(abea_server *s, int64_t ticket, int32_t wait_us, abea_result *out, int32_t *pairs, int32_t cap,
                     double *latency_us)
{
    if (!s || !out || ticket < 0 || wait_us < 0 || cap < 0 || (cap > 0 && !pairs)) return ABEA_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->m);
    const int32_t idx = (int32_t)(ticket % s->cfg.max_requests);
    Request &r = s->table[idx];
    if (r.ticket != ticket || r.state == State::Free) return ABEA_ERR_ARG;
    if (r.state != State::Done && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us),
                            [&] { return r.ticket != ticket || r.state == State::Done; });
    if (r.ticket != ticket) return ABEA_ERR_ARG;
    if (r.state != State::Done) return ABEA_ERR_TIMEOUT;
    if (r.err != ABEA_OK) {
        const int err = r.err;
        retire(s, idx);
        return err;
    }
    *out = r.res;
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    const int64_t np = (int64_t)r.pairs.size() / 2;
    if (r.res.status == ABEA_READ_OK && r.res.n_pairs > cap) return ABEA_ERR_CAPACITY;
    if (np > 0) std::memcpy(pairs, r.pairs.data(), 8 * (size_t)np);
    retire(s, idx);
    return ABEA_OK;
}

int abea_server_stop(abea_server *s)
{
    if (!s) return ABEA_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &x : s->slots) {
        abea_destroy(x.ctx);
        x.seq.release();
        x.ev.release();
        x.out.release();
        x.pairs.release();
    }
    delete s;
    return ABEA_OK;
}

}  // extern "C"
