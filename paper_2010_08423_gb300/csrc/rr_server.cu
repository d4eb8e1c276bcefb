// rr_server.cu -- serving loop with continuous batching over a resident graph.
//
// A server owns `slots` execution slots, each a CUDA stream plus the scratch
// of one in-flight query. Its thread admits queued queries in arrival order as
// soon as a slot is free and the device-memory budget holds the query's
// scratch, enqueues the query's layer launches on the slot's stream (so the
// work of queries admitted at different times overlaps on the GPU), and
// retires queries whose completion event has fired. Results are bit-identical
// to rr_reach_sync: every query runs the same kernels on its own scratch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "rr_internal.h"

namespace rr {

using Clock = std::chrono::steady_clock;

struct Ticket {
    rr_query q{};
    std::vector<uint8_t> motif;
    enum State { Queued, Running, Done, Failed, Canceled } state = Queued;
    bool cancel_requested = false;
    rr_status status = RR_OK;
    std::string error;
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<uint64_t> witness;  // filled when Done
    int slot = -1;
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t *h_witness = nullptr;  // pinned, n entries
    uint64_t reserved = 0;          // bytes of budget this slot holds
    uint64_t ticket = 0;
    bool busy = false;
};

struct Server {
    const Graph *g = nullptr;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::deque<Slot> slots;  // deque: slots are never relocated
    std::mutex mu;
    std::condition_variable cv_work;   // server thread wakes on submit / stop
    std::condition_variable cv_done;   // pollers wake on completion
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::shared_ptr<Ticket>> tickets;
    struct Times {
        Clock::time_point submit, admit, done;
    };
    std::map<uint64_t, Times> collected;  // timings of tickets already polled
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    int dev = 0;

    uint64_t need_bytes(uint32_t k, uint64_t share) const
    {
        return query_scratch_bytes(*g, k, share);
    }

    void run();
};

void Server::run()
{
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(mu);
    const uint64_t share = budget / (slots.empty() ? 1 : slots.size());
    while (true) {
        // retire finished slots
        bool any_busy = false;
        for (size_t si = 0; si < slots.size(); ++si) {
            Slot &sl = slots[si];
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            auto it = tickets.find(sl.ticket);
            if (it != tickets.end()) {
                Ticket &t = *it->second;
                t.t_done = Clock::now();
                if (q != cudaSuccess) {
                    t.state = Ticket::Failed;
                    t.status = RR_ECUDA;
                    t.error = std::string("query failed on device: ") + cudaGetErrorString(q);
                } else if (t.cancel_requested) {
                    t.state = Ticket::Canceled;
                    t.status = RR_ECANCELED;
                } else {
                    t.witness.assign(sl.h_witness, sl.h_witness + g->n);
                    t.state = Ticket::Done;
                }
            }
            sl.busy = false;
            used -= sl.reserved;
            sl.reserved = 0;
            cv_done.notify_all();
        }
        // admit queued queries in order while a slot and memory are free
        while (!queue.empty()) {
            uint64_t id = queue.front();
            auto it = tickets.find(id);
            if (it == tickets.end() || it->second->state != Ticket::Queued) {
                queue.pop_front();
                continue;
            }
            Ticket &t = *it->second;
            int free_slot = -1;
            for (size_t si = 0; si < slots.size(); ++si)
                if (!slots[si].busy) { free_slot = (int)si; break; }
            if (free_slot < 0) break;
            uint64_t need = need_bytes(t.q.k, share);
            if (need == UINT64_MAX || used + need > budget) break;
            queue.pop_front();
            Slot &sl = slots[free_slot];
            t.q.motif = t.motif.empty() ? nullptr : t.motif.data();
            t.t_admit = Clock::now();
            t.state = Ticket::Running;
            t.slot = free_slot;
            rr_status st = RR_OK;
            if (sl.ws.S.reserve((size_t)g->n * 8) != cudaSuccess) st = RR_ENOMEM;
            if (st == RR_OK) st = reach_on_stream(*g, sl.ws, &t.q, nullptr, sl.ws.S.as<uint64_t>(),
                                                  share, sl.stream);
            if (st == RR_OK &&
                cudaMemcpyAsync(sl.h_witness, sl.ws.S.p, (size_t)g->n * 8, cudaMemcpyDeviceToHost,
                                sl.stream) != cudaSuccess)
                st = RR_ECUDA;
            if (st == RR_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = RR_ECUDA;
            if (st != RR_OK) {
                t.state = Ticket::Failed;
                t.status = st;
                t.error = rr_last_error();
                t.t_done = Clock::now();
                cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            sl.ticket = id;
            sl.reserved = need;
            used += need;
            any_busy = true;
        }
        if (stop && !any_busy) break;
        if (any_busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        } else {
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        }
    }
}

}  // namespace rr

struct rr_server : public rr::Server {};

using namespace rr;

extern "C" {

rr_status rr_server_create(const rr_graph *g, uint64_t device_mem_budget, uint32_t max_slots,
                           rr_server **out)
{
    clear_error();
    if (!g || !out) return fail(RR_EINVAL, "rr_server_create: NULL argument");
    *out = nullptr;
    std::unique_ptr<rr_server> s(new rr_server());
    s->g = g;
    s->dev = g->dev;
    RR_CUDA(cudaSetDevice(g->dev));
    if (device_mem_budget == 0) {
        size_t free_b = 0, total_b = 0;
        RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
        device_mem_budget = (uint64_t)(0.6 * (double)free_b);
    }
    s->budget = device_mem_budget;
    if (max_slots == 0) max_slots = 4;
    if (max_slots > 64) max_slots = 64;
    s->slots.resize(max_slots);
    // Each slot's scratch is reserved up front for the largest query its share
    // of the budget admits, so that admission never calls cudaMalloc (which
    // would serialise the device and stop queries from overlapping).
    const uint64_t share = s->budget / max_slots;
    uint64_t state_bytes = 0;
    for (uint32_t k = 2; k <= 20; ++k) {
        const uint64_t b = query_scratch_bytes(*g, k, share);
        if (b == UINT64_MAX)
            return fail(RR_ENOMEM, "rr_server_create: budget too small for one point chunk per slot");
        state_bytes = std::max<uint64_t>(state_bytes, b - (uint64_t)g->n * k * 8ull);
    }
    for (auto &sl : s->slots) {
        RR_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        RR_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        RR_CUDA(cudaMallocHost(&sl.h_witness, (size_t)g->n * 8));
        RR_CUDA(sl.ws.state.reserve(state_bytes));
        RR_CUDA(sl.ws.z.reserve((size_t)g->n * 20 * 8));
        RR_CUDA(sl.ws.S.reserve((size_t)g->n * 8));
        RR_CUDA(sl.ws.shade.reserve(sizeof(ShadeTable)));
    }
    s->th = std::thread([p = s.get()] { p->run(); });
    *out = s.release();
    return RR_OK;
}

rr_status rr_server_destroy(rr_server *s)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_server_destroy: NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &kv : s->tickets)
            if (kv.second->state == Ticket::Queued) {
                kv.second->state = Ticket::Canceled;
                kv.second->status = RR_ECANCELED;
            }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->dev);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_witness) cudaFreeHost(sl.h_witness);
    }
    delete s;
    return RR_OK;
}

rr_status rr_query_submit(rr_server *s, const rr_query *q, uint64_t *ticket)
{
    clear_error();
    if (!s || !q || !ticket) return fail(RR_EINVAL, "rr_query_submit: NULL argument");
    rr_status vs = validate_query(*s->g, q);
    if (vs != RR_OK) return vs;
    const uint64_t share = s->budget / s->slots.size();
    if (s->need_bytes(q->k, share) > s->budget || s->need_bytes(q->k, share) == UINT64_MAX)
        return fail(RR_ENOMEM, "rr_query_submit: query can never fit the server's memory budget");
    auto t = std::make_shared<Ticket>();
    t->q = *q;
    if (q->motif) t->motif.assign(q->motif, q->motif + q->k);
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(RR_EINVAL, "rr_query_submit: server is stopping");
        *ticket = s->next_ticket++;
        s->tickets[*ticket] = t;
        s->queue.push_back(*ticket);
    }
    s->cv_work.notify_all();
    return RR_OK;
}

rr_status rr_query_poll(rr_server *s, uint64_t ticket, int32_t timeout_ms, uint8_t *bitmap,
                        uint64_t *witness)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_query_poll: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RR_EINVAL, "rr_query_poll: unknown ticket");
    std::shared_ptr<Ticket> t = it->second;
    auto finished = [&] {
        return t->state == Ticket::Done || t->state == Ticket::Failed ||
               t->state == Ticket::Canceled;
    };
    if (!finished()) {
        if (timeout_ms == 0) return RR_EAGAIN;
        if (timeout_ms < 0) s->cv_done.wait(lk, finished);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
            return RR_EAGAIN;
    }
    s->tickets.erase(ticket);
    s->collected[ticket] = {t->t_submit, t->t_admit, t->t_done};
    if (t->state != Ticket::Done)
        return fail(t->status, t->error.empty() ? "query did not complete" : t->error);
    const uint32_t n = s->g->n;
    if (witness) std::memcpy(witness, t->witness.data(), (size_t)n * 8);
    if (bitmap) {
        std::memset(bitmap, 0, (n + 7) / 8);
        for (uint32_t v = 0; v < n; ++v)
            if (t->witness[v]) bitmap[v >> 3] |= (uint8_t)(1u << (v & 7));
    }
    return RR_OK;
}

rr_status rr_query_cancel(rr_server *s, uint64_t ticket)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_query_cancel: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RR_EINVAL, "rr_query_cancel: unknown ticket");
    Ticket &t = *it->second;
    if (t.state == Ticket::Queued) {
        t.state = Ticket::Canceled;
        t.status = RR_ECANCELED;
        t.t_done = Clock::now();
        s->cv_done.notify_all();
    } else if (t.state == Ticket::Running) {
        t.cancel_requested = true;
    }
    return RR_OK;
}

rr_status rr_query_times(rr_server *s, uint64_t ticket, double *queue_us, double *total_us)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_query_times: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    Server::Times tm;
    auto it = s->tickets.find(ticket);
    if (it != s->tickets.end()) {
        tm = {it->second->t_submit, it->second->t_admit, it->second->t_done};
    } else {
        auto jt = s->collected.find(ticket);
        if (jt == s->collected.end()) return fail(RR_EINVAL, "rr_query_times: unknown ticket");
        tm = jt->second;
    }
    auto us = [](Clock::time_point a, Clock::time_point b) {
        return std::chrono::duration<double, std::micro>(b - a).count();
    };
    const Clock::time_point zero{};
    if (queue_us) *queue_us = tm.admit != zero ? us(tm.submit, tm.admit) : -1.0;
    if (total_us) *total_us = tm.done != zero ? us(tm.submit, tm.done) : -1.0;
    return RR_OK;
}

}  // extern "C"
