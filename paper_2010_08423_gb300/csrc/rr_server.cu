// rr_server.cu -- serving loop with continuous batching over a resident graph.
//
// A server owns `slots` execution slots, each a CUDA stream plus the scratch
// of one in-flight query. Its thread admits queued queries in arrival order as
// soon as a slot is free and the device-memory budget holds the query's
// scratch, enqueues the query's layer launches on the slot's stream (so the
// work of queries admitted at different times overlaps on the GPU), and
// retires queries whose completion event has fired. With batching turned on
// (rr_server_set_batching), a backlog of at least min_batch queued queries of
// the reduced-state engine goes instead, up to max_batch at a time, to one of
// two batch lanes, each running the persistent batch kernel over its queries;
// with two lanes the next batch is planned while the current one runs.
// Batching is off by default: the slots' concurrent launch sequences (each
// query a captured CUDA graph of programmatically dependent launches) serve
// faster than the batch kernel both where one query's layers are short
// (n = 1e5, m = 1e6, plain k ~ U{6..12}, a burst of 160 queries: about
// 13,000 queries/s on 4 slots against 9,000 with batches of up to 64) and
// where they fill the GPU (n = 1e7, m = 1e8). Results are bit-identical to
// rr_reach_sync either way.
#include <algorithm>
#include <atomic>
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
    int result = -1;  // index of the result buffer holding witness and bitmap (Done)
    int slot = -1;
};

// Pinned host buffers a query's witness and bitmap are copied into. A slot
// holds one while its query runs; on completion it passes to the ticket (no
// copy) and the slot takes a free one from the pool.
struct ResultBuf {
    uint64_t *w = nullptr;  // n entries
    uint8_t *bm = nullptr;  // ceil(n/8) bytes
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int result = -1;                // result buffer of the running query
    uint64_t reserved = 0;          // bytes of budget this slot holds
    uint64_t ticket = 0;
    bool busy = false;
};

// A batch of admitted queries running on one stream: their witnesses and
// bitmaps land in the lane's device buffers and are then copied into each
// query's own pinned result buffer.
struct BatchLane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf w, bm, status;            // lane_cap witnesses / bitmaps / abort statuses
    int32_t *h_status = nullptr;     // pinned copy of the statuses
    std::vector<uint64_t> tickets;   // the batch's queries, in order
    std::vector<int> results;        // their result buffers
    bool busy = false;
};

constexpr uint32_t kMinBatch = 8;    // lanes exist when both hold at least this many queries
constexpr uint32_t kLaneCap = 256;  // largest batch a lane's buffers hold

struct Server {
    const Graph *g = nullptr;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::deque<Slot> slots;  // deque: slots are never relocated
    BatchLane lanes[2];
    uint32_t lane_cap = 0;   // queries a lane's buffers hold (0: no lanes)
    bool lanes_ready = false;  // lane streams and buffers allocated
    uint32_t min_batch = 0;  // backlog that starts a batch (0: no batching)
    uint32_t max_batch = 0;  // queries per batch
    std::vector<ResultBuf> results;    // all result buffers (index = id)
    std::vector<int> free_results;     // ids of unused ones
    std::atomic<bool> woken{false};    // a query's copies finished (host callback)
    std::mutex mu;
    std::condition_variable cv_work;   // server thread wakes on submit / stop / completion
    std::condition_variable cv_done;   // pollers wake on completion
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::shared_ptr<Ticket>> tickets;
    struct Times {
        Clock::time_point submit, admit, done;
    };
    std::map<uint64_t, Times> collected;  // timings of tickets already polled
    uint64_t next_ticket = 1;
    uint64_t n_single = 0, n_batched = 0, n_batches = 0;
    bool stop = false;
    std::thread th;
    int dev = 0;

    uint64_t need_bytes(uint32_t k, uint64_t share) const
    {
        return query_scratch_bytes(*g, k, share);
    }

    // a free result buffer (a new pinned one when the pool is empty), or -1
    int take_result()
    {
        if (!free_results.empty()) {
            const int id = free_results.back();
            free_results.pop_back();
            return id;
        }
        ResultBuf b;
        if (cudaMallocHost(&b.w, (size_t)g->n * 8) != cudaSuccess) return -1;
        if (cudaMallocHost(&b.bm, ((size_t)g->n + 7) / 8 + 1) != cudaSuccess) {
            cudaFreeHost(b.w);
            return -1;
        }
        results.push_back(b);
        return (int)results.size() - 1;
    }

    rr_status make_lanes();
    bool admit_batch(BatchLane &ln);
    void retire_batch(BatchLane &ln);
    uint32_t batchable_queued() const;
    void run();
};

// Runs on a driver thread once a query's result copies have finished: wakes
// the server thread. It makes no CUDA call and never blocks on the server's
// lock (the server thread makes CUDA calls while holding it); when the lock
// is busy it notifies without it, and the server thread's bounded wait covers
// a wake-up lost in between.
static void CUDART_CB on_query_copied(void *arg)
{
    Server *s = static_cast<Server *>(arg);
    s->woken.store(true);
    std::unique_lock<std::mutex> lk(s->mu, std::try_to_lock);
    s->cv_work.notify_one();
}

// Allocates both lanes' streams and buffers (once).
rr_status Server::make_lanes()
{
    if (lanes_ready) return RR_OK;
    const size_t nb = ((size_t)g->n + 7) / 8;
    for (BatchLane &ln : lanes) {
        if (!ln.stream) RR_CUDA(cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking));
        if (!ln.done) RR_CUDA(cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming));
        RR_CUDA(ln.w.reserve((size_t)lane_cap * g->n * 8));
        RR_CUDA(ln.bm.reserve((size_t)lane_cap * nb));
        RR_CUDA(ln.status.reserve((size_t)lane_cap * 4));
        if (!ln.h_status) RR_CUDA(cudaMallocHost(&ln.h_status, (size_t)lane_cap * 4));
    }
    lanes_ready = true;
    return RR_OK;
}

// Queued queries the batch kernel can take (reduced-state engine), counted
// from the front of the queue up to min_batch.
uint32_t Server::batchable_queued() const
{
    if (!min_batch) return 0;
    uint32_t c = 0;
    for (uint64_t id : queue) {
        auto it = tickets.find(id);
        if (it == tickets.end() || it->second->state != Ticket::Queued) continue;
        if (!uses_v2(*g, it->second->q.k)) break;
        if (++c >= min_batch) break;
    }
    return c;
}

// Admits up to max_batch queued queries, in queue order, to the idle lane
// `ln`. Takes the graph's lock without waiting (the batch kernel uses the
// graph's scratch); returns false, admitting nothing, when it is busy.
bool Server::admit_batch(BatchLane &ln)
{
    std::unique_lock<std::mutex> glk(g->mu, std::try_to_lock);
    if (!glk.owns_lock()) return false;
    std::vector<rr_query> qs;
    ln.tickets.clear();
    ln.results.clear();
    while (!queue.empty() && qs.size() < max_batch) {
        const uint64_t id = queue.front();
        auto it = tickets.find(id);
        if (it == tickets.end() || it->second->state != Ticket::Queued) {
            queue.pop_front();
            continue;
        }
        Ticket &t = *it->second;
        if (!uses_v2(*g, t.q.k)) break;
        const int rb = take_result();
        if (rb < 0) break;
        queue.pop_front();
        t.q.motif = t.motif.empty() ? nullptr : t.motif.data();
        t.t_admit = Clock::now();
        t.state = Ticket::Running;
        t.slot = -1;
        qs.push_back(t.q);
        ln.tickets.push_back(id);
        ln.results.push_back(rb);
    }
    if (qs.empty()) return false;
    const uint32_t nq = (uint32_t)qs.size();
    const size_t nb = ((size_t)g->n + 7) / 8;
    rr_status st;
    {
        ScratchOrder order(*g, ln.stream);
        st = batch_device(*g, qs.data(), nq, ln.bm.as<uint8_t>(), ln.w.as<uint64_t>(),
                          ln.status.as<int32_t>(), ln.stream);
    }
    glk.unlock();
    for (uint32_t i = 0; st == RR_OK && i < nq; ++i) {
        const ResultBuf &rb = results[ln.results[i]];
        if (cudaMemcpyAsync(rb.w, ln.w.as<uint64_t>() + (size_t)i * g->n, (size_t)g->n * 8,
                            cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess ||
            cudaMemcpyAsync(rb.bm, ln.bm.as<uint8_t>() + i * nb, nb, cudaMemcpyDeviceToHost,
                            ln.stream) != cudaSuccess)
            st = RR_ECUDA;
    }
    if (st == RR_OK && cudaMemcpyAsync(ln.h_status, ln.status.p, (size_t)nq * 4,
                                       cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess)
        st = RR_ECUDA;
    if (st == RR_OK && cudaEventRecord(ln.done, ln.stream) != cudaSuccess) st = RR_ECUDA;
    if (st == RR_OK && cudaLaunchHostFunc(ln.stream, on_query_copied, this) != cudaSuccess)
        st = RR_ECUDA;
    if (st != RR_OK) {
        const std::string err = rr_last_error();
        // the lane's stream may still hold work: wait for it before the
        // result buffers go back to the pool
        cudaStreamSynchronize(ln.stream);
        for (uint32_t i = 0; i < nq; ++i) {
            Ticket &t = *tickets[ln.tickets[i]];
            t.state = Ticket::Failed;
            t.status = st;
            t.error = err;
            t.t_done = Clock::now();
            free_results.push_back(ln.results[i]);
        }
        ln.tickets.clear();
        ln.results.clear();
        cv_done.notify_all();
        return true;
    }
    ln.busy = true;
    n_batched += nq;
    ++n_batches;
    return true;
}

// Retires a lane whose completion event has fired (or failed).
void Server::retire_batch(BatchLane &ln)
{
    const cudaError_t q = cudaEventQuery(ln.done);
    for (size_t i = 0; i < ln.tickets.size(); ++i) {
        auto it = tickets.find(ln.tickets[i]);
        bool handed = false;
        if (it != tickets.end()) {
            Ticket &t = *it->second;
            t.t_done = Clock::now();
            if (q != cudaSuccess) {
                t.state = Ticket::Failed;
                t.status = RR_ECUDA;
                t.error = std::string("batched query failed on device: ") + cudaGetErrorString(q);
            } else if (ln.h_status[i] != 0) {
                t.state = Ticket::Failed;
                t.status = RR_ECUDA;
                t.error = "batched query aborted: a bounded wait of the batch kernel expired";
            } else if (t.cancel_requested) {
                t.state = Ticket::Canceled;
                t.status = RR_ECANCELED;
            } else {
                t.result = ln.results[i];
                t.state = Ticket::Done;
                handed = true;
            }
        }
        if (!handed) free_results.push_back(ln.results[i]);
    }
    ln.tickets.clear();
    ln.results.clear();
    ln.busy = false;
    cv_done.notify_all();
}

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
                    t.result = sl.result;  // hand the pinned buffers over
                    sl.result = -1;
                    t.state = Ticket::Done;
                }
            }
            if (sl.result >= 0) {  // failed or cancelled: buffers back to the pool
                free_results.push_back(sl.result);
                sl.result = -1;
            }
            sl.busy = false;
            used -= sl.reserved;
            sl.reserved = 0;
            cv_done.notify_all();
        }
        for (BatchLane &ln : lanes) {
            if (!ln.busy) continue;
            if (cudaEventQuery(ln.done) == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            retire_batch(ln);
        }
        // under a backlog, queued queries go to an idle batch lane first
        for (BatchLane &ln : lanes) {
            if (ln.busy || !min_batch || batchable_queued() < min_batch) continue;
            if (!admit_batch(ln)) break;
            any_busy = any_busy || ln.busy;
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
            const size_t nb = ((size_t)g->n + 7) / 8;
            if (sl.result < 0) sl.result = take_result();
            if (sl.result < 0) st = RR_ENOMEM;
            if (st == RR_OK && (sl.ws.S.reserve((size_t)g->n * 8) != cudaSuccess ||
                                sl.ws.bitmap.reserve(nb) != cudaSuccess))
                st = RR_ENOMEM;
            if (st == RR_OK)
                st = reach_on_stream(*g, sl.ws, &t.q, sl.ws.bitmap.as<uint8_t>(), sl.ws.S.as<uint64_t>(),
                                     share, sl.stream);
            if (st == RR_OK) {
                const ResultBuf &rb = results[sl.result];
                if (cudaMemcpyAsync(rb.w, sl.ws.S.p, (size_t)g->n * 8, cudaMemcpyDeviceToHost,
                                    sl.stream) != cudaSuccess ||
                    cudaMemcpyAsync(rb.bm, sl.ws.bitmap.p, nb, cudaMemcpyDeviceToHost, sl.stream) !=
                        cudaSuccess)
                    st = RR_ECUDA;
            }
            if (st == RR_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = RR_ECUDA;
            if (st == RR_OK && cudaLaunchHostFunc(sl.stream, on_query_copied, this) != cudaSuccess)
                st = RR_ECUDA;
            if (st != RR_OK) {
                t.state = Ticket::Failed;
                t.status = st;
                t.error = rr_last_error();
                t.t_done = Clock::now();
                cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            ++n_single;
            sl.ticket = id;
            sl.reserved = need;
            used += need;
            any_busy = true;
        }
        if (stop && !any_busy) break;
        // sleep until a query's copies finish (host callback), a query
        // arrives while a slot is free, or the server stops; the 2 ms bound
        // only guards against a missed wake-up
        auto can_admit = [&] {
            if (queue.empty()) return false;
            for (const Slot &sl : slots)
                if (!sl.busy) return true;
            for (const BatchLane &ln : lanes)
                if (!ln.busy && min_batch && batchable_queued() >= min_batch) return true;
            return false;
        };
        cv_work.wait_for(lk, std::chrono::milliseconds(2),
                         [&] { return stop || woken.load() || can_admit(); });
        woken.store(false);
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
        sl.result = s->take_result();
        if (sl.result < 0) return fail(RR_ENOMEM, "rr_server_create: pinned result buffers");
        RR_CUDA(sl.ws.state.reserve(state_bytes));
        RR_CUDA(sl.ws.bitmap.reserve(((size_t)g->n + 7) / 8));
        RR_CUDA(sl.ws.z.reserve((size_t)g->n * 20 * 8));
        RR_CUDA(sl.ws.S.reserve((size_t)g->n * 8));
        RR_CUDA(sl.ws.shade.reserve(sizeof(ShadeTable)));
    }
    // one spare result buffer per slot: completed queries keep theirs until
    // polled, and serving allocates only when more than that are waiting
    std::vector<int> spares;
    for (size_t i = 0; i < s->slots.size(); ++i) {
        const int id = s->take_result();
        if (id < 0) return fail(RR_ENOMEM, "rr_server_create: pinned result buffers");
        spares.push_back(id);
    }
    s->free_results = spares;
    // batch lanes (allocated when rr_server_set_batching turns batching on),
    // when the graph runs the reduced-state engine and a quarter of the budget
    // holds two lanes' outputs for at least kMinBatch queries
    const uint64_t per_query = (uint64_t)g->n * 8 + ((uint64_t)g->n + 7) / 8;
    const uint64_t fit = s->budget / 4 / (2 * per_query);
    if (uses_v2(*g, 2) && fit >= kMinBatch) s->lane_cap = (uint32_t)std::min<uint64_t>(kLaneCap, fit);
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
    }
    for (BatchLane &ln : s->lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.h_status) cudaFreeHost(ln.h_status);
    }
    for (ResultBuf &b : s->results) {
        if (b.w) cudaFreeHost(b.w);
        if (b.bm) cudaFreeHost(b.bm);
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
    // the ticket owns its result buffer now: copy out without holding the lock
    const ResultBuf rb = s->results[t->result];
    lk.unlock();
    const uint32_t n = s->g->n;
    if (witness) std::memcpy(witness, rb.w, (size_t)n * 8);
    if (bitmap) std::memcpy(bitmap, rb.bm, ((size_t)n + 7) / 8);
    lk.lock();
    s->free_results.push_back(t->result);
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

rr_status rr_server_stats(rr_server *s, uint64_t *single, uint64_t *batched, uint64_t *batches)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_server_stats: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (single) *single = s->n_single;
    if (batched) *batched = s->n_batched;
    if (batches) *batches = s->n_batches;
    return RR_OK;
}

rr_status rr_server_set_batching(rr_server *s, uint32_t min_batch, uint32_t max_batch)
{
    clear_error();
    if (!s) return fail(RR_EINVAL, "rr_server_set_batching: NULL server");
    if (min_batch && (max_batch < min_batch || min_batch < 2))
        return fail(RR_EINVAL, "rr_server_set_batching: need 2 <= min_batch <= max_batch");
    std::lock_guard<std::mutex> lk(s->mu);
    if (min_batch && !s->lane_cap)
        return fail(RR_EINVAL, "rr_server_set_batching: this server has no batch lanes");
    if (min_batch && max_batch > s->lane_cap)
        return fail(RR_EINVAL, "rr_server_set_batching: max_batch above the lanes' capacity");
    if (min_batch) {
        rr_status ls = s->make_lanes();
        if (ls != RR_OK) return ls;
    }
    s->min_batch = min_batch;
    s->max_batch = min_batch ? max_batch : 0;
    s->cv_work.notify_all();
    return RR_OK;
}

}  // extern "C"
