// rr_capi.cu -- the extern "C" entry points declared in include/restless_reach.h:
// argument checks, error reporting and dispatch into the rr:: implementation.
#include <cstring>
#include <memory>
#include <string>

#include "rr_internal.h"

namespace rr {

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_timing{false};

namespace {
struct TimingRec {
    cudaEvent_t e0, e1;
    int kind;
};
std::mutex g_tmu;
std::vector<TimingRec> g_tpending;      // slots handed out by timing_begin
std::vector<int> g_tfree;               // recycled slots
double g_tms[kTimeKinds] = {0};
uint64_t g_tcount[kTimeKinds] = {0};
std::vector<int> g_tdone;               // slots whose end event is recorded
}  // namespace

int timing_begin(cudaStream_t st)
{
    if (!g_timing.load(std::memory_order_relaxed)) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    int slot;
    if (!g_tfree.empty()) {
        slot = g_tfree.back();
        g_tfree.pop_back();
    } else {
        TimingRec r{};
        if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess)
            return -1;
        g_tpending.push_back(r);
        slot = (int)g_tpending.size() - 1;
    }
    cudaEventRecord(g_tpending[slot].e0, st);
    return slot;
}

void timing_end(int slot, int kind, cudaStream_t st)
{
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tpending[slot].kind = kind;
    cudaEventRecord(g_tpending[slot].e1, st);
    g_tdone.push_back(slot);
}
static thread_local std::string t_error;

void set_error(const std::string &msg) { t_error = msg; }
void clear_error() { t_error.clear(); }

rr_status fail(rr_status st, const std::string &msg)
{
    t_error = msg;
    return st;
}

rr_status cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    const char *base = std::strrchr(file, '/');
    t_error = std::string(what) + " failed: " + cudaGetErrorString(e) + " (" +
              (base ? base + 1 : file) + ":" + std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();  // allocation failures are not sticky
        return RR_ENOMEM;
    }
    return RR_ECUDA;
}

rr_status graph_load(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                     const uint32_t *t, const uint32_t *delta, const uint8_t *color,
                     uint32_t flags, rr_graph **out);
rr_status debug_point_sums(const Graph &g, const rr_query *q, const uint32_t *masks,
                           uint32_t nmasks, uint64_t *out);
rr_status debug_ztable(const Graph &g, const rr_query *q, uint64_t *out);
rr_status debug_gf_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t count);
rr_status bench_gf_mul(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *d_sink,
                       uint64_t *mults, cudaStream_t st);
rr_status debug_wait_probe(uint64_t timeout_ns, int abort_preset, int32_t *status,
                           uint64_t *elapsed_ns);
rr_status debug_draw(uint64_t key, uint64_t first, uint64_t count, uint64_t *out);
rr_status autotune(Graph &g, uint32_t k, uint32_t *ppl, uint32_t *chunk);
rr_status autotune_batch(Graph &g, const rr_query *qs, uint32_t nq, uint32_t *minb,
                         uint32_t *ranges, uint32_t *max_chunk);
rr_status atmost_device(const Graph &g, uint32_t source, uint32_t k, uint64_t seed,
                        uint8_t *d_bitmap, uint64_t *d_witness, cudaStream_t st);

}  // namespace rr

using namespace rr;

extern "C" {

rr_status rr_graph_load(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                        const uint32_t *t, const uint32_t *delta, const uint8_t *color,
                        uint32_t flags, rr_graph **out)
{
    clear_error();
    try {
        return graph_load(n, m, src, dst, t, delta, color, flags, out);
    } catch (const std::exception &e) {
        return fail(RR_ENOMEM, std::string("rr_graph_load: ") + e.what());
    }
}

rr_status rr_graph_free(rr_graph *g)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_graph_free: NULL graph");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->dev);
    if (g->scratch_ev) {
        cudaEventSynchronize(g->scratch_ev);  // the last call's work, on whatever stream
        cudaEventDestroy(g->scratch_ev);
    }
    if (g->stream) {
        cudaStreamSynchronize(g->stream);
        cudaStreamDestroy(g->stream);
    }
    delete g;
    cudaSetDevice(cur);
    return RR_OK;
}

rr_status rr_graph_get_info(const rr_graph *g, rr_graph_info *out)
{
    clear_error();
    if (!g || !out) return fail(RR_EINVAL, "rr_graph_get_info: NULL argument");
    out->n = g->n;
    out->m = g->m;
    out->state_rows = g->state_rows;
    out->window_rows = g->window_rows;
    out->max_in_degree = g->max_in_degree;
    out->num_items = g->nitems;
    out->device_bytes = g->device_bytes();
    out->has_colors = g->has_colors ? 1 : 0;
    out->compact = g->compact ? 1 : 0;
    out->producer_window_rows = g->state_list.count;
    out->state_compute_rows = g->state_compute_rows;
    out->tail_rows = g->tail_list.count;
    out->deep_compute_rows = g->deep_compute_rows;
    out->deep_tail_rows = g->tail3_list.count;
    out->deep_head_runs = g->deep_head_runs;
    out->pair_layer3_min_k = g->pair_force == 2 ? 6 : (g->pair_force == 1 ? 21 : (int)kPairMinK);
    out->deep_max_range_rows = g->deep_max_item;
    out->deep_heads = g->deep_list.nheads;
    out->head_table = g->head_table_force ? (g->head_table_force == 2 ? 1 : 0)
                                          : (2ull * g->deep_list.nheads <= g->deep_compute_rows ? 1 : 0);
    out->pair_tail = g->pair_tail_off ? 0 : 1;
    return RR_OK;
}

rr_status rr_reach_sync(const rr_graph *g, const rr_query *q, uint8_t *bitmap, uint64_t *witness)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_reach_sync: NULL graph");
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, g->stream);
    const size_t nb = (g->n + 7) / 8;
    RR_CUDA(g->ws.S.reserve((size_t)g->n * 8));
    RR_CUDA(g->ws.bitmap.reserve(nb));
    rr_status s = reach_on_stream(*g, g->ws, q, g->ws.bitmap.as<uint8_t>(),
                                  g->ws.S.as<uint64_t>(), 0, g->stream);
    if (s != RR_OK) return s;
    if (witness)
        RR_CUDA(cudaMemcpyAsync(witness, g->ws.S.p, (size_t)g->n * 8, cudaMemcpyDeviceToHost,
                                g->stream));
    if (bitmap)
        RR_CUDA(cudaMemcpyAsync(bitmap, g->ws.bitmap.p, nb, cudaMemcpyDeviceToHost, g->stream));
    RR_CUDA(cudaStreamSynchronize(g->stream));
    return RR_OK;
}

rr_status rr_reach_device(const rr_graph *g, const rr_query *q, uint8_t *d_bitmap,
                          uint64_t *d_witness, void *stream)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_reach_device: NULL graph");
    if (!d_witness) return fail(RR_EINVAL, "rr_reach_device: d_witness is required");
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return reach_on_stream(*g, g->ws, q, d_bitmap, d_witness, 0, (cudaStream_t)stream);
}

rr_status rr_reach_range_device(const rr_graph *g, const rr_query *q, uint32_t first,
                                uint32_t count, uint64_t *d_witness, void *stream)
{
    clear_error();
    if (!g || !q) return fail(RR_EINVAL, "rr_reach_range_device: NULL graph or query");
    if (!d_witness) return fail(RR_EINVAL, "rr_reach_range_device: d_witness is required");
    rr_status s = validate_query(*g, q);
    if (s != RR_OK) return s;
    const uint64_t npts = 1ull << q->k;
    if (count != 0 && first % kRangeAlign)
        return fail(RR_EINVAL, "rr_reach_range_device: first must be a multiple of " +
                                   std::to_string(kRangeAlign));
    if ((uint64_t)first + count > npts)
        return fail(RR_EINVAL, "rr_reach_range_device: first + count exceeds 2^k = " +
                                   std::to_string(npts));
    if (q->k <= 3 && count != 0 && count != npts)
        return fail(RR_EINVAL, "rr_reach_range_device: k <= 3 sums every point in closed form; "
                               "count must be 0 or 2^k");
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    if (count == 0) {
        RR_CUDA(cudaMemsetAsync(d_witness, 0, (size_t)g->n * 8, (cudaStream_t)stream));
        return RR_OK;
    }
    PointRange range;
    range.first = first;
    range.end = first + count;
    return reach_on_stream(*g, g->ws, q, nullptr, d_witness, 0, (cudaStream_t)stream, nullptr,
                           nullptr, nullptr, range);
}

rr_status rr_reach_batch_device(const rr_graph *g, const rr_query *qs, uint32_t nq,
                                uint8_t *d_bitmaps, uint64_t *d_witness, int32_t *d_status,
                                void *stream)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_reach_batch_device: NULL graph");
    if (nq && (!qs || !d_witness)) return fail(RR_EINVAL, "rr_reach_batch_device: NULL argument");
    for (uint32_t i = 0; i < nq; ++i) {
        rr_status s = validate_query(*g, &qs[i]);
        if (s != RR_OK) return fail(s, "query " + std::to_string(i) + ": " + rr_last_error());
    }
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return batch_device(*g, qs, nq, d_bitmaps, d_witness, d_status, (cudaStream_t)stream);
}

rr_status rr_reach_arrival_device(const rr_graph *g, const rr_query *q, uint64_t *d_witness,
                                  uint64_t *d_edge_sums, uint32_t *d_arrival, uint8_t *d_bitmap,
                                  void *stream)
{
    clear_error();
    if (!g || !q) return fail(RR_EINVAL, "rr_reach_arrival_device: NULL graph or query");
    if (!d_witness || !d_arrival)
        return fail(RR_EINVAL, "rr_reach_arrival_device: d_witness and d_arrival are required");
    rr_status s = validate_query(*g, q);
    if (s != RR_OK) return s;
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return arrival_device(*g, q, d_witness, d_edge_sums, d_arrival, d_bitmap, (cudaStream_t)stream);
}

rr_status rr_reach_sources_device(const rr_graph *g, const uint32_t *sources, uint32_t nsources,
                                  uint32_t k, uint64_t seed, const uint8_t *motif,
                                  const uint8_t *d_separators, uint8_t *d_bitmap, uint64_t *d_witness,
                                  void *stream)
{
    clear_error();
    if (!g || !sources || nsources == 0 || !d_witness)
        return fail(RR_EINVAL, "rr_reach_sources_device: NULL argument or empty source set");
    for (uint32_t i = 0; i < nsources; ++i) {
        const rr_query q{sources[i], k, seed, motif};
        rr_status s = validate_query(*g, &q);
        if (s != RR_OK) return s;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return sources_device(*g, sources, nsources, k, seed, motif, d_separators, d_bitmap, d_witness,
                          (cudaStream_t)stream);
}

rr_status rr_extract_path(const rr_graph *g, const rr_query *q, uint32_t target, uint32_t *vertices,
                          uint32_t *edges, uint32_t *times)
{
    clear_error();
    if (!g || !q || !vertices || !edges || !times)
        return fail(RR_EINVAL, "rr_extract_path: NULL argument");
    rr_status s = validate_query(*g, q);
    if (s != RR_OK) return s;
    if (target >= g->n || target == q->source)
        return fail(RR_EINVAL, "rr_extract_path: target must be a vertex other than the source");
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, g->stream);
    return extract_path(*g, q, target, vertices, edges, times);
}

rr_status rr_reach_bounded_device(const rr_graph *g, uint32_t source, uint32_t k, uint64_t seed,
                                  uint32_t *d_arrival, uint8_t *d_length, uint8_t *d_bitmap,
                                  void *stream)
{
    clear_error();
    if (!g || !d_arrival) return fail(RR_EINVAL, "rr_reach_bounded_device: NULL argument");
    rr_query q{source, k, seed, nullptr};
    rr_status s = validate_query(*g, &q);
    if (s != RR_OK) return s;
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return atmost_arrival_device(*g, source, k, seed, d_arrival, d_length, d_bitmap,
                                 (cudaStream_t)stream);
}

rr_status rr_reach_atmost_device(const rr_graph *g, uint32_t source, uint32_t k, uint64_t seed,
                                 uint8_t *d_bitmap, uint64_t *d_witness, void *stream)
{
    clear_error();
    if (!g || !d_witness) return fail(RR_EINVAL, "rr_reach_atmost_device: NULL argument");
    rr_query q{source, k, seed, nullptr};
    rr_status s = validate_query(*g, &q);
    if (s != RR_OK) return s;
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, (cudaStream_t)stream);
    return atmost_device(*g, source, k, seed, d_bitmap, d_witness, (cudaStream_t)stream);
}

rr_status rr_autotune(rr_graph *g, uint32_t k, uint32_t *best_ppl, uint32_t *best_chunk)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_autotune: NULL graph");
    if (k < 2 || k > 20) return fail(RR_EINVAL, "rr_autotune: k must be in [2, 20]");
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, g->stream);
    return autotune(*g, k, best_ppl, best_chunk);
}

rr_status rr_autotune_batch(rr_graph *g, const rr_query *qs, uint32_t nq, rr_batch_tuning *best)
{
    clear_error();
    if (!g || !qs || nq == 0) return fail(RR_EINVAL, "rr_autotune_batch: NULL graph or no queries");
    for (uint32_t i = 0; i < nq; ++i) {
        rr_status s = validate_query(*g, &qs[i]);
        if (s != RR_OK) return fail(s, "query " + std::to_string(i) + ": " + rr_last_error());
    }
    std::lock_guard<std::mutex> lk(g->mu);
    ScratchOrder order(*g, g->stream);
    uint32_t mb = 0, rg = 0, mc = 0;
    rr_status s = autotune_batch(*g, qs, nq, &mb, &rg, &mc);
    if (s != RR_OK) return s;
    if (best) {
        best->blocks_per_sm = mb;
        best->ranges = rg;
        best->max_chunk = mc;
    }
    return RR_OK;
}

rr_status rr_set_batch_tuning(rr_graph *g, const rr_batch_tuning *t)
{
    clear_error();
    if (!g || !t) return fail(RR_EINVAL, "rr_set_batch_tuning: NULL argument");
    if (t->blocks_per_sm != 0 && t->blocks_per_sm != 2 && t->blocks_per_sm != 4 && t->blocks_per_sm != 5 &&
        t->blocks_per_sm != 6)
        return fail(RR_EINVAL, "rr_set_batch_tuning: blocks_per_sm must be 0, 2, 4, 5 or 6");
    if (t->ranges > 2) return fail(RR_EINVAL, "rr_set_batch_tuning: ranges must be 0, 1 or 2");
    if (t->max_chunk != 0 && t->max_chunk != 128 && t->max_chunk != 256 && t->max_chunk != 512 &&
        t->max_chunk != 1024)
        return fail(RR_EINVAL, "rr_set_batch_tuning: max_chunk must be 0, 128, 256, 512 or 1024");
    std::lock_guard<std::mutex> lk(g->mu);
    g->batch_minb = t->blocks_per_sm;
    g->batch_ranges = t->ranges;
    g->batch_max_chunk = t->max_chunk;
    return RR_OK;
}

rr_status rr_get_batch_tuning(const rr_graph *g, rr_batch_tuning *out)
{
    clear_error();
    if (!g || !out) return fail(RR_EINVAL, "rr_get_batch_tuning: NULL argument");
    std::lock_guard<std::mutex> lk(g->mu);
    out->blocks_per_sm = g->batch_minb;
    out->ranges = g->batch_ranges;
    out->max_chunk = g->batch_max_chunk;
    return RR_OK;
}

rr_status rr_set_tuning(rr_graph *g, uint32_t k, uint32_t ppl, uint32_t chunk)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_set_tuning: NULL graph");
    if (k < 2 || k > 20) return fail(RR_EINVAL, "rr_set_tuning: k must be in [2, 20]");
    if (ppl != 0 && ppl != 2 && ppl != 4) return fail(RR_EINVAL, "rr_set_tuning: ppl must be 0, 2 or 4");
    if (chunk != 0 && (chunk < 64 || chunk > 2048 || (chunk % 64)))
        return fail(RR_EINVAL, "rr_set_tuning: chunk must be 0 or a multiple of 64 in [64, 2048]");
    if (ppl == 4 && chunk != 0 && (chunk % 128))
        return fail(RR_EINVAL, "rr_set_tuning: chunk must be a multiple of 128 with ppl 4");
    std::lock_guard<std::mutex> lk(g->mu);
    g->tune_ppl[k] = ppl;
    g->tune_chunk[k] = chunk;
    g->tune_gen++;
    return RR_OK;
}

rr_status rr_debug_point_sums(const rr_graph *g, const rr_query *q, const uint32_t *masks,
                              uint32_t nmasks, uint64_t *out)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_debug_point_sums: NULL graph");
    return debug_point_sums(*g, q, masks, nmasks, out);
}

rr_status rr_debug_graph(const rr_graph *g, uint32_t *off, uint32_t *row_eid, uint32_t *row_lo,
                         uint32_t *row_hi)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_debug_graph: NULL graph");
    std::lock_guard<std::mutex> lk(g->mu);
    if (off) RR_CUDA(cudaMemcpy(off, g->off.p, (size_t)(g->n + 1) * 4, cudaMemcpyDeviceToHost));
    if (g->m) {
        if (row_eid) RR_CUDA(cudaMemcpy(row_eid, g->row_eid.p, g->m * 4, cudaMemcpyDeviceToHost));
        if (row_lo) RR_CUDA(cudaMemcpy(row_lo, g->row_lo.p, g->m * 4, cudaMemcpyDeviceToHost));
        if (row_hi) RR_CUDA(cudaMemcpy(row_hi, g->row_hi.p, g->m * 4, cudaMemcpyDeviceToHost));
    }
    return RR_OK;
}

rr_status rr_debug_ztable(const rr_graph *g, const rr_query *q, uint64_t *out)
{
    clear_error();
    if (!g || !out) return fail(RR_EINVAL, "rr_debug_ztable: NULL argument");
    return debug_ztable(*g, q, out);
}

rr_status rr_debug_wait_probe(uint64_t timeout_ns, int32_t abort_preset, int32_t *status,
                              uint64_t *elapsed_ns)
{
    clear_error();
    return debug_wait_probe(timeout_ns, abort_preset, status, elapsed_ns);
}

rr_status rr_bench_gf_mul(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *d_sink,
                          uint64_t *mults, void *stream)
{
    clear_error();
    return bench_gf_mul(blocks, threads, iters, d_sink, mults, (cudaStream_t)stream);
}

rr_status rr_debug_gf_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t count)
{
    clear_error();
    return debug_gf_mul(a, b, out, count);
}

rr_status rr_debug_draw(uint64_t key, uint64_t first, uint64_t count, uint64_t *out)
{
    clear_error();
    return debug_draw(key, first, count, out);
}

rr_status rr_timing_enable(int enable)
{
    clear_error();
    g_timing.store(enable != 0);
    return RR_OK;
}

rr_status rr_timing_read(rr_kernel_times *out, int reset)
{
    clear_error();
    std::lock_guard<std::mutex> lk(g_tmu);
    for (int slot : g_tdone) {
        TimingRec &r = g_tpending[slot];
        RR_CUDA(cudaEventSynchronize(r.e1));
        float ms = 0;
        RR_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
        g_tms[r.kind] += ms;
        g_tcount[r.kind] += 1;
        g_tfree.push_back(slot);
    }
    g_tdone.clear();
    if (out)
        for (int i = 0; i < kTimeKinds; ++i) {
            out->ms[i] = g_tms[i];
            out->launches[i] = g_tcount[i];
        }
    if (reset)
        for (int i = 0; i < kTimeKinds; ++i) {
            g_tms[i] = 0;
            g_tcount[i] = 0;
        }
    return RR_OK;
}

const char *rr_last_error(void) { return t_error.c_str(); }

uint64_t rr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
