// rr_internal.h -- library-internal structures shared by the .cu/.cpp files.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/restless_reach.h"

namespace rr {

// -------- errors -----------------------------------------------------------
void set_error(const std::string &msg);
void clear_error();
rr_status fail(rr_status st, const std::string &msg);
rr_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
extern std::atomic<uint64_t> g_launches;

// Kernel timing (rr_timing_*): kinds as in rr_kernel_times.
enum TimingKind {
    kTimeFirst = 0, kTimeMid = 1, kTimeLast = 2, kTimeZ = 3, kTimeBatch = 4, kTimeSecond = 5,
    kTimeTail = 6, kTimeThird = 7, kTimeLabelTail = 8, kTimeKinds = 9
};
extern std::atomic<bool> g_timing;
// Records a start event on st when timing is enabled; returns an opaque slot.
int timing_begin(cudaStream_t st);
void timing_end(int slot, int kind, cudaStream_t st);

#define RR_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return ::rr::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define RR_LAUNCHED()                                                        \
    do {                                                                     \
        ::rr::g_launches.fetch_add(1, std::memory_order_relaxed);            \
        cudaError_t _e = cudaGetLastError();                                 \
        if (_e != cudaSuccess) return ::rr::cuda_fail(_e, "kernel launch", __FILE__, __LINE__); \
    } while (0)

// -------- device buffer ----------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // Grows to at least `want` bytes (contents are not preserved).
    cudaError_t reserve(size_t want)
    {
        if (want <= bytes && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, want ? want : 16);
        if (e == cudaSuccess) bytes = want ? want : 16;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Per-query values the reduced-state engine's kernels read from device
// memory, so that one captured launch sequence serves every query of a shape.
struct QueryDesc {
    uint32_t source, k, colored, pad;
    uint64_t key_y, key_z, key_g, key_o;
    uint64_t *S;        // witness output (n)
    uint8_t *bitmap;    // bitmap output or null
    uint64_t *E;        // per-edge last-layer sums (m, by input edge index) or null
    const uint8_t *vmask;  // deleted vertices (n flags: z rows are zero) or null
    uint32_t shades[512];  // first shade [0..255], multiplicity [256..511]
};

// Scratch of one in-flight query: double-buffered prefix state, z-table,
// witness sums, shade table and bitmap, plus the query descriptor and the
// cache of captured launch sequences (CUDA graphs) keyed by query shape.
struct Workspace {
    DevBuf state;   // engine scratch
    DevBuf z;       // n * k * 8
    DevBuf S;       // n * 8
    DevBuf shade;   // 512 uint32
    DevBuf bitmap;  // ceil(n/8)
    DevBuf desc;    // QueryDesc
    DevBuf edges;   // m * 8: per-edge sums (fine-grained output) when the caller gives none
    DevBuf arrival; // n * 4: minimum arrival times (path extraction)
    DevBuf vmask;   // n: deleted vertices (path extraction)
    DevBuf pick;    // 8: the extraction step's choice
    DevBuf srcmask; // n: a set of sources (rr_reach_sources_device)
    DevBuf bS, bE, bR;  // at-most-k branches' witnesses (n), per-edge sums (m), arrivals (n)
    cudaStream_t capture = nullptr;           // stream used only to capture graphs
    // captured launch sequences keyed by (query shape, sieve-point range)
    std::vector<std::pair<std::pair<uint64_t, uint64_t>, cudaGraphExec_t>> graphs;
    std::vector<uint64_t> graph_kernels;      // kernel nodes per cached graph
    void *graph_state = nullptr;              // state.p the graphs were captured with
    void *graph_z = nullptr;
    // pinned staging ring for query descriptors: slot i may be rewritten once
    // ring_ev[i] (recorded after the launch that consumed it) has completed
    static constexpr int kRing = 64;
    QueryDesc *h_ring = nullptr;
    // at-most-k branches (reach_v2's bfirst): their descriptors, staged per
    // ring slot (kMaxBranches each) and uploaded to bdesc
    static constexpr uint32_t kMaxBranches = 16;
    QueryDesc *h_bring = nullptr;
    DevBuf bdesc;
    cudaStream_t side = nullptr;  // the branches' stream
    cudaEvent_t bev[4] = {};
    cudaEvent_t ring_ev[kRing] = {};
    bool ring_used[kRing] = {};
    uint32_t ring_pos = 0;
    // launch the query's kernels with programmatic dependent launch (off for
    // workspaces whose queries run concurrently with others)
    bool pdl = true;
    // shape chosen per k (0 = not chosen yet) and the tuning generation it used
    uint32_t shape_ppl[32] = {0}, shape_chunk[32] = {0};
    uint64_t shape_gen[32] = {0};
    size_t bytes() const
    {
        return state.bytes + z.bytes + S.bytes + shade.bytes + bitmap.bytes + desc.bytes + edges.bytes +
               arrival.bytes + vmask.bytes + pick.bytes + srcmask.bytes + bS.bytes + bE.bytes + bR.bytes;
    }
    void drop_graphs()
    {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
        graph_kernels.clear();
    }
    ~Workspace()
    {
        drop_graphs();
        if (capture) cudaStreamDestroy(capture);
        for (int i = 0; i < kRing; ++i)
            if (ring_ev[i]) cudaEventDestroy(ring_ev[i]);
        if (h_ring) cudaFreeHost(h_ring);
        if (h_bring) cudaFreeHost(h_bring);
        if (side) cudaStreamDestroy(side);
        for (cudaEvent_t e : bev)
            if (e) cudaEventDestroy(e);
    }
};

// A list of CSR rows (a subsequence of the in-edge CSR, so still sorted by
// head vertex, then time), with the per-entry fields some layer needs and
// head-aligned scheduling ranges [entry_begin, entry_end).
struct RowList {
    uint64_t count = 0;
    DevBuf head, eid, src;  // uint32 per entry
    DevBuf a0, b0;          // window in producer-prefix indices (scalar first-layer prefix)
    DevBuf a1, b1;          // window in state-row indices (state rows = producers with a window)
    DevBuf a3, b3;          // window in deep-row indices (deep rows = state rows whose window
                            // holds a state row: the only rows non-zero at layers >= 3)
    DevBuf items;           // uint2 ranges, largest first (fine: one-query kernels)
    uint32_t nitems = 0;
    DevBuf items_coarse;    // uint2 ranges of about 32 entries (persistent batch)
    uint32_t nitems_coarse = 0;
    // Head segments longer than kMaxRun entries are cut into pieces of kMaxRun
    // that run in parallel, each computing a prefix from zero; `chains` lists
    // every cut segment as (first entry, end entry) so that a fix-up pass can
    // XOR the running carry into the later pieces.
    static constexpr uint32_t kMaxRun = 128;
    DevBuf chains;          // uint2 (begin, end) of every cut segment
    uint32_t nchains = 0;
    DevBuf fix2;            // uint2 (chain, first row slot) of every phase-2 fix-up task
    uint32_t nfix2 = 0;
    // deep list only, for the one-query kernels' per-point state: instead of
    // fixing the later pieces' rows in place, the fix-up stores the carry into
    // every piece after the first (one row of a carry table per piece, slot 0
    // a zero row) and readers add the carries of both window ends. row_carry
    // (count + 1 entries, by state row) = the carry slot of the row's piece;
    // chain_slot0 (per chain) = the slot of its second piece.
    DevBuf row_carry, chain_slot0;
    uint32_t ncarry = 1;    // carry slots including the zero slot
    // deep list only: the distinct heads of its rows (in row order) and, per
    // entry, the rank there of its tail u (the head of the rows its window
    // covers; UINT32_MAX when u heads none)
    DevBuf heads, trank;
    uint32_t nheads = 0;
    size_t bytes() const
    {
        return head.bytes + eid.bytes + src.bytes + a0.bytes + b0.bytes + a1.bytes + b1.bytes +
               a3.bytes + b3.bytes + items.bytes + items_coarse.bytes + chains.bytes + fix2.bytes +
               heads.bytes + trank.bytes + row_carry.bytes + chain_slot0.bytes;
    }
};

// Device buffers of the persistent batched launch, kept per graph, and a
// pinned staging area for the batch plan (reused once the event recorded
// after its last upload has completed, so uploads never wait on the stream).
struct BatchBuffers {
    DevBuf units, segs, descs, zoff, pyoff, z, py, slots, done, ctl, status, task_seg, pr2, pr2off;
    char *h_stage = nullptr;
    size_t h_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    bool stage_pending = false;
    // occupancy of the persistent kernel's variants (index: the blocks per SM
    // its register budget is set for; 0 = not queried yet)
    int occupancy[8] = {0};
    int sms = 0;
    ~BatchBuffers()
    {
        if (stage_ev) cudaEventDestroy(stage_ev);
        if (h_stage) cudaFreeHost(h_stage);
    }
};

// Lanes for single queries that run concurrently (the k' = 2..k queries of
// at-most-k): a workspace and a stream per lane, forked from and joined back
// to the caller's stream with events.
struct FanOut {
    std::vector<std::unique_ptr<Workspace>> ws;
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    size_t bytes() const
    {
        size_t b = 0;
        for (const auto &w : ws) b += w->bytes();
        return b;
    }
    ~FanOut()
    {
        for (cudaStream_t s : st) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        for (cudaEvent_t e : done) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
};

// -------- graph ------------------------------------------------------------
// In-edge CSR: rows sorted by (head v, time, input edge index). Vertex v owns
// rows [off[v], off[v+1]).
//
// Windowed prefix state: for a point chunk, state row 0 is all zero and each
// "producer" row r (a row inside the restless window of some edge) owns state
// row row_s[r] >= 1 holding the XOR of its own and the earlier producer rows'
// layer values within its head's segment. A consumer row e reads its window
// sum as state[row_a[e]] ^ state[row_b[e]] (row_a == 0 <=> empty window).
// Smallest k whose layer 3 runs in pair-label space unless the graph's load
// flags choose (rr_sieve2.cu): from k = 9 it was faster on every graph
// measured (uniform n = 1e5 and Chung-Lu n = 2e5, 1e6), at k = 8 level or slower.
constexpr uint32_t kPairMinK = 9;
// Deep-row ranges of at most this many rows build the pair rows in one launch.
constexpr uint32_t kPairFusedMaxRows = 4;

struct Graph {
    uint32_t n = 0;
    uint64_t m = 0;
    int dev = 0;
    bool has_colors = false;
    bool compact = true;
    uint64_t state_rows = 1;   // 1 + producers
    uint64_t window_rows = 0;  // rows with a non-empty window
    uint64_t producer_window_rows = 0;  // producer rows with a non-empty window
    uint64_t state_compute_rows = 0;    // state rows whose window holds a state row
    uint64_t deep_compute_rows = 0;     // deep rows whose window holds a deep row
    uint64_t deep_head_runs = 0;        // head runs over the deep list's fine ranges
    uint32_t deep_max_item = 0;         // rows of the deep list's longest fine range
    // layer 3 in pair-label space (6 <= k <= 20): 0 = by k (k >= kPairMinK),
    // 1 = forced off, 2 = forced on (load flags)
    uint32_t pair_force = 0;
    // layer 4 of the pair form takes x_u x_s from a per-chunk table of the
    // deep rows' heads (0 = when heads <= compute rows / 2, 1 = never, 2 = always)
    uint32_t head_table_force = 0;
    // layers k-2 and k-1 from the pair sums of layer k-3 (label-space layer
    // k-2) unless the load flags turn it off
    bool pair_tail_off = false;
    // k = 4 per point (layer 2 over the sieve points) instead of the closed
    // form over the label-space layer 2 (load flags)
    bool k4_per_point = false;
    // k = 5 in closed form over the pair-label layer 3 instead of per point
    // (load flags; per point is faster on the measured graphs, the closed form
    // there as an exact alternative)
    bool k5_closed = false;
    // at-most-k: k' >= the first branch from the k query's layers (2), every
    // k' on its own lane (1), or by the k query's per-point work (0; load flags)
    uint32_t atmost_branches = 0;
    uint32_t max_in_degree = 0;

    DevBuf off;      // n+1 uint32
    DevBuf row_a;    // m uint32
    DevBuf row_b;    // m uint32
    DevBuf row_s;    // m uint32
    DevBuf row_eid;  // m uint32
    DevBuf row_src;  // m uint32
    DevBuf row_lo;   // m uint32 (debug / tests)
    DevBuf row_hi;   // m uint32
    DevBuf row_t;    // m uint32: time of the row's edge
    DevBuf row_head; // m uint32: head v of the row (the row lies in v's segment)
    DevBuf color;    // n uint8 (if coloured)
    // n uint32 (if coloured): the vertices by colour, ascending (stable), so
    // that the threads of a warp that build a motif query's z-table share one
    // shade count
    DevBuf color_order;
    DevBuf items;    // uint2 (v0, v1) vertex ranges, largest first
    uint32_t nitems = 0;
    std::vector<uint32_t> h_item_rows;  // rows per item (host copy, same order)

    // Row lists of the reduced-state engine (see rr_sieve2.cu):
    //   prod_list  rows inside some window (first-layer scalar prefix)
    //   state_list producers whose own window is non-empty (state rows)
    //   win_list   rows with a non-empty window (k = 3 last layer)
    //   tail_list  rows whose window holds at least one state row (last layer, k = 4)
    //   deep_list  state rows whose window holds a state row (layers >= 3)
    //   tail3_list rows whose window holds a deep row (last layer, k >= 5)
    RowList prod_list, state_list, win_list, tail_list, deep_list, tail3_list;

    // per-graph scratch for rr_reach_device / rr_reach_sync (serialised by mu)
    mutable std::mutex mu;
    mutable Workspace ws;
    mutable BatchBuffers batch;
    mutable FanOut fan;
    // device-side order of calls that use the scratch above: each such call's
    // stream waits for this event (recorded after the previous call's last
    // work), so calls issued on different streams never overlap on it
    mutable cudaEvent_t scratch_ev = nullptr;
    mutable bool scratch_pending = false;
    mutable cudaStream_t stream = nullptr;

    // tuning per k (index k): 0 = automatic; tune_gen changes on every update
    uint32_t tune_ppl[32] = {0};
    uint32_t tune_chunk[32] = {0};
    uint64_t tune_gen = 1;
    // shape of the persistent batch (rr_autotune_batch / rr_set_batch_tuning;
    // 0 = the automatic rule): kernel variant by blocks per SM (2, 4 or 6),
    // scheduling ranges (1 fine, 2 coarse) and the largest point chunk
    uint32_t batch_minb = 0, batch_ranges = 0, batch_max_chunk = 0;

    size_t device_bytes() const
    {
        return off.bytes + row_a.bytes + row_b.bytes + row_s.bytes + row_eid.bytes +
               row_src.bytes + row_lo.bytes + row_hi.bytes + row_t.bytes + row_head.bytes +
               color.bytes + color_order.bytes + items.bytes +
               prod_list.bytes() + state_list.bytes() + win_list.bytes() + tail_list.bytes() +
               deep_list.bytes() + tail3_list.bytes();
    }
};

// -------- query plan -------------------------------------------------------
// Sieve points [first, end) of a query (end == 0: all 2^k points). The
// per-vertex sums are XOR-linear in the points (Eq. (2) sums over L), so the
// sums of disjoint ranges XOR to the full query's. first is a multiple of
// kRangeAlign (every lane group of the kernels starts on such a multiple).
constexpr uint32_t kRangeAlign = 128;
struct PointRange {
    uint32_t first = 0, end = 0;
    bool full(uint32_t k) const { return first == 0 && (end == 0 || end == (1u << k)); }
    uint32_t stop(uint32_t k) const { return end ? end : (1u << k); }
};

struct QueryKeys {
    uint64_t key_y, key_z, key_gamma, key_omega;
};

// Shade layout of a motif: first shade and multiplicity per colour.
struct ShadeTable {
    uint32_t first[256];
    uint32_t mu[256];
};

rr_status validate_query(const Graph &g, const rr_query *q);
QueryKeys make_keys(uint64_t seed);
void make_shades(const uint8_t *motif, uint32_t k, ShadeTable *out);

// Chooses points-per-lane and points-per-chunk for a query of size k such that
// the double-buffered state (2 * state_rows * chunk * 8 bytes) fits budget.
// Returns false if even the smallest chunk does not fit.
bool choose_shape(const Graph &g, uint32_t k, uint64_t budget, uint32_t *ppl, uint32_t *chunk);
// The same with the (ppl, chunk) preference given explicitly (0 = automatic)
// instead of read from the graph's tuning; shape_ppl is the points per lane it
// uses (the smallest chunk is 32 * that many points).
bool choose_shape_tuned(const Graph &g, uint32_t k, uint64_t budget, uint32_t tune_ppl,
                        uint32_t tune_chunk, uint32_t *ppl, uint32_t *chunk);
uint32_t shape_ppl(uint32_t k, uint32_t tune_ppl);

// -------- kernels (rr_sieve.cu) --------------------------------------------
struct LayerParams;
rr_status launch_ztable(const Graph &g, uint32_t k, const QueryKeys &keys, bool colored,
                        const uint32_t *d_shades /* 512 or null */, uint64_t *d_z,
                        cudaStream_t st, const uint8_t *d_vmask = nullptr);
rr_status launch_bitmap(const uint64_t *d_S, uint32_t n, uint8_t *d_bitmap, cudaStream_t st);

// Runs all chunks and layers of one query; d_S must be zeroed by the caller
// unless debug masks are given (then d_out = nmasks*n, zeroed by the caller).
// d_E (m, zeroed by the caller, or null) gets the per-edge sums of the last layer.
rr_status run_query_layers(const Graph &g, const rr_query *q, const uint64_t *d_z,
                           uint64_t *d_state, uint32_t ppl, uint32_t chunk, uint64_t *d_S,
                           const uint32_t *d_masks, uint32_t nmasks, uint64_t *d_debug_out,
                           cudaStream_t st, uint64_t *d_E = nullptr,
                           const uint8_t *d_srcmask = nullptr, PointRange range = PointRange());
// Runs one query on `st` with scratch `ws`; d_witness (n) required. `budget`
// bounds the state buffers (0 = 60% of free device memory). d_E (m, zeroed by
// the caller, or null) gets for every input edge the sum over all sieve points
// of its last-layer value.
// d_vmask (n flags, device, or null) deletes vertices: their z rows are zero,
// so no walk through them contributes. d_srcmask (n flags, device, or null)
// starts walks at every flagged vertex instead of q->source.
// range: the sieve points to sum (default all; a part needs k >= 4 and gives
// no bitmap).
// bfirst / b_witness / b_edges: at-most-k branches as in reach_v2 (the
// reduced-state engine only; RR_EINVAL otherwise).
rr_status reach_on_stream(const Graph &g, Workspace &ws, const rr_query *q, uint8_t *d_bitmap,
                          uint64_t *d_witness, uint64_t budget, cudaStream_t st,
                          uint64_t *d_E = nullptr, const uint8_t *d_vmask = nullptr,
                          const uint8_t *d_srcmask = nullptr, PointRange range = PointRange(),
                          uint32_t bfirst = 0, uint64_t *b_witness = nullptr,
                          uint64_t *b_edges = nullptr);
// Bytes of scratch one query of size k needs with the shape chosen for budget.
uint64_t query_scratch_bytes(const Graph &g, uint32_t k, uint64_t budget);

// Reduced-state engine (rr_sieve2.cu), used for k >= 3 on compact graphs.
bool uses_v2(const Graph &g, uint32_t k);
// Queries qs[0..nq) through the persistent batch kernel (rr_batch.cu);
// query i's witness at d_witness + i*n, bitmap at d_bitmaps + i*ceil(n/8),
// abort status at d_status[i]. Uses the graph's scratch: hold its lock.
rr_status batch_device(const Graph &g, const rr_query *qs, uint32_t nq, uint8_t *d_bitmaps,
                       uint64_t *d_witness, int32_t *d_status, cudaStream_t st);
bool choose_shape_v2(const Graph &g, uint32_t k, uint64_t budget, uint32_t *ppl, uint32_t *chunk);
uint32_t v2_reduced_stride(uint32_t ppl, uint32_t chunk);
uint64_t v2_scratch_bytes(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k,
                          bool branches = false);
// Enqueues the whole launch sequence of one k >= 3 query (z-table, witness
// clear, all layers, bitmap) reading per-query values from d_desc; returns
// the number of kernels enqueued in *kernels.
// table: z is read from a z-table built from the descriptor (motif queries and
// queries with deleted vertices); otherwise plain z is drawn on the fly.
// At-most-k branches (bfirst > 0, plain queries): the k'-vertex queries for
// k' = bfirst..k-1 are taken from this query's layers -- for the same seed their
// per-point states equal this query's on their first 2^k' points -- so after
// its per-point layer k'-2 the query also writes k''s transformed state and
// runs k''s last layer with descriptor d_bdesc[k' - bfirst]. bfirst must be at
// least atmost_first_branch(g, k); with the pair-label layer 3, branch 5 is the
// closed form over this query's pair rows. With the pair tail, branch k-1 is k-1's
// last layer alone, over the single-label slots of layer k-3's pair sums (the
// pair tail stays off where a point group would straddle 2^(k-1)).
// side (or null: st) runs the branches beside the query, bev[0..3] (four
// events) ordering them: each branch starts after its layer, the query waits
// for the branch's transform after its next layer, before the next chunk's
// pair sums for branch k-1, and for all branches at its end.
rr_status enqueue_query_v2(const Graph &g, uint32_t k, bool table, bool bitmap, uint32_t ppl,
                           uint32_t chunk, uint64_t *d_z, uint64_t *d_scratch,
                           const QueryDesc *d_desc, cudaStream_t st, uint64_t *kernels,
                           bool pdl = true, PointRange range = PointRange(),
                           const QueryDesc *d_bdesc = nullptr, uint32_t bfirst = 0,
                           cudaStream_t side = nullptr, cudaEvent_t *bev = nullptr);
// b_witness / b_edges: witness (n values) and per-edge sums (m values, or
// null) of branch k' at offset (k' - bfirst) rows; the branches' witness rows
// must be zero before the call.
rr_status reach_v2(const Graph &g, Workspace &ws, const rr_query *q, uint8_t *d_bitmap,
                   uint64_t *d_witness, uint32_t ppl, uint32_t chunk, cudaStream_t st,
                   uint64_t *d_E = nullptr, const uint8_t *d_vmask = nullptr,
                   PointRange range = PointRange(), uint32_t bfirst = 0,
                   uint64_t *b_witness = nullptr, uint64_t *b_edges = nullptr);
// Smallest k' an at-most-k query of size k can take from its own layers (the
// first per-point layer + 2), or 0 when none.
uint32_t atmost_first_branch(const Graph &g, uint32_t k);
// The first branch at-most-k takes from the k query (0: every k' on its own
// lane): the load flags' choice, else atmost_first_branch where the k query's
// per-point layers are long.
uint32_t atmost_branches(const Graph &g, uint32_t k);

// Held (under the graph's lock) by every call that uses the graph's scratch:
// the call's stream first waits for the previous such call's work, and the
// call's own last work is marked for the next one.
struct ScratchOrder {
    const Graph &g;
    cudaStream_t st;
    ScratchOrder(const Graph &g_, cudaStream_t st_) : g(g_), st(st_)
    {
        if (g.scratch_pending) cudaStreamWaitEvent(st, g.scratch_ev, 0);
    }
    ~ScratchOrder()
    {
        if (!g.scratch_ev && cudaEventCreateWithFlags(&g.scratch_ev, cudaEventDisableTiming) != cudaSuccess) {
            g.scratch_ev = nullptr;
            return;
        }
        g.scratch_pending = cudaEventRecord(g.scratch_ev, st) == cudaSuccess;
    }
};

// Fine-grained outputs (rr_fine.cu): the query with per-edge sums d_E (m, or
// null for the workspace's buffer), minimum arrival times d_R (n) and the set
// D as a bitmap (or null); d_vmask deletes vertices.
rr_status arrival_device(const Graph &g, const rr_query *q, uint64_t *d_witness, uint64_t *d_E,
                         uint32_t *d_R, uint8_t *d_bitmap, cudaStream_t st,
                         const uint8_t *d_vmask = nullptr);
// The fine-grained query on workspace `ws` (budget as reach_on_stream).
// bfirst > 0: also the at-most-k branches k' = bfirst..k-1 (reach_v2), their
// witnesses, per-edge sums and minimum arrivals in ws.bS / ws.bE / ws.bR at
// row k' - bfirst.
rr_status arrival_on(const Graph &g, Workspace &ws, const rr_query *q, uint64_t *d_witness,
                     uint64_t *d_E, uint32_t *d_R, uint8_t *d_bitmap, cudaStream_t st,
                     const uint8_t *d_vmask, uint64_t budget, uint32_t bfirst = 0);
// Bounded RestlessReach: minimum arrival over k' = 2..k, shortest length, D.
rr_status atmost_arrival_device(const Graph &g, uint32_t source, uint32_t k, uint64_t seed,
                                uint32_t *d_R, uint8_t *d_L, uint8_t *d_bitmap, cudaStream_t st);
// Makes sure the graph has at least `lanes` concurrent-query lanes (rr_batch.cu).
rr_status ensure_fan_lanes(const Graph &g, uint32_t lanes);
// A set of sources and optional separators (n flags, device).
rr_status sources_device(const Graph &g, const uint32_t *sources, uint32_t nsources, uint32_t k,
                         uint64_t seed, const uint8_t *motif, const uint8_t *d_separators,
                         uint8_t *d_bitmap, uint64_t *d_witness, cudaStream_t st);
// One optimal restless path to `target` by k-1 fine-grained queries (host outputs).
rr_status extract_path(const Graph &g, const rr_query *q, uint32_t target, uint32_t *vertices,
                       uint32_t *edges, uint32_t *times);

}  // namespace rr

struct rr_graph : public rr::Graph {};
