/*
 * restless_reach.h -- C ABI of the GB300 (sm_103a) constrained multilinear
 * sieve for k-RestlessReach and k-RestlessMotifReach ("Restless reachability
 * problems in temporal graphs", arXiv 2010.08423).
 *
 * What is computed (edge-layer form of Eq. (1) with the sieve of Eq. (2)/(3),
 * the per-vertex output of Algorithm 1):
 *   for every sieve point L subset of [k] and every edge e = (u_e, v_e, t_e):
 *     x_u^L     = sum_{j in L} z_{u,j}
 *     P_1^L[e]  = [u_e = s] y_{e,1} x_s^L x_{v_e}^L
 *     P_l^L[e]  = y_{e,l} x_{v_e}^L sum_{f: v_f = u_e, t_f <= t_e <= t_f + delta(u_e)} P_{l-1}^L[f]
 *   witness[v]  = sum_L sum_{e: v_e = v} P_{k-1}^L[e]
 *   reach[v]    = (witness[v] != 0)
 * All arithmetic is in GF(2^64) = GF(2)[x]/(x^64 + x^4 + x^3 + x + 1), elements
 * stored as uint64 with bit i the coefficient of x^i; "sum" is XOR.
 * A non-zero witness proves a restless path with exactly k vertices from s to v
 * (whose colours agree with the motif M for motif queries); a path is missed
 * with probability at most (3k-1)/2^64 per vertex (Schwartz-Zippel; the paper
 * quotes (2k-1)/2^b for the uncoloured sieve).
 *
 * Random values (counter-form splitmix64; Steele, Lea & Flood 2014):
 *   mix(z)        = standard splitmix64 finaliser
 *   draw(key, i)  = mix(key + (i+1) * 0x9E3779B97F4A7C15)
 *   key_F         = mix(seed ^ F), F = 1 (y), 2 (z), 3 (gamma), 4 (omega)
 *   y_{e,l}       = draw(key_1, e*32 + l-1)        e = input edge index
 *   plain:   z_{u,j} = draw(key_2, u*32 + j-1)
 *   motif:   z_{u,j} = sum_{d in S_{c(u)}} draw(key_3, u*32 + d) * draw(key_4, d*32 + j-1)
 *            (Eq. (3); shades d = 0..k-1 assigned colour by colour in ascending
 *             colour order; z_{u,j} = 0 if c(u) is not in M)
 *
 * Conventions shared by every entry point:
 *   - Vertices are 0..n-1; edge e is (src[e], dst[e], t[e]) with e the input
 *     index; timestamps and waiting times are uint32; delta(v) = 0 is allowed.
 *     The wait bound is the delta of the vertex being left, both window ends
 *     inclusive (restless-walk definition).
 *   - k counts path vertices (the path has k-1 edges); 2 <= k <= 20.
 *   - Bitmaps: bit v is byte v>>3, bit v&7; ceil(n/8) bytes.
 *   - Host buffers passed in are only read during the call; outputs are
 *     caller-allocated. Handles are owned by the library (free with the
 *     matching *_free / *_destroy).
 *   - Every call returns an rr_status; on failure rr_last_error() gives a
 *     thread-local message. No call aborts the process.
 *   - All device work runs on the current CUDA device of the calling thread.
 */
#ifndef RESTLESS_REACH_H
#define RESTLESS_REACH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RR_OK = 0,
    RR_EINVAL = 1,    /* invalid argument (bad k, source, endpoint, self-loop, motif without colours) */
    RR_ENOMEM = 2,    /* device memory cannot hold the request (admission refused) */
    RR_EAGAIN = 3,    /* query queued or still running */
    RR_ETIMEDOUT = 4, /* a bounded device wait gave up; results of that query are invalid */
    RR_ECANCELED = 5, /* query was cancelled */
    RR_ECUDA = 6,     /* a CUDA runtime call failed */
    RR_ENOPATH = 7    /* rr_extract_path: no path of k vertices reaches the target */
} rr_status;

typedef struct rr_graph rr_graph;
typedef struct rr_server rr_server;

/* One reachability query. motif == NULL: plain k-RestlessReach (uncoloured
 * sieve, Eq. (2)). motif != NULL: k-RestlessMotifReach with the multiset M
 * given as k colour values (any order; Eq. (3)); needs a coloured graph. */
typedef struct {
    uint32_t source;
    uint32_t k;
    uint64_t seed;
    const uint8_t *motif;
} rr_query;

typedef struct {
    uint32_t n;
    uint64_t m;
    uint64_t state_rows;     /* rows of the windowed prefix state (1 + producer rows) */
    uint64_t window_rows;    /* edges whose restless window is non-empty */
    uint32_t max_in_degree;
    uint32_t num_items;      /* vertex ranges the layer kernels are scheduled over */
    uint64_t device_bytes;   /* bytes the resident graph holds on the device */
    int has_colors;
    int compact;             /* 1: state stores only rows inside some window */
    uint64_t producer_window_rows; /* rows inside some window whose own window is non-empty */
    uint64_t state_compute_rows;   /* of those, rows whose window holds another such row ("deep") */
    uint64_t tail_rows;            /* rows whose window holds a producer row with a window */
    uint64_t deep_compute_rows;    /* deep rows whose window holds a deep row */
    uint64_t deep_tail_rows;       /* rows whose window holds a deep row */
    uint64_t deep_head_runs;       /* head runs over the deep rows' scheduling ranges */
    int pair_layer3_min_k;         /* smallest k whose layer 3 runs in pair-label
                                      space (21: none; see rr_graph_load's flags) */
    uint32_t deep_max_range_rows;  /* rows of the longest deep-row scheduling range (at
                                      most 4: the pair rows are built in one launch) */
    uint32_t deep_heads;           /* distinct heads of the deep rows */
    int head_table;                /* 1: layer 4 of the pair form reads x_u x_s from a
                                      per-chunk table of those heads */
    int pair_tail;                 /* 1: queries with k >= 6 (k >= 7 with layer 3 in
                                      pair-label space) and at most 8 point groups per
                                      chunk run layer k-2 in label space from the pair
                                      sums of layer k-3 (rr_graph_load's flags) */
} rr_graph_info;

/* ---- graph ----------------------------------------------------------------
 * rr_graph_load: copies the temporal multigraph to the device and builds the
 * in-edge CSR sorted by (head, time, edge index), the restless window of
 * every edge (Eq. (1)'s j in {0..delta}: rows of the tail's in-segment with
 * t_e - delta(u_e) <= t_f <= t_e) and the scheduling ranges. Host arrays are
 * read only; src/dst/t have m entries, delta n, color n (or NULL).
 * flags: bit 0 set = keep the dense state layout (one state row per edge)
 * instead of storing only rows that lie in some window. Layer 3 in pair-label
 * space stores per deep row the k(k+1)/2 values of a symmetric label-pair
 * matrix Q, independent of the sieve points, and layer 4 evaluates
 * x_u^L x_s^L sum_{i,j in L} dQ_ij over each window; queries with 9 <= k <=
 * 20 use it. Bit 1 set = use it from k = 6, bit 2 set = never (layer 3 per
 * point from the label-space prefix). Layer 4 takes x_u x_s from a per-chunk
 * table of the deep rows' heads when they number at most half the deep rows
 * with a non-empty window; bit 3 / bit 4 set = always / never. Both bits of a
 * pair set is RR_EINVAL. The last layer needs of layer k-2 only its sums over
 * the points of a group times x_w^L, and with layer k-2's factor y x_v^L those
 * are bilinear forms over layer k-3's sums on the points holding one or two
 * given labels: with the pair tail, layer k-3 stores those sums (a 32-value
 * block per deep row and group of points) instead of per-point state, and
 * layer k-2 keeps 16 label-space values per deep row; bit 5 set = never (layer
 * k-2 per point, writing its sums over single labels). Bit 6 / bit 7 set =
 * rr_reach_atmost_device runs every k' as a query of its own / always takes
 * the k' it can from the k query's layers (by default: when those layers are
 * long). A k = 4 query over all its points runs layer 2 in label space and
 * its last layer in closed form (per row, y_{e,3} times the 4 x 4 permanent of
 * z_s, z_v, z_w and the window's label-space sums); bit 8 set = per point
 * instead. Bit 9 set = a k = 5 query over all its points runs layer 3 in
 * pair-label space and its last layer in closed form (per row, y_{e,4} times
 * the sum over the splits of the five labels into one for z_w, a pair for z_v
 * and z_s and a pair for the window's pair sums) instead of per point (the
 * default; the two measured within 4% of each other). Results are
 * bit-identical in every form. The pair
 * rows ((deep rows + 1) * k(k+1)/2 words) and the head table (heads * chunk
 * words) are part of a query's scratch and, unlike the per-point state, do not
 * shrink with the point chunk: a server whose per-slot budget cannot hold them
 * for its largest k refuses to start (RR_ENOMEM); bit 2 avoids that.
 * Errors: RR_EINVAL for n == 0, m >= 2^31, an endpoint >= n or a self-loop;
 * RR_ENOMEM / RR_ECUDA on device failure (nothing is leaked). */
rr_status rr_graph_load(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                        const uint32_t *t, const uint32_t *delta, const uint8_t *color,
                        uint32_t flags, rr_graph **out);
rr_status rr_graph_free(rr_graph *g);
rr_status rr_graph_get_info(const rr_graph *g, rr_graph_info *out);

/* ---- one query, one launch sequence (the plain GPU form) --------------------
 * rr_reach_sync: runs one query to completion on the library's internal
 * stream and copies results to HOST buffers bitmap (ceil(n/8) bytes, may be
 * NULL) and witness (n uint64, may be NULL). Thread-safe per graph (calls on
 * one graph are serialised). */
rr_status rr_reach_sync(const rr_graph *g, const rr_query *q, uint8_t *bitmap,
                        uint64_t *witness);

/* rr_reach_device: same computation, enqueued on `stream` (a cudaStream_t,
 * NULL = legacy default stream) with DEVICE outputs d_bitmap (ceil(n/8)
 * bytes, may be NULL) and d_witness (n uint64, required). Returns once the
 * work is enqueued. The graph's scratch is reused by the next call: calls on
 * one graph that use it (this one, rr_reach_sync, the batched, at-most-k,
 * fine-grained, set-of-sources and extraction calls, rr_autotune) may be
 * issued on different streams -- each call's stream first waits, on the
 * device, for the previous such call's work. */
rr_status rr_reach_device(const rr_graph *g, const rr_query *q, uint8_t *d_bitmap,
                          uint64_t *d_witness, void *stream);

/* rr_reach_range_device: the part of rr_reach_device's witness that the sieve
 * points L = first .. first+count-1 contribute (Eq. (2): the polynomial is a
 * sum over L of independent evaluations, and Algorithm 1 sums its per-vertex
 * values over L, so the parts of disjoint ranges XOR to the full witness):
 *   d_witness[v] = sum_{L in [first, first+count)} sum_{e: v_e = v} P_{k-1}^L[e]
 * (n uint64, device, required; overwritten). This is how one query is split
 * across GPUs or processes: each evaluates its range on its own copy of the
 * graph and the parts are XOR-combined (an all-gather, then a local XOR).
 * first must be a multiple of 128 and first + count <= 2^k; count == 0 writes
 * zeros (first then only needs first <= 2^k). For k <= 3 the library sums all points at once in closed form, so
 * count must be 0 or 2^k there. No bitmap: reachability needs the full sum.
 * Same engine, scratch, stream ordering and errors as rr_reach_device;
 * RR_EINVAL for a misaligned or out-of-range part. */
rr_status rr_reach_range_device(const rr_graph *g, const rr_query *q, uint32_t first,
                                uint32_t count, uint64_t *d_witness, void *stream);

/* rr_reach_device_noalloc: the computation of rr_reach_device for callers that
 * must not allocate device memory while they serve queries -- a process whose
 * device memory is already owned by another allocator's pool, or a
 * latency-critical loop that cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree brings. It calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch (z-table, shade table, both prefix-state
 * buffers) is one static device array of 256 MiB in the library, resident on
 * every device where the library's device code is loaded until the process
 * exits (with CUDA's default lazy module loading from the first use of that
 * code on the device; with CUDA_MODULE_LOADING=EAGER on every device the
 * process creates a context on), and counted as used by cudaMemGetInfo-based
 * budgets such as rr_server_create's. The paper has no counterpart; this is a
 * deployment variant of the same sieve.
 * Arguments are those of rr_reach_device; the graph's device must be current.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * starts. Queries whose scratch would exceed 256 MiB (n*k*8 bytes of z-table
 * plus 2 * state_rows * c * 8 bytes of state for the smallest point chunk, c =
 * 32 * points per lane: 64 points for k <= 6, 128 from k = 7 unless
 * rr_set_tuning chose 2 points per lane) are rejected with RR_ENOMEM and a
 * message giving both sizes. The graph's tuning for k is read under the
 * graph's lock, so rr_autotune and rr_set_tuning may run beside it. Every call
 * shares the array and clears what must start at zero itself; calls whose
 * work overlaps on the GPU (unordered streams) race on it, so order them on
 * one stream. */
rr_status rr_reach_device_noalloc(const rr_graph *g, const rr_query *q, uint8_t *d_bitmap,
                                  uint64_t *d_witness, void *stream);

/* ---- many queries, one persistent launch (batched form) --------------------
 * rr_reach_batch_device: runs nq queries of any mix of k, sources and motifs
 * in ONE persistent kernel launch. Work is split into (query, point chunk,
 * layer, vertex range) items drained from a device queue in dependency order;
 * a layer item waits (bounded spin) for the previous layer of its chunk.
 * Outputs: d_witness (nq*n uint64, row q = query q) and d_bitmaps (nq *
 * ceil(n/8) bytes, may be NULL), device memory, enqueued on `stream`.
 * d_status (nq int32, device, may be NULL) receives RR_OK or RR_ETIMEDOUT per
 * query. Results equal rr_reach_device's bit for bit. */
rr_status rr_reach_batch_device(const rr_graph *g, const rr_query *qs, uint32_t nq,
                                uint8_t *d_bitmaps, uint64_t *d_witness, int32_t *d_status,
                                void *stream);

/* rr_reach_arrival_device: the fine-grained decision oracle (Algorithm 1; Sec.
 * "A fine-grained decision oracle") for one query. Algorithm 1 keeps a
 * polynomial per (vertex u, time i) for the walks of k vertices ending at u
 * with a last edge at time i; here that polynomial is the XOR of the per-edge
 * sums over the edges into u at time i.
 *   d_witness   (n uint64, device, required) per-vertex sums, as rr_reach_device;
 *   d_edge_sums (m uint64, device, may be NULL) for every input edge e, the sum
 *               over all 2^k sieve points of e's last-layer value (the walks of
 *               k vertices whose last edge is e);
 *   d_arrival   (n uint32, device, required) R_u = the smallest i whose
 *               polynomial is non-zero, UINT32_MAX if there is none (the minimum
 *               reachability time of Algorithm 1);
 *   d_bitmap    (ceil(n/8) bytes, device, may be NULL) Algorithm 1's D: bit u set
 *               iff R_u < UINT32_MAX.
 * Enqueued on `stream`. Without d_edge_sums the library keeps an m * 8-byte
 * buffer with the graph. Errors: RR_EINVAL for a NULL required argument or an
 * invalid query (as rr_reach_device); RR_ENOMEM, RR_ECUDA as rr_reach_device. */
rr_status rr_reach_arrival_device(const rr_graph *g, const rr_query *q, uint64_t *d_witness,
                                  uint64_t *d_edge_sums, uint32_t *d_arrival, uint8_t *d_bitmap,
                                  void *stream);

/* rr_reach_sources_device: k-RestlessReach (or MotifReach) from a set of
 * sources, optionally avoiding separators (Sec. "Discussion": the set-of-sources
 * variant; Sec. on separators in the case study). Walks start at every edge
 * leaving any of the nsources vertices in `sources` (host array), so the
 * witness is the XOR of the single-source witnesses with the same seed, and a
 * vertex is reached iff some restless path of k vertices from some source
 * (with colours M when `motif` is given) ends at it. d_separators (n flags,
 * device, may be NULL): vertices no path may use (their z rows are zero).
 * One source runs the same engine as rr_reach_device; several run the
 * per-point engine. d_witness (n uint64, device, required) and d_bitmap
 * (ceil(n/8), device, may be NULL) as rr_reach_device. Enqueued on `stream`.
 * Errors: RR_EINVAL for NULL sources/d_witness, nsources == 0 or an invalid
 * query for any source; RR_ENOMEM, RR_ECUDA as rr_reach_device. */
rr_status rr_reach_sources_device(const rr_graph *g, const uint32_t *sources, uint32_t nsources,
                                  uint32_t k, uint64_t seed, const uint8_t *motif,
                                  const uint8_t *d_separators, uint8_t *d_bitmap, uint64_t *d_witness,
                                  void *stream);

/* rr_extract_path: one optimal restless path (Sec. "Extracting an optimal
 * solution using k queries"; the k-RestlessPath / k-RestlessMotif problems):
 * k vertices from q->source to `target`, their colours equal to q->motif's
 * multiset when given, whose last edge time is the target's minimum arrival
 * time (the smallest possible largest timestamp). It takes k-1 fine-grained
 * queries: for k vertices, then for l = k-1 .. 2 vertices on the graph without
 * the vertices already chosen (deleted vertices have zero z rows) and without
 * their colours in the motif. The next vertex back is the tail u of an edge
 * (u, cur, t_cur) whose restless window t_cur - delta(u) <= i <= t_cur holds a
 * time i with a non-zero (u, i) polynomial; ties go to the earliest i, then to
 * the smallest input edge index, and the first edge is the smallest-index edge
 * from the source at the chosen time. Every step is certified by a non-zero
 * polynomial, so the path returned is always a valid restless path.
 *   vertices (k uint32, host) u_1 = source .. u_k = target;
 *   edges    (k-1 uint32, host) input edge index of (u_j, u_{j+1});
 *   times    (k-1 uint32, host) that edge's time.
 * Synchronous; uses the graph's own stream and scratch. Errors: RR_EINVAL for
 * NULL outputs, target >= n, target == source or an invalid query; RR_ENOPATH
 * if the target has no arrival (or, with probability <= (3k-1)/2^64 per step, a
 * step's polynomials vanished); RR_ENOMEM / RR_ECUDA on device failure. */
rr_status rr_extract_path(const rr_graph *g, const rr_query *q, uint32_t target, uint32_t *vertices,
                          uint32_t *edges, uint32_t *times);

/* rr_reach_atmost_device: at-most-k-RestlessReach (Sec. "Discussion"; Algorithm 2
 * with its loop over k' stopped at k): the plain queries (source, k', seed) for
 * k' = 2..k. d_witness ((k-1) * n uint64, device) gets the witness of k' in row
 * k'-2; d_bitmap (ceil(n/8) bytes, device, may be NULL) gets the union of the
 * reach sets: vertices reached by a restless path of at most k vertices.
 * For one seed the k'-vertex query's per-point layers agree with the
 * k-vertex query's on the first 2^k' points, so the k query also yields the
 * queries k' >= 5: after its per-point layer k'-2 it forms k''s sums over
 * single labels from its stored rows and runs k''s last layer (with the pair
 * tail, k-1's last layer reads those sums straight from layer k-3's pair sums;
 * with the pair-label layer 3, k' = 5 is the closed form over its pair rows). That is done where the k query's per-point layers are
 * long (deep rows with a window times min(2^k, 1024) at least 2^23; with
 * short layers the concurrent queries finish first; rr_graph_load's bits 6
 * and 7 force either form). Ordered on
 * `stream`: the k query and the smaller queries run concurrently on streams of
 * the library's own that start after the work already on `stream` and that
 * `stream` waits for; when their scratch does not fit 60% of free device memory
 * together every k' runs as its own query, one after another on `stream`.
 * Scratch stays allocated with the graph. Errors as rr_reach_device. */
rr_status rr_reach_atmost_device(const rr_graph *g, uint32_t source, uint32_t k, uint64_t seed,
                                 uint8_t *d_bitmap, uint64_t *d_witness, void *stream);

/* rr_reach_bounded_device: RestlessReach bounded by k (Algorithm 2 with its
 * loop over k' stopped at k, its outputs R and D accumulated over the loop):
 * the fine-grained query (rr_reach_arrival_device) for every k' = 2..k from
 * `source`, plain colours.
 *   d_arrival (n uint32, device, required): R_v = the smallest time at which a
 *             restless path of at most k vertices from the source can end at
 *             v (the minimum over k' of the k'-vertex minimum arrival), or
 *             UINT32_MAX if none;
 *   d_length  (n uint8, device, may be NULL): the vertex count of a shortest
 *             restless path from the source to v (2..k), 0 if none;
 *   d_bitmap  (ceil(n/8) bytes, device, may be NULL): D = {v : R_v defined}.
 * The k-1 queries run concurrently on the library's lanes (as
 * rr_reach_atmost_device) when their scratch (including m*8 bytes of per-edge
 * sums each) fits 60% of free device memory, else one after another. Ordered on
 * `stream`. Errors as rr_reach_device. */
rr_status rr_reach_bounded_device(const rr_graph *g, uint32_t source, uint32_t k, uint64_t seed,
                                  uint32_t *d_arrival, uint8_t *d_length, uint8_t *d_bitmap,
                                  void *stream);

/* ---- serving: continuous batching over a resident graph --------------------
 * rr_server_create: starts a server thread that admits queries while device
 * memory (device_mem_budget bytes of scratch, 0 = 60% of free memory) and
 * max_slots (concurrent point chunks, 0 = automatic) allow, runs every
 * admitted chunk's layers as they become ready, and retires queries as their
 * last chunk finishes, so that queries arriving while others run share the
 * GPU with them. rr_server_set_batching can instead admit a backlog of queued
 * queries on the reduced-state engine in batches to the persistent batch
 * kernel (rr_reach_batch_device), on one of two batch lanes whose outputs
 * take at most a quarter of the budget; that is off by default, since the
 * slots' concurrent launch sequences serve faster (n = 1e5, m = 1e6, plain
 * k ~ U{6..12}, a burst of 160 queries: about 13,000 queries/s on 4 slots
 * against 9,000 with batches of up to 64). Results are identical to
 * rr_reach_sync's either way. */
rr_status rr_server_create(const rr_graph *g, uint64_t device_mem_budget, uint32_t max_slots,
                           rr_server **out);
rr_status rr_server_destroy(rr_server *s);
/* Copies the query (and motif); returns a ticket. RR_ENOMEM if the query can
 * never fit the budget, RR_EINVAL on a bad query. */
rr_status rr_query_submit(rr_server *s, const rr_query *q, uint64_t *ticket);
/* Waits up to timeout_ms (0 = do not wait, <0 = forever). RR_OK: results
 * copied to the host buffers (either may be NULL) and the ticket released;
 * RR_EAGAIN: not finished; RR_ECANCELED / RR_ETIMEDOUT: final, ticket released. */
rr_status rr_query_poll(rr_server *s, uint64_t ticket, int32_t timeout_ms, uint8_t *bitmap,
                        uint64_t *witness);
rr_status rr_query_cancel(rr_server *s, uint64_t ticket);
/* Per-ticket timing in microseconds: submit->admit, submit->done. */
rr_status rr_query_times(rr_server *s, uint64_t ticket, double *queue_us, double *total_us);
/* Counts since creation: queries admitted one at a time to a slot, queries
 * admitted in batches, and batches launched. Any pointer may be NULL. */
rr_status rr_server_stats(rr_server *s, uint64_t *single, uint64_t *batched, uint64_t *batches);
/* Batch admission: a backlog of min_batch queued queries starts a batch of up
 * to max_batch (2 <= min_batch <= max_batch <= the lanes' capacity: 256, or
 * fewer where a quarter of the budget holds fewer); min_batch = 0 turns
 * batching off. The lanes' buffers are allocated on the first call that
 * turns batching on (RR_ENOMEM / RR_ECUDA if that fails). RR_EINVAL on other
 * values or on a server without lanes (per-point engine graphs). */
rr_status rr_server_set_batching(rr_server *s, uint32_t min_batch, uint32_t max_batch);

/* ---- tuning ----------------------------------------------------------------
 * Kernel shape used for a (graph, k): points per lane (2 or 4) and points per
 * chunk. rr_autotune times the candidates on the resident graph for the given
 * k and stores the winner in the graph; rr_set_tuning forces one. */
rr_status rr_autotune(rr_graph *g, uint32_t k, uint32_t *best_ppl, uint32_t *best_chunk);
rr_status rr_set_tuning(rr_graph *g, uint32_t k, uint32_t ppl, uint32_t chunk);

/* Shape of the persistent batch (rr_reach_batch_device and the server's batch
 * lanes), kept per graph; 0 in a field = the automatic rule.
 *   blocks_per_sm  kernel variant by the blocks per SM its register budget is
 *                  set for: 2 (168 registers), 4 (128), 5 (96, a few spills) or 6
 *                  (80, more spills);
 *   ranges         1 = fine scheduling ranges (one head run each), 2 = coarse
 *                  (about 32 row-list entries each);
 *   max_chunk      largest point chunk of a unit: 128, 256, 512 or 1024 (a query
 *                  with at least 128 points takes chunks of at least 128).
 * The automatic rule takes coarse ranges with 5 blocks when the first wave's
 * tasks are at least half the resident warps, else fine ranges with 2, and
 * chunks up to 512. rr_autotune_batch picks the batch's tile (scheduling range)
 * and sieve points per block by measurement: it runs the batch qs[0..nq) once
 * untimed and twice timed per candidate -- the 24 combinations of 2/4/5/6
 * blocks, fine/coarse ranges and 256/512/1024-point chunks -- keeps the fastest in
 * the graph and returns it in *best (may be NULL). Results are bit-identical in
 * every shape. Uses the graph's scratch (ordered as rr_reach_device). Errors:
 * RR_EINVAL for a NULL graph, nq == 0 or an invalid query; RR_ENOMEM / RR_ECUDA. */
typedef struct {
    uint32_t blocks_per_sm;
    uint32_t ranges;
    uint32_t max_chunk;
} rr_batch_tuning;
rr_status rr_autotune_batch(rr_graph *g, const rr_query *qs, uint32_t nq, rr_batch_tuning *best);
/* Forces a batch shape (fields as above; RR_EINVAL for other values). */
rr_status rr_set_batch_tuning(rr_graph *g, const rr_batch_tuning *t);
rr_status rr_get_batch_tuning(const rr_graph *g, rr_batch_tuning *out);

/* ---- verification entry points ---------------------------------------------
 * rr_debug_point_sums: per-vertex sums of single sieve points: out[p*n + v] =
 * sum_{e: v_e = v} P_{k-1}^{L_p}[e] for L_p = masks[p] (HOST arrays). */
rr_status rr_debug_point_sums(const rr_graph *g, const rr_query *q, const uint32_t *masks,
                              uint32_t nmasks, uint64_t *out);
/* rr_debug_graph: copies the build's CSR back to HOST arrays: off (n+1),
 * row_eid, row_lo, row_hi (m each; window [lo,hi) as absolute CSR rows of the
 * tail's segment). Any pointer may be NULL. */
rr_status rr_debug_graph(const rr_graph *g, uint32_t *off, uint32_t *row_eid, uint32_t *row_lo,
                         uint32_t *row_hi);
/* rr_debug_ztable: z_{u,j} table of a query (HOST out, n*k, row u). */
rr_status rr_debug_ztable(const rr_graph *g, const rr_query *q, uint64_t *out);
/* rr_debug_gf_mul: out[i] = a[i]*b[i] in GF(2^64) on the device, HOST arrays. */
rr_status rr_debug_gf_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t count);
/* rr_bench_gf_mul: the device GF(2^64) multiply at its peak rate, for the
 * arithmetic roofline of the sieve kernels (not part of the paper's method).
 * Enqueues blocks x threads threads on `stream`, each running `iters` steps of
 * four independent products in registers, every operand value entering
 * exactly one product (as in the sieve kernels, so no operand preparation is
 * shared between products); *mults (host) receives the number of
 * multiplications enqueued;
 * d_sink (one uint64, device) keeps the results live and is practically never
 * written. Errors: RR_EINVAL for threads == 0 or > 1024, blocks == 0 or a NULL
 * pointer; RR_ECUDA if the launch fails. */
rr_status rr_bench_gf_mul(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *d_sink,
                          uint64_t *mults, void *stream);
/* rr_debug_wait_probe: runs the bounded wait of the persistent batched kernel
 * (the wait a task does for the tasks it depends on) on a counter that nothing
 * increments, so that its failure path can be tested without a fault: the wait
 * must give up after timeout_ns of device time (or at once when abort_preset is
 * non-zero: the batch's abort flag is set), report RR_ETIMEDOUT in *status (host)
 * and leave the context usable. *elapsed_ns (host) = the wait's duration.
 * Synchronous, default stream. Errors: RR_EINVAL for NULL outputs or a timeout
 * above 10 s. Not part of the paper's method. */
rr_status rr_debug_wait_probe(uint64_t timeout_ns, int32_t abort_preset, int32_t *status,
                              uint64_t *elapsed_ns);
/* rr_debug_draw: out[i] = draw(key, first + i) on the device, HOST out. */
rr_status rr_debug_draw(uint64_t key, uint64_t first, uint64_t count, uint64_t *out);

/* ---- kernel timing ---------------------------------------------------------
 * While enabled (process-wide), every kernel launch of the sieve is bracketed
 * by CUDA events on the stream it is launched on; rr_timing_read waits for the
 * recorded events and returns the summed durations and launch counts per
 * kind: 0 = first layer, 1 = middle layers reading state, 2 = last layer with
 * the fused per-vertex reduce, 3 = z-table, 4 = persistent batched kernel,
 * 5 = second layer (window sums from the first layer's scalar prefix),
 * 6 = the last per-point layer, writing the transformed state (layer k-2, or
 * k-3 with the pair tail), 7 = layer 3 in pair-label space, 8 = the pair
 * tail's layer k-2 in label space. While timing is enabled the
 * launches are issued one by one instead of as a captured CUDA graph. */
typedef struct {
    double ms[9];
    uint64_t launches[9];
} rr_kernel_times;
rr_status rr_timing_enable(int enable);
rr_status rr_timing_read(rr_kernel_times *out, int reset);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char *rr_last_error(void);
/* Number of kernel launches this library issued since load (all threads). */
uint64_t rr_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* RESTLESS_REACH_H */
