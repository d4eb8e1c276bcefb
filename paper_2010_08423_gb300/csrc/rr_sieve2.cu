// rr_sieve2.cu -- the reduced-state engine: same per-vertex sums as the
// per-point engine (rr_sieve.cu), with exact rewrites of the work.
//
// 1. Layer 1 as a scalar. P_1^L[f] = [u_f = s] y_{f,1} x_s^L x_{v_f}^L, so
//    the layer-2 window sum of edge e = (u, v) is W_2^L[e] = Y_e x_s^L x_u^L with
//    the scalar Y_e = sum of y_{f,1} over the source's edges f inside e's window.
//    Layer 1 therefore stores one GF(2^64) prefix per producer row (PY), not one
//    per sieve point.
// 2. Layer 2 in label space (k >= 5): P_2^L[f] = x_v^L x_s^L sum_{j in L}
//    (y Y)_f z_{u_f,j}, so layer 2 keeps k values per state row (rows whose
//    own window is non-empty), independent of the point chunk.
// 3. Layer 3 from that label-space prefix, factored per head:
//    acc^L = (x_v x_s)^L sum_e x_{u_e}^L (y rho_e)^L.
// 4. Deep rows only from layer 3 on: state rows whose window holds a state row
//    are the only rows that can be non-zero there.
// 5. The last layer as a linear form. x_v^L = sum_{j in L} z_{v,j}, hence
//        sum_L y_e x_v^L W^L = y_e sum_j z_{v,j} T_j(W),  T_j(W) = sum_{L ni j} W^L,
//    and T_j is XOR-linear, so layer k-2 stores for every row and point group
//    only the lg+1 sums T_j (j below lg = log2 of the group size) and V = the
//    sum over the group (the high labels of a group are fixed, so their T_j is
//    V or 0), and layer k-1 needs one multiplication per stored value instead
//    of one per sieve point.
// 6. k = 2 and k = 3 in closed form (a 2x2 / 3x3 permanent per edge).
// 7. Layer 3 in pair-label space (9 <= k <= 20 by default): the sum in 3. is
//    (x_v x_s)^L times the quadratic form sum_{i,j in L} Q_ij of the label
//    pair matrix Q = XOR over v's rows of z_{u_e} (x) (y rho_e), so layer 3
//    keeps k(k+1)/2 values per deep row, independent of the point chunk, and
//    layer 4 evaluates the form of each window (times x_u x_s) per point.
// 8. The pair tail (chunks of at least 256 points): the last layer uses layer
//    k-2 only through sums over point groups of x_w^L P^L, and with layer
//    k-2's factor y x_v^L those are bilinear forms in the z values of w and v
//    over layer k-3's sums on the points holding one or two given labels; so
//    layer k-3 stores those sums and layer k-2 runs in label space
//    (label_tail_warp in rr_v2_device.cuh).
// 9. At-most-k from one query: for one seed a k'-vertex query's per-point
//    layers equal the k-vertex query's on its first 2^k' points, so the k
//    query, after its layer k'-2, forms k''s single-label sums from its rows
//    and runs k''s last layer (the branches of enqueue_query_v2).
// Only the order of summation changes; every result is bit-identical to the
// per-point engine and the oracle. One query's launch sequence is captured
// once per shape as a CUDA graph and its kernels use programmatic dependent
// launch.
#include <algorithm>
#include <cstring>

#include "rr_v2_device.cuh"

namespace rr {

// Launches a kernel of the single-query sequence with programmatic stream
// serialisation: it may be scheduled while the previous kernel of the stream
// still runs, and waits for it in pdl_enter() before touching memory. Captured
// into the per-shape CUDA graph as a programmatic dependency.
// Off for workspaces whose queries run beside others on concurrent streams:
// there a grid waiting for its predecessor holds SM slots the other streams'
// kernels could use.
static thread_local bool t_pdl = true;

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = t_pdl ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// What a query clears before its layers: the witness (n values; n = 0 skips
// it) and the zero rows of the scratch -- row 0 of the scalar prefix, of both
// full state buffers (chunk values each), of the transformed buffer (rstride
// values: its row width), of the label-space prefix (kpr2 values) and of the
// pair tail's rows. Null pointers skip.
struct ZeroRows {
    uint64_t *py, *full0, *full1, *red, *pr2;
    uint32_t n, chunk, rstride, kpr2;
    uint64_t *pr3;
    uint32_t npr3;
    uint64_t *carry;  // the carry table's zero row (chunk values) or null
    uint64_t *lrows;  // the pair tail's label-space rows (kLabelTailWidth values) or null
    uint64_t *bred;   // the at-most-k branches' transformed buffer (bred_w values) or null
    uint32_t bred_w;
};

__device__ __forceinline__ void zero_rows(const QueryDesc *__restrict__ qd, const ZeroRows &z)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t *S = qd->S;
    for (uint32_t v = tid; v < z.n; v += stride) S[v] = 0;
    if (z.py && tid == 0) z.py[0] = 0;
    if (z.full0)
        for (uint32_t i = tid; i < z.chunk; i += stride) {
            z.full0[i] = 0;
            z.full1[i] = 0;
        }
    if (z.red)
        for (uint32_t i = tid; i < z.rstride; i += stride) z.red[i] = 0;
    if (z.pr2)
        for (uint32_t i = tid; i < z.kpr2; i += stride) z.pr2[i] = 0;
    if (z.pr3)
        for (uint32_t i = tid; i < z.npr3; i += stride) z.pr3[i] = 0;
    if (z.carry)
        for (uint32_t i = tid; i < z.chunk; i += stride) z.carry[i] = 0;
    if (z.lrows)
        for (uint32_t i = tid; i < kLabelTailWidth; i += stride) z.lrows[i] = 0;
    if (z.bred)
        for (uint32_t i = tid; i < z.bred_w; i += stride) z.bred[i] = 0;
}

// Layer 1; its grid also clears what zero_rows lists (saving a launch).
__global__ void __launch_bounds__(kW2 * 32) k_first_scalar(const V2Params p, uint64_t *__restrict__ py,
                                                           const ZeroRows zr)
{
    pdl_enter();
    zero_rows(p.qd, zr);
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    first_scalar_warp(p, task, py);
}

template <int PPL, bool FROM_Y, int OUT, bool FROM_R2 = false, bool PAIR = false>
__global__ void __launch_bounds__(kW2 * 32) k_layer_v2(const V2Params p)
{
    // pdl_enter() inside layer_warp, after the graph- and query-only loads
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems * p.ngroups) return;
    const uint32_t item = task / p.ngroups;
    layer_warp<PPL, FROM_Y, OUT, false, FROM_R2, PAIR>(p, item, task - item * p.ngroups);
}

// Carry fix-up of cut head segments (rr_v2_device.cuh): phase 1 one block
// per cut segment, phase 2 one block per task of kFixRows row slots.
__global__ void k_fix1(const uint2 *__restrict__ chains, uint32_t nchains, uint64_t *buf,
                       uint32_t width)
{
    pdl_enter();
    if (blockIdx.x >= nchains) return;
    const uint2 ch = chains[blockIdx.x];
    fixup_phase1<false>(buf, width, ch.x, ch.y, threadIdx.x, blockDim.x);
}

__global__ void k_fix2(const uint2 *__restrict__ chains, const uint2 *__restrict__ tasks,
                       uint32_t ntasks, uint64_t *buf, uint32_t width)
{
    pdl_enter();
    if (blockIdx.x >= ntasks) return;
    const uint2 t = tasks[blockIdx.x];
    const uint2 ch = chains[t.x];
    fixup_phase2<false>(buf, width, ch.x, ch.y, t.y, threadIdx.x, blockDim.x);
}

// The carry table of the deep list's per-point state (rr_v2_device.cuh
// carry_rows): one block per cut segment.
__global__ void k_carry(const uint2 *__restrict__ chains, const uint32_t *__restrict__ slot0,
                        uint32_t nchains, const uint64_t *buf, uint64_t *carry, uint32_t width)
{
    pdl_enter();
    if (blockIdx.x >= nchains) return;
    const uint2 ch = chains[blockIdx.x];
    carry_rows(buf, carry, width, ch.x, ch.y, slot0[blockIdx.x], threadIdx.x, blockDim.x);
}

static rr_status launch_fixup(const RowList &L, uint64_t *buf, uint32_t width, cudaStream_t st,
                              uint64_t *nk)
{
    if (L.nchains == 0) return RR_OK;
    RR_CUDA(launch_pdl(k_fix1, dim3(L.nchains), dim3(128), st, L.chains.as<uint2>(), L.nchains, buf,
                       width));
    RR_LAUNCHED();
    ++*nk;
    if (L.nfix2) {
        RR_CUDA(launch_pdl(k_fix2, dim3(L.nfix2), dim3(256), st, L.chains.as<uint2>(),
                           L.fix2.as<uint2>(), L.nfix2, buf, width));
        RR_LAUNCHED();
        ++*nk;
    }
    return RR_OK;
}

__global__ void __launch_bounds__(kW2 * 32) k_second_label(const V2Params p, uint64_t *__restrict__ pr2)
{
    // pdl_enter() inside second_label_scan_warp, after the graph- and query-only loads
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    second_label_scan_warp<true>(p, task, pr2);
}

__global__ void __launch_bounds__(kW2 * 32) k_third_pair(const V2Params p, uint32_t count,
                                                         uint64_t *__restrict__ pr3)
{
    // pdl_enter() inside third_pair_row, after the graph- and query-only loads
    const uint32_t e = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (e >= count) return;
    third_pair_row(p, e, pr3);
}

__global__ void __launch_bounds__(kW2 * 32) k_third_pair_fused(const V2Params p, uint64_t *__restrict__ pr3)
{
    // pdl_enter() inside third_pair_fused, after the graph- and query-only loads
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    third_pair_fused(p, task, pr3);
}

template <int PPL>
__global__ void __launch_bounds__(kW2 * 32) k_head_factor(const V2Params p)
{
    // pdl_enter() inside head_factor_warp, before its stores
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.ndheads * p.ngroups) return;
    const uint32_t r = task / p.ngroups;
    head_factor_warp<PPL>(p, r, task - r * p.ngroups);
}

__global__ void __launch_bounds__(kW2 * 32) k_pair_prefix(const V2Params p, uint64_t *__restrict__ pr3)
{
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    pair_prefix_warp(p, task, pr3);
}

__global__ void k_first2(const V2Params p, const uint32_t *__restrict__ off,
                         const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ row_eid,
                         uint32_t m)
{
    pdl_enter();
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
        first2_closed(p, off, row_src, row_eid, r);
}

__global__ void k_last3(const V2Params p, uint32_t count)
{
    pdl_enter();
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        last3_closed(p, e);
}

// k = 4: the last layer in closed form over the label-space layer 2
// (last4_closed), a quad of lanes per row of the tail list.
__global__ void __launch_bounds__(256) k_last4(const V2Params p, uint32_t count)
{
    const uint32_t j = threadIdx.x & 3u;
    const uint64_t zs_j = zval(p, p.qd->source, j);  // reads the z table
    pdl_enter();
    // warp-uniform steps of 8 rows: every warp stays whole for its shuffles
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = gridDim.x * blockDim.x / 32u;
    for (uint64_t base = (uint64_t)warp * 8u; base < count; base += (uint64_t)nwarps * 8u)
        last4_closed(p, (uint32_t)base + ((threadIdx.x & 31u) >> 2), count, zs_j);
}

// k = 5: the last layer in closed form over the pair-label layer 3
// (last5_closed), eight lanes per row of the deep-tail list; np = values per
// pair row (pair_count of the query that wrote them).
__global__ void __launch_bounds__(256) k_last5(const V2Params p, uint32_t count, uint32_t np)
{
    const uint32_t c = threadIdx.x & 7u;
    const bool act = c < 5u;
    const uint32_t s = p.qd->source;
    const uint64_t zs0 = act ? zval(p, s, c) : 0ull;  // reads the z table
    const uint64_t zs1 = act ? zval(p, s, (c + 1u) % 5u) : 0ull;
    const uint64_t zs2 = act ? zval(p, s, (c + 2u) % 5u) : 0ull;
    pdl_enter();
    // warp-uniform steps of 4 rows: every warp stays whole for its shuffles
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = gridDim.x * blockDim.x / 32u;
    for (uint64_t base = (uint64_t)warp * 4u; base < count; base += (uint64_t)nwarps * 4u)
        last5_closed(p, (uint32_t)base + ((threadIdx.x & 31u) >> 3), count, np, zs0, zs1, zs2);
}

// PB: from the pair tail's sums of a larger query (at-most-k branch k-1).
template <int LG, bool PB = false>
__global__ void __launch_bounds__(kW2 * 32) k_last_v2(const V2Params p)
{
    // pdl_enter() inside last_warp, after the graph- and query-only loads
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    last_warp<LG, false, PB>(p, task);
}

// Pair tail (rr_v2_device.cuh): layer k-2 in label space from layer k-3's
// pair sums, and the last layer from its rows.
template <int LG>
__global__ void __launch_bounds__(kW2 * 32) k_label_tail(const V2Params p)
{
    __shared__ uint64_t sm[kW2][192];
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    label_tail_warp<LG, false>(p, task, sm[threadIdx.x >> 5]);
}

template <int LG>
__global__ void __launch_bounds__(kW2 * 32) k_last_label(const V2Params p)
{
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= p.nitems) return;
    last_label_warp<LG, false>(p, task);
}

// At-most-k branch: one layer's stored rows as a smaller query's transformed
// state (transform_rows_warp).
template <int PPL>
__global__ void __launch_bounds__(kW2 * 32) k_branch_transform(const V2Params p, uint32_t nrows)
{
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= (nrows + 31) / 32 * p.ngroups) return;
    transform_rows_warp<PPL>(p, task, nrows);
}

static unsigned blocks_for(uint64_t tasks)
{
    return (unsigned)((tasks + kW2 - 1) / kW2);
}

// Fills the list fields of V2Params; `win` selects the window indices:
// 0 = producer prefix (a0, b0), 1 = state rows (a1, b1), 3 = deep rows (a3, b3).
static void set_list(V2Params &vp, const RowList &L, int win)
{
    vp.head = L.head.as<uint32_t>();
    vp.eid = L.eid.as<uint32_t>();
    vp.src = L.src.as<uint32_t>();
    vp.ia = win == 0 ? L.a0.as<uint32_t>() : (win == 1 ? L.a1.as<uint32_t>() : L.a3.as<uint32_t>());
    vp.ib = win == 0 ? L.b0.as<uint32_t>() : (win == 1 ? L.b1.as<uint32_t>() : L.b3.as<uint32_t>());
    vp.items = L.items.as<uint2>();
    vp.nitems = L.nitems;
    vp.trank = L.trank.as<uint32_t>();  // deep list only (else unused)
}

// src: 0 = window sums from the per-point state, 1 = from the scalar layer-1
// prefix (layer 2), 2 = from the label-space layer-2 prefix (layer 3), 3 = from
// pair-label layer-3 windows (layer 4).
template <int PPL>
static rr_status launch_v2(const V2Params &vp, int src, int out, cudaStream_t st)
{
    const uint64_t tasks = (uint64_t)vp.nitems * vp.ngroups;
    if (tasks == 0) return RR_OK;
    // pair sums (out 2) come only from a middle layer: the pair tail needs
    // 256-point chunks, so k >= 8 and layer k-3 >= 5
    if (out == 2 && src != 0) return fail(RR_EINVAL, "internal: pair sums from a first per-point layer");
    const int tslot = timing_begin(st);
    const unsigned blocks = blocks_for(tasks);
    const dim3 B(kW2 * 32);
    if (src == 1) {
        if (out == 0) RR_CUDA(launch_pdl(k_layer_v2<PPL, true, 0>, dim3(blocks), B, st, vp));
        else RR_CUDA(launch_pdl(k_layer_v2<PPL, true, 1>, dim3(blocks), B, st, vp));
    } else if (src == 2) {
        if (out == 1) RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 1, true>, dim3(blocks), B, st, vp));
        else RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 0, true>, dim3(blocks), B, st, vp));
    } else if (src == 3) {
        if (out == 0) RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 0, false, true>, dim3(blocks), B, st, vp));
        else RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 1, false, true>, dim3(blocks), B, st, vp));
    } else {
        if (out == 0) RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 0>, dim3(blocks), B, st, vp));
        else if (out == 2) RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 2>, dim3(blocks), B, st, vp));
        else RR_CUDA(launch_pdl(k_layer_v2<PPL, false, 1>, dim3(blocks), B, st, vp));
    }
    timing_end(tslot, src == 1 ? kTimeSecond : (out != 0 ? kTimeTail : kTimeMid), st);
    RR_LAUNCHED();
    return RR_OK;
}

// Number of 8-byte values one transformed state row holds.
uint32_t v2_reduced_stride(uint32_t ppl, uint32_t chunk)
{
    const uint32_t lg = ppl == 4 ? 7u : 6u;
    return chunk / (32u * ppl) * (lg + 1u);
}

// Layer 3 in pair-label space (third_pair_row), layer 4 reading its windows:
// queries with 6 <= k <= 20 when the graph's load flags force it, else with
// k >= kPairMinK unless they turn it off.
static bool pair_layer3(const Graph &g, uint32_t k)
{
    if (k < 6 || pair_count(k) > kMaxPairs) return false;
    return g.pair_force ? g.pair_force == 2 : k >= kPairMinK;
}

// Layer 4 of the pair form reads x_u x_s from a per-chunk table of the deep
// rows' heads (one product per head and point) instead of forming it for every
// row with a non-empty window: when there are at most half as many heads.
static bool head_table(const Graph &g)
{
    if (g.head_table_force) return g.head_table_force == 2;
    return 2ull * g.deep_list.nheads <= g.deep_compute_rows;
}

// Words of the carry table of the deep list's per-point state (zero when no
// head segment of the deep list is cut or no layer keeps per-point state there).
static uint64_t carry_words(const Graph &g, uint32_t chunk, uint32_t k)
{
    return (k >= 6 && g.deep_list.nchains) ? ((uint64_t)g.deep_list.ncarry * chunk + 31) / 32 * 32 : 0;
}

// Layers k-2 and k-1 from layer k-3's pair sums (the pair tail): when layer
// k-3 keeps per-point state (k >= 6; k >= 7 with layer 3 in pair-label space)
// and a chunk has kPairTailMinChunk points or more in at most
// kPairTailMaxGroups point groups, unless the load flags turn it off. (256
// points need k >= 8: layer k-3 is then a middle layer.)
static bool pair_tail(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k)
{
    const uint32_t first = pair_layer3(g, k) ? 4u : 3u;  // the first per-point layer
    return !g.pair_tail_off && k >= 6 && first + 3 <= k && chunk >= kPairTailMinChunk &&
           chunk / (32u * ppl) <= kPairTailMaxGroups;
}

uint32_t atmost_first_branch(const Graph &g, uint32_t k)
{
    // first per-point layer + 2 (5, or 6 with the pair-label layer 3, where
    // k' = 5 is the closed form over the k query's pair rows)
    (void)g;
    return 5u < k ? 5u : 0u;
}

uint32_t atmost_branches(const Graph &g, uint32_t k)
{
    if (!uses_v2(g, k) || g.atmost_branches == 1) return 0;
    // by default only where the k query's per-point layers are long: with
    // short, latency-bound layers the concurrent queries finish first (n = 1e5,
    // m = 1e6, k = 10: 0.24 ms against 0.27, k = 12: 0.63 against 0.68; a
    // Chung-Lu n = 2e5 graph, k = 10: 8.2 ms against 5.4)
    const bool long_layers =
        (uint64_t)g.deep_compute_rows * std::min<uint64_t>(1ull << k, 1024) >= (1ull << 23);
    return g.atmost_branches == 2 || long_layers ? atmost_first_branch(g, k) : 0u;
}

// Words of the pair tail's label-space rows (layer k-2), zero when it is off.
static uint64_t label_tail_words(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k)
{
    return pair_tail(g, ppl, chunk, k) ? ((uint64_t)g.deep_list.count + 1) * kLabelTailWidth : 0;
}

// Words of each part of the engine's scratch, in layout order: scalar layer-1
// prefix, label-space layer-2 prefix (k per state row), pair rows, head table,
// two per-point buffers, one transformed buffer (then the carry table, the
// pair tail's label-space rows and the at-most-k branches' transformed buffer).
static void v2_layout(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k, uint64_t *py_w,
                      uint64_t *pr2_w, uint64_t *pr3_w, uint64_t *tx_w, uint64_t *full_w,
                      uint64_t *red_w)
{
    const uint64_t srows = g.state_list.count + 1;  // layer 2 (label space; k = 4 transformed)
    const uint64_t drows = g.deep_list.count + 1;   // layers >= 3
    // k = 2 and k = 3 are closed forms: no per-point state
    *py_w = k >= 3 ? (g.prod_list.count + 1 + 31) / 32 * 32 : 0;
    *pr2_w = k >= 4 ? (srows * k + 31) / 32 * 32 : 0;  // k = 4: the closed-form last layer's
    // (k = 5: the closed-form last layer's)
    *pr3_w = pair_layer3(g, k) || k == 5 ? (drows * pair_count(k) + 31) / 32 * 32 : 0;
    *tx_w = pair_layer3(g, k) && head_table(g) ? (uint64_t)std::max<uint32_t>(1, g.deep_list.nheads) * chunk : 0;
    *full_w = k >= 4 ? drows * chunk : 0;
    // whole 256-byte blocks: the next buffer (the carry table) is read with
    // 16-byte vector loads, and a transformed row holds 7 values per group
    // with 2 points per lane
    *red_w = k >= 4 ? (std::max(srows, drows) * v2_reduced_stride(ppl, chunk) + 31) / 32 * 32 : 0;
    // with the pair tail it holds layer k-3's pair sums (a 32-value block per
    // deep row and point group)
    if (pair_tail(g, ppl, chunk, k))
        *red_w = std::max<uint64_t>(*red_w, drows * (chunk / (32u * ppl)) * kPairTailSlots);
}

// At-most-k branches' own transformed buffer (single-label sums, the
// per-point tail's row width), after the pair tail's rows.
static uint64_t branch_words(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k)
{
    const uint64_t drows = g.deep_list.count + 1;
    return k >= 6 ? (drows * v2_reduced_stride(ppl, chunk) + 31) / 32 * 32 : 0;
}

uint64_t v2_scratch_bytes(const Graph &g, uint32_t ppl, uint32_t chunk, uint32_t k, bool branches)
{
    uint64_t py_w, pr2_w, pr3_w, tx_w, full_w, red_w;
    v2_layout(g, ppl, chunk, k, &py_w, &pr2_w, &pr3_w, &tx_w, &full_w, &red_w);
    return (py_w + pr2_w + pr3_w + tx_w + 2 * full_w + red_w + carry_words(g, chunk, k) +
            (label_tail_words(g, ppl, chunk, k) + 31) / 32 * 32 +
            (branches ? branch_words(g, ppl, chunk, k) : 0)) * 8ull + 4096;
}

// z_{u,j} from the descriptor's keys (plain iid draws or Eq. (3) shades); rows
// of deleted vertices are zero. Coloured graphs visit the vertices in colour
// order (`order`), so a warp's shade loops have one length.
__global__ void k_ztable_q(uint32_t n, uint32_t k, const QueryDesc *__restrict__ qd,
                           const uint8_t *__restrict__ color, const uint32_t *__restrict__ order,
                           uint64_t *__restrict__ z)
{
    pdl_enter();
    const uint64_t total = (uint64_t)n * k;
    const bool colored = qd->colored != 0;
    const uint64_t kz = qd->key_z, kg = qd->key_g, ko = qd->key_o;
    for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pos = total <= 0xffffffffull ? (uint64_t)((uint32_t)idx / k) : idx / k;
        const uint32_t j = (uint32_t)(idx - pos * k);
        const uint64_t u = colored && order ? order[pos] : pos;
        uint64_t val = 0;
        if (!colored) {
            val = sm_draw(kz, u * 32u + j);
        } else {
            const uint32_t c = color[u];
            const uint32_t d0 = qd->shades[c], mu = qd->shades[256 + c];
            for (uint32_t d = d0; d < d0 + mu; ++d)
                val ^= gf64_mul(sm_draw(kg, u * 32u + d), sm_draw(ko, (uint64_t)d * 32u + j));
        }
        if (qd->vmask && qd->vmask[u]) val = 0;
        z[u * k + j] = val;
    }
}

__global__ void k_zero_q(const QueryDesc *__restrict__ qd, const ZeroRows zr)
{
    pdl_enter();
    zero_rows(qd, zr);
}

__global__ void k_bitmap_q(uint32_t n, const QueryDesc *__restrict__ qd)
{
    pdl_enter();
    const uint64_t *S = qd->S;
    uint8_t *bm = qd->bitmap;
    const uint32_t nb = (n + 7) / 8;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t i = 0; i < 8; ++i) {
            const uint32_t v = b * 8 + i;
            if (v < n && S[v] != 0) bits |= 1u << i;
        }
        bm[b] = (uint8_t)bits;
    }
}

static unsigned grid_cap(uint64_t count, unsigned block)
{
    uint64_t g = (count + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152ull * 64) g = 152ull * 64;
    return (unsigned)g;
}

// At-most-k branch kb after per-point layer kb - 2 (vp: that layer's launch
// parameters, vp.st_out its rows; carry: the carry table k_carry wrote for it,
// or null): the rows' sums over single labels of the point groups below
// 2^kb into `red`, then kb's last layer with descriptor d_bd.
static rr_status enqueue_branch(const Graph &g, const V2Params &vp, uint32_t kb, const QueryDesc *d_bd,
                                uint64_t *carry, uint64_t *red, uint32_t ppl, uint64_t stop_k,
                                cudaStream_t st, cudaEvent_t tr_done, uint64_t *nk)
{
    V2Params vb = vp;
    const uint64_t stop = std::min<uint64_t>(stop_k, 1ull << kb);  // the branch's points end
    const uint32_t gs = 32u * ppl;
    vb.ngroups = (uint32_t)std::min<uint64_t>(vp.ngroups, (stop - vp.chunk_base + gs - 1) / gs);
    vb.npoints = (uint32_t)stop;
    vb.st_in = vp.st_out;
    vb.st_out = red;
    vb.carry = carry;
    vb.row_carry = carry ? g.deep_list.row_carry.as<uint32_t>() : nullptr;
    const uint32_t nrows = (uint32_t)g.deep_list.count;
    const uint64_t tasks = (uint64_t)(nrows + 31) / 32 * vb.ngroups;
    if (tasks) {
        const int tslot = timing_begin(st);
        if (ppl == 4) RR_CUDA(launch_pdl(k_branch_transform<4>, dim3(blocks_for(tasks)), dim3(kW2 * 32), st, vb, nrows));
        else RR_CUDA(launch_pdl(k_branch_transform<2>, dim3(blocks_for(tasks)), dim3(kW2 * 32), st, vb, nrows));
        timing_end(tslot, kTimeTail, st);
        RR_LAUNCHED();
        ++*nk;
    }
    if (tr_done) RR_CUDA(cudaEventRecord(tr_done, st));
    vb.qd = d_bd;
    vb.k = kb;
    vb.layer = kb - 1;
    vb.st_in = red;
    vb.carry = nullptr;
    vb.row_carry = nullptr;
    set_list(vb, g.tail3_list, 3);
    if (vb.nitems) {
        const int tslot = timing_begin(st);
        const dim3 grid(blocks_for(vb.nitems)), B(kW2 * 32);
        if (ppl == 4) RR_CUDA(launch_pdl(k_last_v2<7>, grid, B, st, vb));
        else RR_CUDA(launch_pdl(k_last_v2<6>, grid, B, st, vb));
        timing_end(tslot, kTimeLast, st);
        RR_LAUNCHED();
        ++*nk;
    }
    return RR_OK;
}

// At-most-k branch k-1 with the pair tail (vp: the launch parameters of the k
// query's layer k-3, its pair sums in vp.st_out after their fix-up): their
// single-label slots are what layer k-3 of the (k-1)-vertex query would store
// for its point groups below 2^(k-1), so the branch is that query's last layer
// alone. The groups must not straddle 2^(k-1).
static rr_status enqueue_pair_branch(const Graph &g, const V2Params &vp, uint32_t kb, const QueryDesc *d_bd,
                                     uint32_t ppl, uint64_t stop_k, cudaStream_t st, uint64_t *nk)
{
    V2Params vb = vp;
    const uint64_t stop = std::min<uint64_t>(stop_k, 1ull << kb);
    const uint32_t gs = 32u * ppl;
    if (stop % gs) return fail(RR_EINVAL, "internal: a point group straddles the branch's points");
    vb.ngroups = (uint32_t)std::min<uint64_t>(vp.ngroups, (stop - vp.chunk_base) / gs);
    vb.blk_groups = vp.ngroups;
    vb.npoints = (uint32_t)stop;
    vb.qd = d_bd;
    vb.k = kb;
    vb.layer = kb - 1;
    vb.st_in = vp.st_out;
    vb.carry = nullptr;
    vb.row_carry = nullptr;
    set_list(vb, g.tail3_list, 3);
    if (vb.nitems && vb.ngroups) {
        const int tslot = timing_begin(st);
        const dim3 grid(blocks_for(vb.nitems)), B(kW2 * 32);
        if (ppl == 4) RR_CUDA(launch_pdl(k_last_v2<7, true>, grid, B, st, vb));
        else RR_CUDA(launch_pdl(k_last_v2<6, true>, grid, B, st, vb));
        timing_end(tslot, kTimeLast, st);
        RR_LAUNCHED();
        ++*nk;
    }
    return RR_OK;
}

rr_status enqueue_query_v2(const Graph &g, uint32_t k, bool table, bool bitmap, uint32_t ppl,
                           uint32_t chunk, uint64_t *d_z, uint64_t *d_scratch,
                           const QueryDesc *d_desc, cudaStream_t st, uint64_t *kernels, bool pdl,
                           PointRange range, const QueryDesc *d_bdesc, uint32_t bfirst,
                           cudaStream_t side, cudaEvent_t *bev)
{
    // k <= 3 sums all points in closed form: only the whole range exists there
    if (k <= 3 && !range.full(k)) return fail(RR_EINVAL, "a part of the sieve points needs k >= 4");
    if (range.first % kRangeAlign || range.first > range.stop(k) || range.stop(k) > (1u << k))
        return fail(RR_EINVAL, "bad sieve-point range");
    struct PdlScope {
        bool saved;
        explicit PdlScope(bool on) : saved(t_pdl) { t_pdl = on; }
        ~PdlScope() { t_pdl = saved; }
    } pdl_scope(pdl);
    uint64_t nk = 0;
    uint64_t py_w, pr2_w, pr3_w, tx_w, full_w, red_w;
    v2_layout(g, ppl, chunk, k, &py_w, &pr2_w, &pr3_w, &tx_w, &full_w, &red_w);
    const bool pair = pair_layer3(g, k);
    // k = 5 over the whole range with the load flag: layer 3 in pair-label
    // space and the last layer in closed form (no per-point state)
    const bool closed5 = k == 5 && range.full(k) && g.k5_closed;
    const bool prows = pair || closed5;  // layer 3's pair rows
    uint64_t *py = d_scratch;
    uint64_t *pr2 = py + py_w;
    uint64_t *pr3 = pr2 + pr2_w;
    uint64_t *tx = pr3 + pr3_w;
    uint64_t *full0 = tx + tx_w;
    uint64_t *full1 = full0 + full_w;
    uint64_t *red = full1 + full_w;
    uint64_t *carry = carry_words(g, chunk, k) ? red + red_w : nullptr;
    const uint32_t rstride = v2_reduced_stride(ppl, chunk);
    // the pair tail: layer k-3 writes pair sums into `red`, layer k-2 its
    // label-space rows after the carry table (with at-most-k branches only
    // where no point group straddles 2^(k-1): branch k-1 reads the sums)
    const bool ptail = pair_tail(g, ppl, chunk, k) && (bfirst == 0 || (1ull << (k - 1)) % (32u * ppl) == 0);
    uint64_t *lrows = ptail ? red + red_w + carry_words(g, chunk, k) : nullptr;
    // at-most-k branches: their transformed buffer, so that they can run on
    // the side stream while the query goes on
    bool side_used = false, red_pending = false;
    if (bfirst && side && !bev) return fail(RR_EINVAL, "internal: branch side stream without events");
    uint64_t *bred = bfirst ? red + red_w + carry_words(g, chunk, k) +
                                  (label_tail_words(g, ppl, chunk, k) + 31) / 32 * 32
                            : nullptr;
    const uint32_t red_width = ptail ? chunk / (32u * ppl) * kPairTailSlots : rstride;

    {
        if (table) {  // plain queries without deletions draw z on the fly
            const int tslot = timing_begin(st);
            RR_CUDA(launch_pdl(k_ztable_q, dim3(grid_cap((uint64_t)g.n * k, 256)), dim3(256), st, g.n, k,
                               d_desc, g.color.as<uint8_t>(), g.color_order.as<uint32_t>(), d_z));
            timing_end(tslot, kTimeZ, st);
            RR_LAUNCHED();
            ++nk;
        }
    }
    // the witness and the scratch's zero rows (k = 2 has no scratch); cleared by
    // the first layer's grid when it runs
    const ZeroRows zr{k >= 3 ? py : nullptr, k >= 4 ? full0 : nullptr, k >= 4 ? full1 : nullptr,
                      k >= 4 ? red : nullptr, k >= 4 ? pr2 : nullptr, g.n, chunk, red_width, k,
                      prows ? pr3 : nullptr, pair_count(k), carry, lrows, bred, rstride};
    const bool zero_in_first = k >= 3 && g.prod_list.nitems > 0;
    if (!zero_in_first) {
        RR_CUDA(launch_pdl(k_zero_q, dim3(grid_cap(g.n, 256)), dim3(256), st, d_desc, zr));
        RR_LAUNCHED();
        ++nk;
    }
    V2Params vp{};
    vp.qd = d_desc;
    vp.z = table ? d_z : nullptr;
    vp.n = g.n;
    vp.k = k;
    vp.chunk = chunk;
    vp.ngroups = chunk / (32u * ppl);
    // points at or past the range's end are masked off in every per-point layer
    vp.npoints = range.stop(k);

    if (k == 2) {
        // the only layer, in closed form
        if (g.m) {
            const int tslot = timing_begin(st);
            RR_CUDA(launch_pdl(k_first2, dim3(grid_cap(g.m, 256)), dim3(256), st, vp, g.off.as<uint32_t>(),
                               g.row_src.as<uint32_t>(), g.row_eid.as<uint32_t>(), (uint32_t)g.m));
            timing_end(tslot, kTimeFirst, st);
            RR_LAUNCHED();
            ++nk;
        }
        if (bitmap) {
            RR_CUDA(launch_pdl(k_bitmap_q, dim3(grid_cap((g.n + 7) / 8, 256)), dim3(256), st, g.n, d_desc));
            RR_LAUNCHED();
            ++nk;
        }
        if (kernels) *kernels = nk;
        return RR_OK;
    }

    // layer 1: scalar prefix (independent of the point chunk)
    set_list(vp, g.prod_list, 0);
    vp.layer = 1;
    if (vp.nitems) {
        const int tslot = timing_begin(st);
        RR_CUDA(launch_pdl(k_first_scalar, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp, py, zr));
        timing_end(tslot, kTimeFirst, st);
        RR_LAUNCHED();
        ++nk;
        rr_status fs = launch_fixup(g.prod_list, py, 1, st, &nk);
        if (fs != RR_OK) return fs;
    }
    vp.py = py;
    vp.pr2 = pr2;
    // k = 4 over the whole range: layer 2 in label space and the last layer in
    // closed form (no per-point state)
    const bool closed4 = k == 4 && range.full(k) && !g.k4_per_point;
    if (k >= 5 || closed4) {
        // layer 2 in label space (independent of the point chunk)
        set_list(vp, g.state_list, 0);
        vp.layer = 2;
        if (vp.nitems) {
            const int tslot = timing_begin(st);
            RR_CUDA(launch_pdl(k_second_label, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp, pr2));
            timing_end(tslot, kTimeSecond, st);
            RR_LAUNCHED();
            ++nk;
            rr_status fs = launch_fixup(g.state_list, pr2, k, st, &nk);
            if (fs != RR_OK) return fs;
        }
    }

    if (prows) {
        // layer 3 in pair-label space (independent of the point chunk), over
        // the deep rows with their state-row windows
        set_list(vp, g.deep_list, 1);
        vp.layer = 3;
        if (vp.nitems) {
            const uint32_t count = (uint32_t)g.deep_list.count;
            const int tslot = timing_begin(st);
            if (g.deep_max_item <= kPairFusedMaxRows) {
                // short ranges only: both passes in one launch
                RR_CUDA(launch_pdl(k_third_pair_fused, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp, pr3));
                RR_LAUNCHED();
                nk += 1;
            } else {
                RR_CUDA(launch_pdl(k_third_pair, dim3(blocks_for(count)), dim3(kW2 * 32), st, vp, count, pr3));
                RR_LAUNCHED();
                RR_CUDA(launch_pdl(k_pair_prefix, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp, pr3));
                RR_LAUNCHED();
                nk += 2;
            }
            timing_end(tslot, kTimeThird, st);
            rr_status fs = launch_fixup(g.deep_list, pr3, pair_count(k), st, &nk);
            if (fs != RR_OK) return fs;
        }
    }
    vp.pr3 = pr3;
    vp.tx = tx_w ? tx : nullptr;
    vp.dheads = g.deep_list.heads.as<uint32_t>();
    vp.ndheads = g.deep_list.nheads;
    const uint32_t ntail3 = (uint32_t)g.tail3_list.count;
    if (closed5 && ntail3) {
        set_list(vp, g.tail3_list, 3);
        vp.layer = 4;
        const int tslot = timing_begin(st);
        RR_CUDA(launch_pdl(k_last5, dim3(grid_cap(((uint64_t)ntail3 + 3) / 4 * 32, 256)), dim3(256), st, vp,
                           ntail3, pair_count(5)));
        timing_end(tslot, kTimeLast, st);
        RR_LAUNCHED();
        ++nk;
    }
    if (bfirst == 5 && pair && ntail3) {
        // at-most-k branch k' = 5: its last layer in closed form over this
        // query's pair rows (labels 0..4), beside the query
        cudaStream_t bs = st;
        if (side) {
            RR_CUDA(cudaEventRecord(bev[0], st));
            RR_CUDA(cudaStreamWaitEvent(side, bev[0], 0));
            bs = side;
            side_used = true;
        }
        V2Params vb = vp;
        vb.qd = d_bdesc;
        vb.k = 5;
        vb.layer = 4;
        vb.z = nullptr;  // branches are plain queries
        set_list(vb, g.tail3_list, 3);
        const int tslot = timing_begin(bs);
        RR_CUDA(launch_pdl(k_last5, dim3(grid_cap(((uint64_t)ntail3 + 3) / 4 * 32, 256)), dim3(256), bs, vb,
                           ntail3, pair_count(k)));
        timing_end(tslot, kTimeLast, bs);
        RR_LAUNCHED();
        ++nk;
    }

    if (k == 3 && g.win_list.count) {
        // last layer in closed form (no sieve points)
        set_list(vp, g.win_list, 0);
        vp.layer = 2;
        const int tslot = timing_begin(st);
        RR_CUDA(launch_pdl(k_last3, dim3(grid_cap(g.win_list.count, 256)), dim3(256), st, vp,
                           (uint32_t)g.win_list.count));
        timing_end(tslot, kTimeLast, st);
        RR_LAUNCHED();
        ++nk;
    }
    if (closed4 && g.tail_list.count) {
        set_list(vp, g.tail_list, 1);
        vp.layer = 3;
        const int tslot = timing_begin(st);
        RR_CUDA(launch_pdl(k_last4, dim3(grid_cap((g.tail_list.count + 7) / 8 * 32, 256)), dim3(256), st, vp,
                           (uint32_t)g.tail_list.count));
        timing_end(tslot, kTimeLast, st);
        RR_LAUNCHED();
        ++nk;
    }
    const uint64_t npts = range.stop(k) - range.first;
    const uint64_t nchunks = k == 3 || closed4 || closed5 ? 0 : (npts + chunk - 1) / chunk;
    for (uint64_t c = 0; c < nchunks; ++c) {
        vp.chunk_base = range.first + (uint32_t)(c * chunk);
        rr_status s = RR_OK;
        // per-point layers 2 (k = 4) or 3 (k >= 5) .. k-2, or .. k-3 with the
        // pair tail; the last of them writes the transformed state (its sums
        // over label sets of the point groups: single labels, or with the
        // pair tail at most two)
        uint64_t *bufs[2] = {full0, full1};
        const uint32_t last_pp = ptail ? k - 3 : k - 2;
        bool tr_pending = false;
        // branch k-1 reads the pair sums in `red` on the side stream until bev[3]
        // with layer 3 in pair-label space the per-point layers start at 4,
        // layer 4 reading the pair windows
        for (uint32_t l = pair ? 4u : (k >= 5 ? 3u : 2u); l <= last_pp; ++l) {
            const int src = (l == 2) ? 1 : (l == 3 ? 2 : (pair && l == 4 ? 3 : 0));
            const int out = l == last_pp ? (ptail ? 2 : 1) : 0;
            // layer 2 (k = 4) runs over the state rows; layers >= 3 over the deep rows,
            // layer 3 reading the label-space prefix at state-row indices
            if (src == 3 && vp.tx && vp.ndheads) {
                // this chunk's x_h x_s table for the heads of the deep rows
                const uint64_t tasks = (uint64_t)vp.ndheads * vp.ngroups;
                const int tslot = timing_begin(st);
                if (ppl == 4)
                    RR_CUDA(launch_pdl(k_head_factor<4>, dim3(blocks_for(tasks)), dim3(kW2 * 32), st, vp));
                else
                    RR_CUDA(launch_pdl(k_head_factor<2>, dim3(blocks_for(tasks)), dim3(kW2 * 32), st, vp));
                timing_end(tslot, kTimeThird, st);
                RR_LAUNCHED();
                ++nk;
            }
            if (src == 1) set_list(vp, g.state_list, 0);
            else set_list(vp, g.deep_list, src == 2 ? 1 : 3);
            vp.layer = l;
            vp.st_in = bufs[(l - 1) & 1u];
            vp.st_out = out != 0 ? red : bufs[l & 1u];
            if (out != 0 && red_pending) {  // the previous chunk's branch k-1 has read `red`
                RR_CUDA(cudaStreamWaitEvent(st, bev[3], 0));
                red_pending = false;
            }
            // per-point state read from the previous layer carries lazily
            vp.carry = src == 0 ? carry : nullptr;
            vp.row_carry = carry ? g.deep_list.row_carry.as<uint32_t>() : nullptr;
            if (src == 2 && out == 0 && ppl == 4) {
                // layer 3 writing full state: the lane-to-point map does not
                // change the stored rows, and 2 points per lane halve the
                // registers of this multiply-heavy layer (twice the warps in flight)
                vp.ngroups = chunk / 64u;
                s = launch_v2<2>(vp, src, out, st);
                vp.ngroups = chunk / (32u * ppl);
            } else {
                s = ppl == 4 ? launch_v2<4>(vp, src, out, st) : launch_v2<2>(vp, src, out, st);
            }
            if (s != RR_OK) return s;
            nk += vp.nitems ? 1 : 0;
            if (tr_pending) {
                // the previous layer's branch has read its rows and carries
                RR_CUDA(cudaStreamWaitEvent(st, bev[1], 0));
                tr_pending = false;
            }
            if (carry && out == 0 && src != 1) {
                // per-point state of the deep list: the carry table, read by the next layer
                RR_CUDA(launch_pdl(k_carry, dim3(g.deep_list.nchains), dim3(128), st,
                                   g.deep_list.chains.as<uint2>(), g.deep_list.chain_slot0.as<uint32_t>(),
                                   g.deep_list.nchains, (const uint64_t *)vp.st_out, carry, chunk));
                RR_LAUNCHED();
                ++nk;
            } else {
                s = launch_fixup(src == 1 ? g.state_list : g.deep_list, vp.st_out,
                                 out == 0 ? chunk : red_width, st, &nk);
                if (s != RR_OK) return s;
            }
            // at-most-k branch: this layer is layer k'-2 of the k'-vertex query
            // (k' = l + 2), whose points below 2^k' it holds; their sums over
            // single labels, then that query's last layer
            // (on the side stream when given: it reads this layer's rows and
            // carries, which the query overwrites after its next layer)
            const uint32_t kb = l + 2;
            if (bfirst && out == 0 && kb >= bfirst && kb < k && (uint64_t)vp.chunk_base < (1ull << kb)) {
                cudaStream_t bs = st;
                if (side) {
                    RR_CUDA(cudaEventRecord(bev[0], st));
                    RR_CUDA(cudaStreamWaitEvent(side, bev[0], 0));
                    bs = side;
                    side_used = tr_pending = true;
                }
                s = enqueue_branch(g, vp, kb, d_bdesc + (kb - bfirst), carry, bred, ppl, range.stop(k), bs,
                                   side ? bev[1] : nullptr, &nk);
                if (s != RR_OK) return s;
            }
            if (bfirst && out == 2 && k - 1 >= bfirst && (uint64_t)vp.chunk_base < (1ull << (k - 1))) {
                // branch k-1 from the fixed-up pair sums
                cudaStream_t bs = st;
                if (side) {
                    RR_CUDA(cudaEventRecord(bev[0], st));
                    RR_CUDA(cudaStreamWaitEvent(side, bev[0], 0));
                    bs = side;
                }
                s = enqueue_pair_branch(g, vp, k - 1, d_bdesc + (k - 1 - bfirst), ppl, range.stop(k), bs, &nk);
                if (s != RR_OK) return s;
                if (side) {
                    RR_CUDA(cudaEventRecord(bev[3], side));
                    side_used = red_pending = true;
                }
            }
        }
        if (ptail) {
            // layer k-2 in label space from the pair sums of its windows
            set_list(vp, g.deep_list, 3);
            vp.layer = k - 2;
            vp.st_in = red;
            vp.st_out = lrows;
            vp.carry = nullptr;
            vp.row_carry = nullptr;
            if (vp.nitems) {
                const int tslot = timing_begin(st);
                if (ppl == 4) RR_CUDA(launch_pdl(k_label_tail<7>, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp));
                else RR_CUDA(launch_pdl(k_label_tail<6>, dim3(blocks_for(vp.nitems)), dim3(kW2 * 32), st, vp));
                timing_end(tslot, kTimeLabelTail, st);
                RR_LAUNCHED();
                ++nk;
                s = launch_fixup(g.deep_list, lrows, kLabelTailWidth, st, &nk);
                if (s != RR_OK) return s;
            }
        }
        // layer k-1 from the transformed state (state-row indices when k = 4)
        // or from the pair tail's label-space rows
        if (k == 4) set_list(vp, g.tail_list, 1);
        else set_list(vp, g.tail3_list, 3);
        vp.layer = k - 1;
        vp.st_in = ptail ? lrows : red;
        if (vp.nitems) {
            const int tslot = timing_begin(st);
            const dim3 grid(blocks_for(vp.nitems)), B(kW2 * 32);
            if (ptail) {
                if (ppl == 4) RR_CUDA(launch_pdl(k_last_label<7>, grid, B, st, vp));
                else RR_CUDA(launch_pdl(k_last_label<6>, grid, B, st, vp));
            } else {
                if (ppl == 4) RR_CUDA(launch_pdl(k_last_v2<7>, grid, B, st, vp));
                else RR_CUDA(launch_pdl(k_last_v2<6>, grid, B, st, vp));
            }
            timing_end(tslot, kTimeLast, st);
            RR_LAUNCHED();
            ++nk;
        }
    }
    if (side_used) {  // the branches' last layers
        RR_CUDA(cudaEventRecord(bev[2], side));
        RR_CUDA(cudaStreamWaitEvent(st, bev[2], 0));
    }
    if (bitmap) {
        RR_CUDA(launch_pdl(k_bitmap_q, dim3(grid_cap((g.n + 7) / 8, 256)), dim3(256), st, g.n, d_desc));
        RR_LAUNCHED();
        ++nk;
    }
    if (kernels) *kernels = nk;
    return RR_OK;
}

// One query with the reduced-state engine: writes the descriptor, then replays
// the captured launch sequence of the query's shape (capturing it on first use)
// or, while kernel timing is enabled, enqueues the launches directly so each
// can be timed.
rr_status reach_v2(const Graph &g, Workspace &ws, const rr_query *q, uint8_t *d_bitmap,
                   uint64_t *d_witness, uint32_t ppl, uint32_t chunk, cudaStream_t st, uint64_t *d_E,
                   const uint8_t *d_vmask, PointRange range, uint32_t bfirst, uint64_t *b_witness,
                   uint64_t *b_edges)
{
    const uint32_t k = q->k;
    RR_CUDA(ws.desc.reserve(sizeof(QueryDesc)));
    QueryDesc hd{};
    const QueryKeys keys = make_keys(q->seed);
    hd.source = q->source;
    hd.k = k;
    hd.colored = q->motif ? 1u : 0u;
    hd.key_y = keys.key_y;
    hd.key_z = keys.key_z;
    hd.key_g = keys.key_gamma;
    hd.key_o = keys.key_omega;
    hd.S = d_witness;
    hd.bitmap = d_bitmap;
    hd.E = d_E;
    hd.vmask = d_vmask;
    if (q->motif) {
        ShadeTable sh;
        make_shades(q->motif, k, &sh);
        std::memcpy(hd.shades, sh.first, sizeof sh.first);
        std::memcpy(hd.shades + 256, sh.mu, sizeof sh.mu);
    }
    const QueryDesc *dd = ws.desc.as<QueryDesc>();
    // stage the descriptor in a pinned ring slot (reused only after the launch
    // that read it has finished) and copy it in stream order
    if (!ws.h_ring) {
        RR_CUDA(cudaMallocHost(&ws.h_ring, sizeof(QueryDesc) * Workspace::kRing));
        for (int i = 0; i < Workspace::kRing; ++i)
            RR_CUDA(cudaEventCreateWithFlags(&ws.ring_ev[i], cudaEventDisableTiming));
    }
    const uint32_t slot = ws.ring_pos++ % Workspace::kRing;
    if (ws.ring_used[slot]) RR_CUDA(cudaEventSynchronize(ws.ring_ev[slot]));
    ws.h_ring[slot] = hd;
    RR_CUDA(cudaMemcpyAsync(ws.desc.p, &ws.h_ring[slot], sizeof hd, cudaMemcpyHostToDevice, st));
    ws.ring_used[slot] = true;
    const uint32_t nb = bfirst ? k - bfirst : 0;  // at-most-k branches k' = bfirst..k-1
    if (nb) {
        if (nb > Workspace::kMaxBranches) return fail(RR_EINVAL, "internal: too many at-most-k branches");
        RR_CUDA(ws.bdesc.reserve(sizeof(QueryDesc) * Workspace::kMaxBranches));
        if (!ws.h_bring)
            RR_CUDA(cudaMallocHost(&ws.h_bring, sizeof(QueryDesc) * Workspace::kRing * Workspace::kMaxBranches));
        QueryDesc *hb = ws.h_bring + (size_t)slot * Workspace::kMaxBranches;  // free with the ring slot
        for (uint32_t b = 0; b < nb; ++b) {
            hb[b] = hd;
            hb[b].k = bfirst + b;
            hb[b].S = b_witness + (size_t)b * g.n;
            hb[b].E = b_edges ? b_edges + (size_t)b * g.m : nullptr;
            hb[b].bitmap = nullptr;
        }
        RR_CUDA(cudaMemcpyAsync(ws.bdesc.p, hb, sizeof(QueryDesc) * nb, cudaMemcpyHostToDevice, st));
    }
    const QueryDesc *dbd = nb ? ws.bdesc.as<QueryDesc>() : nullptr;
    if (nb && !ws.side) {
        RR_CUDA(cudaStreamCreateWithFlags(&ws.side, cudaStreamNonBlocking));
        for (cudaEvent_t &e : ws.bev) RR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const bool table = q->motif != nullptr || d_vmask != nullptr;
    const bool bitmap = d_bitmap != nullptr;
    if (g_timing.load(std::memory_order_relaxed)) {
        rr_status s = enqueue_query_v2(g, k, table, bitmap, ppl, chunk, ws.z.as<uint64_t>(),
                                       ws.state.as<uint64_t>(), dd, st, nullptr, ws.pdl, range, dbd,
                                       nb ? bfirst : 0u, ws.side, ws.bev);
        RR_CUDA(cudaEventRecord(ws.ring_ev[slot], st));
        return s;
    }
    if (ws.graph_state != ws.state.p || ws.graph_z != ws.z.p) {
        ws.drop_graphs();
        ws.graph_state = ws.state.p;
        ws.graph_z = ws.z.p;
    }
    const std::pair<uint64_t, uint64_t> key(
        (uint64_t)k | ((uint64_t)ppl << 8) | ((uint64_t)chunk << 16) | ((uint64_t)table << 40) |
            ((uint64_t)bitmap << 41) | ((uint64_t)(nb ? bfirst : 0u) << 48),
        (uint64_t)range.first | ((uint64_t)range.stop(k) << 32));
    cudaGraphExec_t exec = nullptr;
    uint64_t nkern = 0;
    for (size_t i = 0; i < ws.graphs.size(); ++i)
        if (ws.graphs[i].first == key) {
            exec = ws.graphs[i].second;
            nkern = ws.graph_kernels[i];
        }
    if (!exec) {
        if (!ws.capture) RR_CUDA(cudaStreamCreateWithFlags(&ws.capture, cudaStreamNonBlocking));
        RR_CUDA(cudaStreamBeginCapture(ws.capture, cudaStreamCaptureModeThreadLocal));
        rr_status s = enqueue_query_v2(g, k, table, bitmap, ppl, chunk, ws.z.as<uint64_t>(),
                                       ws.state.as<uint64_t>(), dd, ws.capture, &nkern, ws.pdl,
                                       range, dbd, nb ? bfirst : 0u, ws.side, ws.bev);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ws.capture, &graph);
        if (s != RR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        ws.graphs.emplace_back(key, exec);
        ws.graph_kernels.push_back(nkern);
        g_launches.fetch_sub(nkern, std::memory_order_relaxed);  // capture launched nothing
    }
    RR_CUDA(cudaGraphLaunch(exec, st));
    RR_CUDA(cudaEventRecord(ws.ring_ev[slot], st));
    g_launches.fetch_add(nkern, std::memory_order_relaxed);
    return RR_OK;
}

}  // namespace rr
