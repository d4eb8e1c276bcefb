// rr_batch.cu -- many queries in one persistent launch, and the shape autotuner.
//
// A batch is cut into units (one query's chunk of sieve points). Units run in
// waves over `nslots` memory slots (each slot: two full prefix-state buffers
// and one transformed buffer). Every warp-sized piece of layer work -- (unit,
// layer, scheduling range, point group) -- is a task; tasks are numbered in
// the order wave, layer, unit, so a task only ever depends on tasks with
// smaller numbers:
//   layer l >= 3 of unit U needs every task of U's layers < l,
//   layer 2 of U needs every task of the unit that used U's slot before it.
// The persistent kernel's warps take task numbers from one atomic counter and
// wait (bounded, with backoff) on a per-unit completion counter before they
// start. Because a task's predecessors were all taken earlier by warps that
// are already running, the waits always end unless the device misbehaves; a
// wait that exceeds its time limit marks the query RR_ETIMEDOUT, sets an abort
// flag that makes every later task skip its work, and lets the kernel finish.
// The per-warp work is the same code as the one-query kernels
// (rr_v2_device.cuh), so results are bit-identical.
#include <algorithm>
#include <cstring>

#define RR_OUTLINED_MUL 1  // one out-of-line multiply for the many task kinds of k_batch
#include "rr_v2_device.cuh"

namespace rr {

namespace {

enum BatchKind : uint32_t {
    kSecondFull = 0,   // layer 2, window sums from the scalar prefix, full state out
    kSecondTail = 1,   // layer 2 when k = 4, transformed state out
    // 2: unused (k <= 3 queries finish in the prologue: k_batch_first2, k_batch_last3;
    // so does k = 4 in closed form: k_batch_last4)
    kMidFull = 3,      // layers 3..k-3
    kMidTail = 4,      // layer k-2 (k >= 6), transformed state out
    kLast = 5,         // layer k-1 from the transformed state
    kThirdFull = 6,    // layer 3 (k >= 6) from the label-space layer-2 prefix
    kThirdTail = 7,    // layer 3 when k = 5, transformed state out
    kLastDeep = 8,     // layer k-1 (k >= 5) from the transformed deep-row state
    kFix1 = 9,         // carry fix-up of cut segments, phase 1 (one task per cut segment)
    kFix2 = 10,        // carry fix-up, phase 2 (one task per kFixRows row slots)
    // the pair tail (k >= 8, 256-point chunks): layer k-3 writes its sums over
    // one- and two-label point sets, layer k-2 runs in label space, layer k-1
    // reads its rows
    kMidPair = 12,     // layer k-3, pair sums out
    kLabelTail = 13,   // layer k-2 in label space (one task per scheduling range)
    kLastLabel = 14    // layer k-1 from the label-space rows
};

// does a layer of this kind write prefix state (that cut segments must fix)?
__host__ __device__ inline bool writes_state(uint32_t kind)
{
    return kind == kSecondTail || kind == kThirdFull || kind == kThirdTail || kind == kMidFull ||
           kind == kMidTail || kind == kMidPair || kind == kLabelTail;
}
__host__ __device__ inline bool writes_transformed(uint32_t kind)
{
    return kind == kSecondTail || kind == kThirdTail || kind == kMidTail;
}

struct BatchUnit {
    uint32_t q, k, chunk_base, chunk, ppl, slot;
    uint32_t qi;  // the query's index in the caller's array (status slot)
};

struct BatchSeg {
    uint32_t begin, ntasks, unit, layer, kind, ngroups;
    uint32_t fixed_kind;  // kFix1/kFix2: kind of the layer whose output is fixed
    int32_t wait_unit;  // unit whose completion counter gates this segment (-1: none)
    uint32_t wait_count;
};

struct ListPtrs {
    const uint32_t *head, *eid, *src, *a0, *b0, *a1, *b1, *a3, *b3;
    const uint2 *items;
    uint32_t nitems;
    const uint2 *chains, *fix2;
    uint32_t nchains, nfix2;
};

struct BatchArgs {
    ListPtrs prod, state, tail, deep, tail3;
    uint32_t n;
    const BatchUnit *units;
    const BatchSeg *segs;
    const uint32_t *task_seg;  // segment of every task
    uint32_t nseg, total_tasks;
    const QueryDesc *descs;
    const uint64_t *z_all;
    const uint64_t *z_off;   // per query, in words
    const uint64_t *py_all;
    const uint64_t *py_off;  // per query, in words
    const uint64_t *pr2_all;
    const uint64_t *pr2_off; // per query, in words
    uint64_t *slot_base;
    uint64_t slot_words, rows, full_words;  // rows = state rows + 1; full_words = rows * max chunk
    uint64_t red_words;   // words of a slot's transformed buffer (the label-space rows follow)
    uint32_t *done;       // per unit: tasks completed
    uint32_t *ctl;        // [0] next task, [1] abort
    int32_t *status;      // per query
    uint64_t timeout_ns;
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Lane 0 waits until *ctr >= want; false if the wait timed out or the batch
// was aborted. The wait is bounded by timeout_ns of wall time and by an
// iteration cap.
__device__ bool wait_for(const BatchArgs &a, const uint32_t *ctr, uint32_t want)
{
    const uint64_t t0 = global_ns();
    uint32_t sleep = 32;
    for (uint32_t it = 0; it < 100000000u; ++it) {
        if (ld_acquire(ctr) >= want) return true;
        if (*(volatile uint32_t *)(a.ctl + 1)) return false;
        if (global_ns() - t0 > a.timeout_ns) return false;
        __nanosleep(sleep);
        if (sleep < 2048) sleep <<= 1;
    }
    return false;
}

__device__ __forceinline__ void set_list(V2Params &vp, const ListPtrs &L, int win)
{
    vp.head = L.head;
    vp.eid = L.eid;
    vp.src = L.src;
    vp.ia = win == 0 ? L.a0 : (win == 1 ? L.a1 : L.a3);
    vp.ib = win == 0 ? L.b0 : (win == 1 ? L.b1 : L.b3);
    vp.items = L.items;
    vp.nitems = L.nitems;
}

// The label-space layer of the pair tail as a call of its own: inlined, its
// live values raised the register pressure of every task kind of the kernel.
template <int LG>
__device__ __noinline__ void batch_label_tail(const V2Params vp, uint32_t item, uint64_t *sm)
{
    label_tail_warp<LG, true>(vp, item, sm);
}

template <int PPL>
__device__ __forceinline__ void run_task(const BatchArgs &a, const BatchSeg &sg, const BatchUnit &u,
                                         uint32_t local, uint64_t *sm)
{
    V2Params vp{};
    vp.qd = a.descs + u.q;
    vp.z = a.descs[u.q].colored ? a.z_all + a.z_off[u.q] : nullptr;
    vp.py = a.py_all + a.py_off[u.q];
    vp.pr2 = a.pr2_all + a.pr2_off[u.q];
    vp.n = a.n;
    vp.k = u.k;
    vp.layer = sg.layer;
    vp.chunk_base = u.chunk_base;
    vp.chunk = u.chunk;
    vp.ngroups = sg.ngroups;
    vp.npoints = 1u << u.k;
    uint64_t *full0 = a.slot_base + (size_t)u.slot * a.slot_words;
    uint64_t *full1 = full0 + a.full_words;
    uint64_t *red = full1 + a.full_words;
    uint64_t *lrows = red + a.red_words;
    uint64_t *bufs[2] = {full0, full1};
    const uint32_t l = sg.layer;
    // kinds with one task per scheduling range (no point-group split)
    const bool per_item = sg.kind == kLast || sg.kind == kLastDeep || sg.kind == kLabelTail ||
                          sg.kind == kLastLabel;
    const uint32_t item = per_item ? local : local / sg.ngroups;
    const uint32_t group = per_item ? 0u : local - item * sg.ngroups;
    constexpr int LG = PPL == 4 ? 7 : 6;
    switch (sg.kind) {
    case kSecondFull:
        set_list(vp, a.state, 0);
        vp.st_out = bufs[l & 1u];
        layer_warp<PPL, true, 0, true>(vp, item, group);
        break;
    case kSecondTail:
        set_list(vp, a.state, 0);
        vp.st_out = red;
        layer_warp<PPL, true, 1, true>(vp, item, group);
        break;
    case kThirdFull:
        set_list(vp, a.deep, 1);
        vp.st_out = bufs[l & 1u];
        layer_warp<PPL, false, 0, true, true>(vp, item, group);
        break;
    case kThirdTail:
        set_list(vp, a.deep, 1);
        vp.st_out = red;
        layer_warp<PPL, false, 1, true, true>(vp, item, group);
        break;
    case kMidFull:
        set_list(vp, a.deep, 3);
        vp.st_in = bufs[(l - 1) & 1u];
        vp.st_out = bufs[l & 1u];
        layer_warp<PPL, false, 0, true>(vp, item, group);
        break;
    case kMidTail:
        set_list(vp, a.deep, 3);
        vp.st_in = bufs[(l - 1) & 1u];
        vp.st_out = red;
        layer_warp<PPL, false, 1, true>(vp, item, group);
        break;
    case kMidPair:
        set_list(vp, a.deep, 3);
        vp.st_in = bufs[(l - 1) & 1u];
        vp.st_out = red;
        layer_warp<PPL, false, 2, true>(vp, item, group);
        break;
    case kLabelTail:
        set_list(vp, a.deep, 3);
        vp.st_in = red;
        vp.st_out = lrows;
        batch_label_tail<LG>(vp, item, sm);
        break;
    case kLastLabel:
        set_list(vp, a.tail3, 3);
        vp.st_in = lrows;
        last_label_warp<LG, true>(vp, item);
        break;
    case kFix1:
    case kFix2: {
        const ListPtrs &L = sg.fixed_kind == kSecondTail ? a.state : a.deep;
        const uint32_t fk = sg.fixed_kind;
        const bool tr = writes_transformed(fk);
        const bool pr = fk == kMidPair;
        uint64_t *buf = fk == kLabelTail ? lrows : ((tr || pr) ? red : bufs[l & 1u]);
        const uint32_t ng = u.chunk / (32u * PPL);
        const uint32_t width = fk == kLabelTail ? kLabelTailWidth
                               : pr ? ng * kPairTailSlots
                               : tr ? ng * (uint32_t)(LG + 1) : u.chunk;
        const int lane = threadIdx.x & 31;
        if (sg.kind == kFix1) {
            const uint2 ch = L.chains[local];
            fixup_phase1<true>(buf, width, ch.x, ch.y, (uint32_t)lane, 32u);
        } else {
            const uint2 t = L.fix2[local];
            const uint2 ch = L.chains[t.x];
            fixup_phase2<true>(buf, width, ch.x, ch.y, t.y, (uint32_t)lane, 32u);
        }
        break;
    }
    case kLastDeep:
        set_list(vp, a.tail3, 3);
        vp.st_in = red;
        last_warp<LG, true>(vp, item);
        break;
    default:
        set_list(vp, a.tail, 1);
        vp.st_in = red;
        last_warp<LG, true>(vp, item);
        break;
    }
}

// MINB = blocks per SM the register budget is set for: 6 (80 registers, a few
// spilled), 5 (96, fewer spilled) or 4 (128 registers) for large batches,
// where more resident warps hide the tasks' latencies; 2 (no spills) for small
// batches, whose critical path is the per-task time. The automatic rule takes
// 5 for coarse ranges (as fast as 6 within 1%, a sixth of its local-memory
// requests) and 2 for fine ones; rr_autotune_batch times all four.
template <int MINB>
__global__ void __launch_bounds__(kW2 * 32, MINB) k_batch(const BatchArgs a)
{
    const int lane = threadIdx.x & 31;
    __shared__ uint64_t sm_tail[kW2][192];  // the label-space layer's products (per warp)
    uint64_t *sm = sm_tail[threadIdx.x >> 5];
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.ctl, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.total_tasks) return;
        const BatchSeg sg = a.segs[a.task_seg[t]];
        const BatchUnit u = a.units[sg.unit];
        bool ok = true;
        if (lane == 0) {
            if (sg.wait_unit >= 0 && sg.wait_count)
                ok = wait_for(a, a.done + sg.wait_unit, sg.wait_count);
            if (!ok) atomicExch(a.ctl + 1, 1u);
            if (*(volatile uint32_t *)(a.ctl + 1)) ok = false;
            // a skipped task leaves its query's sums incomplete
            if (!ok) atomicExch(a.status + u.qi, (int32_t)RR_ETIMEDOUT);
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
            __threadfence();  // acquire side: see the predecessors' state writes
            // layer 3 writing full state takes 2 points per lane whatever the
            // unit's shape: the stored rows do not depend on the lane-to-point
            // map, and this multiply-heavy layer needs half the registers so
            if (u.ppl == 4 && sg.kind != kThirdFull) run_task<4>(a, sg, u, t - sg.begin, sm);
            else run_task<2>(a, sg, u, t - sg.begin, sm);
        }
        __threadfence();  // release side: publish this task's writes
        __syncwarp();
        if (lane == 0) atomicAdd(a.done + sg.unit, 1u);
    }
}

// Exercises wait_for on a counter that nothing increments (out[0] = 1 if the
// wait ended without the counter, out[1] = nanoseconds it took): the bounded
// wait must give up after timeout_ns, or at once when the abort flag is set,
// and leave the context usable.
__global__ void k_wait_probe(BatchArgs a, const uint32_t *ctr, uint64_t *out)
{
    if (threadIdx.x != 0) return;
    const uint64_t t0 = global_ns();
    const bool ok = wait_for(a, ctr, 1u);
    out[0] = ok ? 0ull : 1ull;
    out[1] = global_ns() - t0;
}

// Prologue / epilogue over all queries of the batch (blockIdx.y = query).
// (the vertices in colour order: a warp's shade loops have one length)
__global__ void k_batch_ztable(uint32_t n, const QueryDesc *__restrict__ descs,
                               const uint8_t *__restrict__ color, const uint32_t *__restrict__ order,
                               uint64_t *__restrict__ z_all, const uint64_t *__restrict__ z_off)
{
    const QueryDesc *qd = descs + blockIdx.y;
    const uint32_t k = qd->k;
    const bool colored = qd->colored != 0;
    if (!colored) return;  // plain queries draw z on the fly
    uint64_t *z = z_all + z_off[blockIdx.y];
    const uint64_t total = (uint64_t)n * k;
    for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pos = total <= 0xffffffffull ? (uint64_t)((uint32_t)idx / k) : idx / k;
        const uint32_t j = (uint32_t)(idx - pos * k);
        const uint64_t u = order ? order[pos] : pos;
        uint64_t val = 0;
        if (!colored) {
            val = sm_draw(qd->key_z, u * 32u + j);
        } else {
            const uint32_t c = color[u];
            const uint32_t d0 = qd->shades[c], mu = qd->shades[256 + c];
            for (uint32_t d = d0; d < d0 + mu; ++d)
                val ^= gf64_mul(sm_draw(qd->key_g, u * 32u + d), sm_draw(qd->key_o, (uint64_t)d * 32u + j));
        }
        z[u * k + j] = val;
    }
}

__global__ void __launch_bounds__(kW2 * 32)
k_batch_first(ListPtrs prod, const QueryDesc *__restrict__ descs, uint64_t *__restrict__ py_all,
              const uint64_t *__restrict__ py_off)
{
    uint64_t *py = py_all + py_off[blockIdx.y];
    if (blockIdx.x == 0 && threadIdx.x == 0) py[0] = 0;
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= prod.nitems) return;
    V2Params vp{};
    vp.qd = descs + blockIdx.y;
    vp.head = prod.head;
    vp.eid = prod.eid;
    vp.src = prod.src;
    vp.items = prod.items;
    vp.nitems = prod.nitems;
    first_scalar_warp(vp, task, py);
}

// layer 2 in label space for the batch's queries with k >= kmin (4, or 5
// with k = 4 per point), the rows across the lanes
__global__ void __launch_bounds__(kW2 * 32)
k_batch_second(ListPtrs state, const QueryDesc *__restrict__ descs, const uint64_t *__restrict__ z_all,
               const uint64_t *__restrict__ z_off, const uint64_t *__restrict__ py_all,
               const uint64_t *__restrict__ py_off, uint64_t *__restrict__ pr2_all,
               const uint64_t *__restrict__ pr2_off, uint32_t n, uint32_t kmin)
{
    const QueryDesc *qd = descs + blockIdx.y;
    const uint32_t k = qd->k;
    if (k < kmin) return;
    uint64_t *pr2 = pr2_all + pr2_off[blockIdx.y];
    if (blockIdx.x == 0 && threadIdx.x < k) pr2[threadIdx.x] = 0;
    const uint32_t task = blockIdx.x * kW2 + (threadIdx.x >> 5);
    if (task >= state.nitems) return;
    V2Params vp{};
    vp.qd = qd;
    vp.z = qd->colored ? z_all + z_off[blockIdx.y] : nullptr;
    vp.py = py_all + py_off[blockIdx.y];
    vp.n = n;
    vp.k = k;
    vp.layer = 2;
    vp.head = state.head;
    vp.eid = state.eid;
    vp.src = state.src;
    vp.ia = state.a0;
    vp.ib = state.b0;
    vp.items = state.items;
    vp.nitems = state.nitems;
    second_label_scan_warp<false>(vp, task, pr2);
}

// the batch's k = 2 queries in closed form (blockIdx.y = query)
__global__ void k_batch_first2(const QueryDesc *__restrict__ descs, const uint64_t *__restrict__ z_all,
                               const uint64_t *__restrict__ z_off, const uint32_t *__restrict__ off,
                               const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ row_eid,
                               uint32_t n, uint32_t m)
{
    const QueryDesc *qd = descs + blockIdx.y;
    if (qd->k != 2) return;
    V2Params vp{};
    vp.qd = qd;
    vp.z = qd->colored ? z_all + z_off[blockIdx.y] : nullptr;
    vp.n = n;
    vp.k = 2;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
        first2_closed(vp, off, row_src, row_eid, r);
}

// the last layer of the batch's k = 3 queries in closed form (blockIdx.y = query)
__global__ void k_batch_last3(ListPtrs win, uint32_t count, const QueryDesc *__restrict__ descs,
                              const uint64_t *__restrict__ z_all, const uint64_t *__restrict__ z_off,
                              const uint64_t *__restrict__ py_all, const uint64_t *__restrict__ py_off,
                              uint32_t n)
{
    const QueryDesc *qd = descs + blockIdx.y;
    if (qd->k != 3) return;
    V2Params vp{};
    vp.qd = qd;
    vp.z = qd->colored ? z_all + z_off[blockIdx.y] : nullptr;
    vp.py = py_all + py_off[blockIdx.y];
    vp.n = n;
    vp.k = 3;
    vp.layer = 2;
    vp.head = win.head;
    vp.eid = win.eid;
    vp.src = win.src;
    vp.ia = win.a0;
    vp.ib = win.b0;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        last3_closed(vp, e);
}

// the batch's k = 4 queries in closed form over their label-space layer 2
// (blockIdx.y = query; last4_closed, a quad of lanes per tail row)
__global__ void __launch_bounds__(256)
k_batch_last4(ListPtrs tail, uint32_t count, const QueryDesc *__restrict__ descs,
              const uint64_t *__restrict__ z_all, const uint64_t *__restrict__ z_off,
              const uint64_t *__restrict__ pr2_all, const uint64_t *__restrict__ pr2_off, uint32_t n)
{
    const QueryDesc *qd = descs + blockIdx.y;
    if (qd->k != 4) return;  // the whole block
    V2Params vp{};
    vp.qd = qd;
    vp.z = qd->colored ? z_all + z_off[blockIdx.y] : nullptr;
    vp.pr2 = pr2_all + pr2_off[blockIdx.y];
    vp.n = n;
    vp.k = 4;
    vp.layer = 3;
    vp.head = tail.head;
    vp.eid = tail.eid;
    vp.src = tail.src;
    vp.ia = tail.a1;
    vp.ib = tail.b1;
    const uint64_t zs_j = zval(vp, qd->source, threadIdx.x & 3u);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = gridDim.x * blockDim.x / 32u;
    for (uint64_t base = (uint64_t)warp * 8u; base < count; base += (uint64_t)nwarps * 8u)
        last4_closed(vp, (uint32_t)base + ((threadIdx.x & 31u) >> 2), count, zs_j);
}

__global__ void k_batch_bitmap(uint32_t n, const QueryDesc *__restrict__ descs)
{
    const QueryDesc *qd = descs + blockIdx.y;
    const uint64_t *S = qd->S;
    uint8_t *bm = qd->bitmap;
    if (!bm) return;
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

// Zero row 0 of both full buffers (width values), of the transformed buffer
// (red_width values) and of the label-space rows of every slot.
__global__ void k_batch_zero_rows(uint64_t *slot_base, uint64_t slot_words, uint64_t full_words,
                                  uint32_t nslots, uint32_t width, uint32_t red_width, uint64_t red_words)
{
    const uint32_t s = blockIdx.x;
    if (s >= nslots) return;
    uint64_t *b = slot_base + (size_t)s * slot_words;
    for (uint32_t i = threadIdx.x; i < width; i += blockDim.x) {
        b[i] = 0;
        b[full_words + i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < red_width; i += blockDim.x) b[2 * full_words + i] = 0;
    for (uint32_t i = threadIdx.x; i < kLabelTailWidth; i += blockDim.x) b[2 * full_words + red_words + i] = 0;
}

ListPtrs list_ptrs(const RowList &L, bool coarse)
{
    return ListPtrs{L.head.as<uint32_t>(), L.eid.as<uint32_t>(), L.src.as<uint32_t>(),
                    L.a0.as<uint32_t>(),   L.b0.as<uint32_t>(),  L.a1.as<uint32_t>(),
                    L.b1.as<uint32_t>(),   L.a3.as<uint32_t>(),  L.b3.as<uint32_t>(),
                    coarse ? L.items_coarse.as<uint2>() : L.items.as<uint2>(),
                    coarse ? L.nitems_coarse : L.nitems,
                    L.chains.as<uint2>(),  L.fix2.as<uint2>(),   L.nchains, L.nfix2};
}

// prologue fix-ups of the per-query scalar (width 1, label_space 0) or
// label-space (width k, queries with k >= label_space only) prefixes:
// blockIdx.y = query
__global__ void k_batch_fix1(ListPtrs L, uint64_t *base, const uint64_t *__restrict__ off,
                             const QueryDesc *__restrict__ descs, int label_space)
{
    if (blockIdx.x >= L.nchains) return;
    const uint32_t k = descs[blockIdx.y].k;
    if (label_space && k < (uint32_t)label_space) return;
    const uint2 ch = L.chains[blockIdx.x];
    fixup_phase1<false>(base + off[blockIdx.y], label_space ? k : 1u, ch.x, ch.y, threadIdx.x,
                        blockDim.x);
}

__global__ void k_batch_fix2(ListPtrs L, uint64_t *base, const uint64_t *__restrict__ off,
                             const QueryDesc *__restrict__ descs, int label_space)
{
    if (blockIdx.x >= L.nfix2) return;
    const uint32_t k = descs[blockIdx.y].k;
    if (label_space && k < (uint32_t)label_space) return;
    const uint2 t = L.fix2[blockIdx.x];
    const uint2 ch = L.chains[t.x];
    fixup_phase2<false>(base + off[blockIdx.y], label_space ? k : 1u, ch.x, ch.y, t.y, threadIdx.x,
                        blockDim.x);
}

static rr_status batch_fixup(const ListPtrs &L, uint64_t *base, const uint64_t *off,
                             const QueryDesc *descs, uint32_t nq, int label_space, cudaStream_t st)
{
    if (!L.nchains) return RR_OK;
    k_batch_fix1<<<dim3(L.nchains, nq), 128, 0, st>>>(L, base, off, descs, label_space);
    RR_LAUNCHED();
    if (L.nfix2) {
        k_batch_fix2<<<dim3(L.nfix2, nq), 256, 0, st>>>(L, base, off, descs, label_space);
        RR_LAUNCHED();
    }
    return RR_OK;
}

// Tasks of layer l of a unit with (k, ppl, chunk), over the coarse or the fine
// scheduling ranges of the layer's row list.
uint32_t layer_tasks(const Graph &g, uint32_t k, uint32_t l, uint32_t chunk, uint32_t ngroups,
                     bool coarse, uint32_t *kind)
{
    auto items = [coarse](const RowList &L) { return coarse ? L.nitems_coarse : L.nitems; };
    if (k <= 3) return 0;  // closed forms in the prologue
    // the pair tail, from 512-point units here (k >= 9; layer k-3 >= 6 is a
    // middle layer): the label-space layer runs one warp per scheduling range,
    // which costs more in the batch's dependency chains than in a one-query
    // launch (256-point units of k = 8 queries were 3% slower with it)
    const bool ptail = !g.pair_tail_off && k >= 9 && chunk >= 2 * kPairTailMinChunk &&
                       ngroups <= kPairTailMaxGroups;
    if (l == k - 1) {
        *kind = k == 4 ? kLast : (ptail ? kLastLabel : kLastDeep);
        return k == 4 ? items(g.tail_list) : items(g.tail3_list);
    }
    if (ptail && l == k - 2) {
        *kind = kLabelTail;
        return items(g.deep_list);
    }
    if (ptail && l == k - 3) {
        *kind = kMidPair;
        return items(g.deep_list) * ngroups;
    }
    if (l == 2) {
        if (k >= 5) return 0;  // label-space layer 2 runs in the prologue
        *kind = kSecondTail;   // k = 4
        return items(g.state_list) * ngroups;
    }
    *kind = l == 3 ? ((k == 5) ? kThirdTail : kThirdFull) : ((l == k - 2) ? kMidTail : kMidFull);
    return items(g.deep_list) * ngroups;
}

}  // namespace

// Values a transformed row holds in a slot of max chunk `chunk`: a 32-value
// block of pair sums per lane group of 128 points (4 points per lane; the sums
// over single labels take 8), one block for a 64-point group (2 points per
// lane).
static uint64_t red_words_for(uint32_t chunk)
{
    return std::max<uint64_t>(kPairTailSlots, (chunk + 127) / 128 * kPairTailSlots);
}

// Words of a slot's transformed buffer for max chunk `chunk`.
static uint64_t red_buffer_words(const Graph &g, uint32_t chunk)
{
    const uint64_t srows = g.state_list.count + 1, drows = g.deep_list.count + 1;
    return std::max(srows, drows) * red_words_for(chunk);
}

// Words of device memory one batch slot holds for max chunk `chunk`: two full
// buffers, the transformed buffer, the pair tail's label-space rows.
static uint64_t slot_words_for(const Graph &g, uint32_t chunk)
{
    const uint64_t drows = g.deep_list.count + 1;
    return drows * chunk * 2 + red_buffer_words(g, chunk) + drows * kLabelTailWidth;
}

rr_status batch_device(const Graph &g, const rr_query *qs, uint32_t nq, uint8_t *d_bitmaps,
                       uint64_t *d_witness, int32_t *d_status, cudaStream_t st)
{
    if (nq == 0) return RR_OK;
    const size_t nb = (g.n + 7) / 8;
    if (d_status) RR_CUDA(cudaMemsetAsync(d_status, 0, (size_t)nq * 4, st));
    // graphs on the per-point engine run one query at a time
    std::vector<uint32_t> bq;
    for (uint32_t i = 0; i < nq; ++i) {
        if (uses_v2(g, qs[i].k)) {
            bq.push_back(i);
            continue;
        }
        rr_status s = reach_on_stream(g, g.ws, &qs[i], d_bitmaps ? d_bitmaps + i * nb : nullptr,
                                      d_witness + (size_t)i * g.n, 0, st);
        if (s != RR_OK) return s;
    }
    if (bq.empty()) return RR_OK;

    BatchBuffers &B = g.batch;
    size_t free_b = 0, total_b = 0;
    RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    uint64_t budget = (uint64_t)(0.6 * (double)free_b);
    const uint64_t rows = g.state_list.count + 1;
    const uint64_t py_words = (g.prod_list.count + 1 + 31) / 32 * 32;

    // queries are processed in groups whose z-tables and prefixes fit half the budget
    size_t gi = 0;
    while (gi < bq.size()) {
        std::vector<uint32_t> grp;
        uint64_t qbytes = 0;
        while (gi < bq.size()) {
            const uint64_t need = ((qs[bq[gi]].motif ? (uint64_t)g.n * qs[bq[gi]].k : 0ull) + 64 +
                                   py_words + rows * qs[bq[gi]].k) * 8;
            if (!grp.empty() && qbytes + need > budget / 2) break;
            qbytes += need;
            grp.push_back(bq[gi++]);
        }
        // largest point chunk (<= 512, or the tuned one) for which at least one
        // slot fits the rest
        uint32_t max_chunk = g.batch_max_chunk ? g.batch_max_chunk : 512;
        // (not below 128: a query with 4 points per lane takes 128-point chunks)
        while (max_chunk > 128 && slot_words_for(g, max_chunk) * 8 > budget - std::min(budget, qbytes))
            max_chunk >>= 1;
        if (slot_words_for(g, max_chunk) * 8 + qbytes > budget)
            return fail(RR_ENOMEM, "rr_reach_batch_device: one query and one slot do not fit device memory");

        // units
        std::vector<BatchUnit> units;
        // the smallest k with a label-space layer 2 (k = 4 in closed form unless the
        // load flags keep it per point)
        const uint32_t kmin2 = g.k4_per_point ? 5u : 4u;
        std::vector<QueryDesc> descs(grp.size());
        std::vector<uint64_t> z_off(grp.size()), py_off(grp.size()), pr2_off(grp.size());
        uint64_t zw = 0, pr2w = 0;
        for (size_t j = 0; j < grp.size(); ++j) {
            const rr_query &q = qs[grp[j]];
            QueryDesc &hd = descs[j];
            std::memset(&hd, 0, sizeof hd);
            const QueryKeys keys = make_keys(q.seed);
            hd.source = q.source;
            hd.k = q.k;
            hd.colored = q.motif ? 1u : 0u;
            hd.key_y = keys.key_y;
            hd.key_z = keys.key_z;
            hd.key_g = keys.key_gamma;
            hd.key_o = keys.key_omega;
            hd.S = d_witness + (size_t)grp[j] * g.n;
            hd.bitmap = d_bitmaps ? d_bitmaps + (size_t)grp[j] * nb : nullptr;
            if (q.motif) {
                ShadeTable sh;
                make_shades(q.motif, q.k, &sh);
                std::memcpy(hd.shades, sh.first, sizeof sh.first);
                std::memcpy(hd.shades + 256, sh.mu, sizeof sh.mu);
            }
            z_off[j] = zw;
            if (q.motif) zw += ((uint64_t)g.n * q.k + 31) / 32 * 32;
            py_off[j] = j * py_words;
            pr2_off[j] = pr2w;
            if (q.k >= kmin2) pr2w += (rows * q.k + 31) / 32 * 32;
            const uint64_t npts = 1ull << q.k;
            const uint32_t ppl = npts >= 128 ? 4u : 2u;
            uint32_t chunk = (uint32_t)std::max<uint64_t>(32ull * ppl, std::min<uint64_t>(npts, max_chunk));
            chunk = std::max<uint32_t>(chunk, 32u * ppl);
            // k <= 3 and k = 4 in closed form finish in the prologue
            const bool prologue = q.k <= 3 || (q.k == 4 && kmin2 == 4);
            const uint64_t nch = prologue ? 0 : (npts + chunk - 1) / chunk;
            for (uint64_t c = 0; c < nch; ++c)
                units.push_back(BatchUnit{(uint32_t)j, q.k, (uint32_t)(c * chunk), chunk, ppl, 0,
                                          grp[j]});
        }
        // Coarse ranges (about 32 entries) keep the task count of large batches
        // low; a batch whose first wave would leave resident warps without a
        // task even at the deepest layers takes the fine ranges (one head run
        // each), which shorten each layer's critical path.
        if (!B.occupancy[2]) {
            int dev = 0;
            RR_CUDA(cudaGetDevice(&dev));
            RR_CUDA(cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, dev));
            RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B.occupancy[2], k_batch<2>, kW2 * 32, 0));
            RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B.occupancy[4], k_batch<4>, kW2 * 32, 0));
            RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B.occupancy[5], k_batch<5>, kW2 * 32, 0));
            RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B.occupancy[6], k_batch<6>, kW2 * 32, 0));
            for (int v : {2, 4, 5, 6}) B.occupancy[v] = std::max(1, B.occupancy[v]);
        }
        const uint64_t resident_warps = (uint64_t)B.sms * B.occupancy[2] * kW2;
        const uint64_t slot_bytes = slot_words_for(g, max_chunk) * 8;
        // as many slots as memory allows (up to every unit at once): units in
        // flight together hide each other's layer-to-layer dependencies
        uint32_t nslots = (uint32_t)std::min<uint64_t>(
            {(uint64_t)units.size(), 4096ull, (budget - qbytes) / slot_bytes});
        nslots = std::max<uint32_t>(1, nslots);
        for (size_t i = 0; i < units.size(); ++i) units[i].slot = (uint32_t)(i % nslots);
        uint64_t wave_tasks = 0;
        for (size_t i = 0; i < std::min<size_t>(units.size(), nslots); ++i)
            wave_tasks += (uint64_t)g.deep_list.nitems_coarse * (units[i].chunk / (32u * units[i].ppl));
        const bool coarse = g.batch_ranges ? g.batch_ranges == 2 : 2 * wave_tasks >= resident_warps;
        const int minb = g.batch_minb ? (int)g.batch_minb : (coarse ? 5 : 2);

        // segments in task order: wave, layer, unit; after a layer that writes
        // prefix state, the unit's carry fix-up segments (phase 1, phase 2)
        std::vector<BatchSeg> segs;
        std::vector<char> started(units.size(), 0);
        std::vector<uint32_t> emitted(units.size(), 0);  // tasks emitted so far per unit
        uint64_t total = 0;
        auto emit = [&](size_t i, uint32_t l, uint32_t kind, uint32_t nt, uint32_t ngroups,
                        uint32_t fixed_kind) {
            BatchSeg sg{};
            sg.begin = (uint32_t)total;
            sg.ntasks = nt;
            sg.unit = (uint32_t)i;
            sg.layer = l;
            sg.kind = kind;
            sg.ngroups = ngroups;
            sg.fixed_kind = fixed_kind;
            if (!started[i]) {
                // the unit's first layer reuses the slot: wait for the unit that
                // held it before to finish
                started[i] = 1;
                const long prev = (long)i - (long)nslots;
                sg.wait_unit = prev >= 0 ? (int32_t)prev : -1;
                sg.wait_count = prev >= 0 ? emitted[prev] : 0;
            } else {
                sg.wait_unit = (int32_t)i;
                sg.wait_count = emitted[i];
            }
            segs.push_back(sg);
            total += nt;
            emitted[i] += nt;
        };
        for (size_t w0 = 0; w0 < units.size(); w0 += nslots) {
            const size_t w1 = std::min(units.size(), w0 + nslots);
            uint32_t maxl = 0;
            for (size_t i = w0; i < w1; ++i) maxl = std::max(maxl, units[i].k - 1);
            for (uint32_t l = 2; l <= maxl; ++l)
                for (size_t i = w0; i < w1; ++i) {
                    const BatchUnit &u = units[i];
                    if (l > u.k - 1) continue;
                    uint32_t ngroups = u.chunk / (32u * u.ppl);
                    uint32_t kind;
                    uint32_t nt = layer_tasks(g, u.k, l, u.chunk, ngroups, coarse, &kind);
                    if (nt == 0) continue;
                    if (kind == kThirdFull && u.ppl == 4) {
                        // layer 3 runs with 2 points per lane (see run_task)
                        ngroups *= 2;
                        nt *= 2;
                    }
                    emit(i, l, kind, nt, ngroups, 0);
                    if (writes_state(kind)) {
                        const RowList &L = kind == kSecondTail ? g.state_list : g.deep_list;
                        if (L.nchains) emit(i, l, kFix1, L.nchains, ngroups, kind);
                        if (L.nfix2) emit(i, l, kFix2, L.nfix2, ngroups, kind);
                    }
                }
        }
        if (total >= (1ull << 32)) return fail(RR_EINVAL, "rr_reach_batch_device: batch too large");
        std::vector<uint32_t> task_seg(total);
        for (size_t si = 0; si < segs.size(); ++si)
            std::fill(task_seg.begin() + segs[si].begin, task_seg.begin() + segs[si].begin + segs[si].ntasks,
                      (uint32_t)si);

        // device buffers (kept by the graph and grown as needed)
        RR_CUDA(B.units.reserve(units.size() * sizeof(BatchUnit)));
        RR_CUDA(B.segs.reserve(std::max<size_t>(1, segs.size()) * sizeof(BatchSeg)));
        RR_CUDA(B.descs.reserve(descs.size() * sizeof(QueryDesc)));
        RR_CUDA(B.zoff.reserve(grp.size() * 8));
        RR_CUDA(B.pyoff.reserve(grp.size() * 8));
        RR_CUDA(B.z.reserve(std::max<uint64_t>(1, zw) * 8));
        RR_CUDA(B.py.reserve(grp.size() * py_words * 8));
        RR_CUDA(B.pr2.reserve(std::max<uint64_t>(1, pr2w) * 8));
        RR_CUDA(B.pr2off.reserve(grp.size() * 8));
        RR_CUDA(B.slots.reserve((size_t)nslots * slot_bytes));
        RR_CUDA(B.done.reserve(units.size() * 4));
        RR_CUDA(B.ctl.reserve(8));
        RR_CUDA(B.task_seg.reserve(std::max<size_t>(1, task_seg.size()) * 4));
        if (!d_status) RR_CUDA(B.status.reserve((size_t)nq * 4));
        int32_t *status = d_status ? d_status : B.status.as<int32_t>();
        if (!d_status) RR_CUDA(cudaMemsetAsync(status, 0, (size_t)nq * 4, st));
        DevBuf &d_units = B.units, &d_segs = B.segs, &d_descs = B.descs, &d_zoff = B.zoff,
               &d_pyoff = B.pyoff, &d_z = B.z, &d_py = B.py, &d_slots = B.slots, &d_done = B.done,
               &d_ctl = B.ctl;
        {
            // pack the plan into pinned staging memory and upload it asynchronously
            struct Part {
                const void *src;
                size_t bytes;
                void *dst;
            } parts[] = {
                {units.data(), units.size() * sizeof(BatchUnit), d_units.p},
                {segs.data(), segs.size() * sizeof(BatchSeg), d_segs.p},
                {descs.data(), descs.size() * sizeof(QueryDesc), d_descs.p},
                {z_off.data(), grp.size() * 8, d_zoff.p},
                {py_off.data(), grp.size() * 8, d_pyoff.p},
                {pr2_off.data(), grp.size() * 8, B.pr2off.p},
                {task_seg.data(), task_seg.size() * 4, B.task_seg.p},
            };
            size_t need = 0;
            for (const Part &pt : parts) need += (pt.bytes + 255) / 256 * 256;
            if (B.stage_pending) {
                RR_CUDA(cudaEventSynchronize(B.stage_ev));
                B.stage_pending = false;
            }
            if (need > B.h_cap) {
                if (B.h_stage) cudaFreeHost(B.h_stage);
                B.h_stage = nullptr;
                B.h_cap = 0;
                RR_CUDA(cudaMallocHost(&B.h_stage, need));
                B.h_cap = need;
            }
            if (!B.stage_ev) RR_CUDA(cudaEventCreateWithFlags(&B.stage_ev, cudaEventDisableTiming));
            size_t off = 0;
            for (const Part &pt : parts) {
                if (pt.bytes) {
                    std::memcpy(B.h_stage + off, pt.src, pt.bytes);
                    RR_CUDA(cudaMemcpyAsync(pt.dst, B.h_stage + off, pt.bytes, cudaMemcpyHostToDevice, st));
                }
                off += (pt.bytes + 255) / 256 * 256;
            }
            RR_CUDA(cudaEventRecord(B.stage_ev, st));
            B.stage_pending = true;
        }
        RR_CUDA(cudaMemsetAsync(d_done.p, 0, units.size() * 4, st));
        RR_CUDA(cudaMemsetAsync(d_ctl.p, 0, 8, st));
        for (uint32_t j : grp) RR_CUDA(cudaMemsetAsync(d_witness + (size_t)j * g.n, 0, (size_t)g.n * 8, st));

        const unsigned gz = (unsigned)std::min<uint64_t>(1024, ((uint64_t)g.n * 20 + 255) / 256);
        int tslot = timing_begin(st);
        k_batch_ztable<<<dim3(gz, (unsigned)grp.size()), 256, 0, st>>>(
            g.n, d_descs.as<QueryDesc>(), g.color.as<uint8_t>(), g.color_order.as<uint32_t>(),
            d_z.as<uint64_t>(), d_zoff.as<uint64_t>());
        timing_end(tslot, kTimeZ, st);
        RR_LAUNCHED();
        const ListPtrs prod = list_ptrs(g.prod_list, false);
        tslot = timing_begin(st);
        k_batch_first<<<dim3(std::max<uint32_t>(1, (prod.nitems + kW2 - 1) / kW2), (unsigned)grp.size()),
                        kW2 * 32, 0, st>>>(prod, d_descs.as<QueryDesc>(), d_py.as<uint64_t>(),
                                           d_pyoff.as<uint64_t>());
        timing_end(tslot, kTimeFirst, st);
        RR_LAUNCHED();
        {
            rr_status fs = batch_fixup(prod, d_py.as<uint64_t>(), d_pyoff.as<uint64_t>(),
                                       d_descs.as<QueryDesc>(), (uint32_t)grp.size(), 0, st);
            if (fs != RR_OK) return fs;
        }
        tslot = timing_begin(st);
        k_batch_second<<<dim3(std::max<uint32_t>(1, (g.state_list.nitems + kW2 - 1) / kW2),
                              (unsigned)grp.size()),
                         kW2 * 32, 0, st>>>(list_ptrs(g.state_list, false), d_descs.as<QueryDesc>(),
                                            d_z.as<uint64_t>(), d_zoff.as<uint64_t>(),
                                            d_py.as<uint64_t>(), d_pyoff.as<uint64_t>(),
                                            B.pr2.as<uint64_t>(), B.pr2off.as<uint64_t>(), g.n, kmin2);
        timing_end(tslot, kTimeSecond, st);
        RR_LAUNCHED();
        {
            rr_status fs = batch_fixup(list_ptrs(g.state_list, false), B.pr2.as<uint64_t>(),
                                       B.pr2off.as<uint64_t>(), d_descs.as<QueryDesc>(),
                                       (uint32_t)grp.size(), (int)kmin2, st);
            if (fs != RR_OK) return fs;
        }
        bool any2 = false, any3 = false, any4 = false;
        for (uint32_t j : grp) {
            any2 |= qs[j].k == 2;
            any3 |= qs[j].k == 3;
            any4 |= qs[j].k == 4 && kmin2 == 4;
        }
        if (any4 && g.tail_list.count) {
            const uint32_t cnt = (uint32_t)g.tail_list.count;
            const int t4 = timing_begin(st);
            k_batch_last4<<<dim3(std::min<uint32_t>(2048, (uint32_t)(((uint64_t)cnt + 7) / 8 * 32 + 255) / 256),
                                 (unsigned)grp.size()),
                            256, 0, st>>>(list_ptrs(g.tail_list, false), cnt, d_descs.as<QueryDesc>(),
                                          d_z.as<uint64_t>(), d_zoff.as<uint64_t>(), B.pr2.as<uint64_t>(),
                                          B.pr2off.as<uint64_t>(), g.n);
            timing_end(t4, kTimeLast, st);
            RR_LAUNCHED();
        }
        if (any2 && g.m) {
            const uint32_t m32 = (uint32_t)g.m;
            const int t2 = timing_begin(st);
            k_batch_first2<<<dim3(std::min<uint32_t>(2048, (m32 + 255) / 256), (unsigned)grp.size()), 256, 0,
                             st>>>(d_descs.as<QueryDesc>(), d_z.as<uint64_t>(), d_zoff.as<uint64_t>(),
                                   g.off.as<uint32_t>(), g.row_src.as<uint32_t>(), g.row_eid.as<uint32_t>(),
                                   g.n, m32);
            timing_end(t2, kTimeFirst, st);
            RR_LAUNCHED();
        }
        if (any3 && g.win_list.count) {
            const uint32_t cnt = (uint32_t)g.win_list.count;
            const int t3 = timing_begin(st);
            k_batch_last3<<<dim3(std::min<uint32_t>(2048, (cnt + 255) / 256), (unsigned)grp.size()), 256, 0,
                            st>>>(list_ptrs(g.win_list, false), cnt, d_descs.as<QueryDesc>(),
                                  d_z.as<uint64_t>(), d_zoff.as<uint64_t>(), d_py.as<uint64_t>(),
                                  d_pyoff.as<uint64_t>(), g.n);
            timing_end(t3, kTimeLast, st);
            RR_LAUNCHED();
        }
        k_batch_zero_rows<<<nslots, 256, 0, st>>>(d_slots.as<uint64_t>(), slot_bytes / 8,
                                                  (g.deep_list.count + 1) * max_chunk, nslots,
                                                  max_chunk, (uint32_t)red_words_for(max_chunk),
                                                  red_buffer_words(g, max_chunk));
        RR_LAUNCHED();

        BatchArgs a{};
        a.prod = prod;
        a.state = list_ptrs(g.state_list, coarse);
        a.tail = list_ptrs(g.tail_list, coarse);
        a.deep = list_ptrs(g.deep_list, coarse);
        a.tail3 = list_ptrs(g.tail3_list, coarse);
        a.n = g.n;
        a.units = d_units.as<BatchUnit>();
        a.segs = d_segs.as<BatchSeg>();
        a.nseg = (uint32_t)segs.size();
        a.task_seg = B.task_seg.as<uint32_t>();
        a.total_tasks = (uint32_t)total;
        a.descs = d_descs.as<QueryDesc>();
        a.z_all = d_z.as<uint64_t>();
        a.z_off = d_zoff.as<uint64_t>();
        a.py_all = d_py.as<uint64_t>();
        a.py_off = d_pyoff.as<uint64_t>();
        a.pr2_all = B.pr2.as<uint64_t>();
        a.pr2_off = B.pr2off.as<uint64_t>();
        a.slot_base = d_slots.as<uint64_t>();
        a.slot_words = slot_bytes / 8;
        a.rows = rows;
        a.full_words = (g.deep_list.count + 1) * max_chunk;
        a.red_words = red_buffer_words(g, max_chunk);
        a.done = d_done.as<uint32_t>();
        a.ctl = d_ctl.as<uint32_t>();
        a.status = status;
        a.timeout_ns = 2000000000ull;
        if (total) {
            const unsigned blocks = (unsigned)std::max(1, B.sms * B.occupancy[minb]);
            const int bslot = timing_begin(st);
            if (minb == 6) k_batch<6><<<blocks, kW2 * 32, 0, st>>>(a);
            else if (minb == 5) k_batch<5><<<blocks, kW2 * 32, 0, st>>>(a);
            else if (minb == 4) k_batch<4><<<blocks, kW2 * 32, 0, st>>>(a);
            else k_batch<2><<<blocks, kW2 * 32, 0, st>>>(a);
            timing_end(bslot, kTimeBatch, st);
            RR_LAUNCHED();
        }
        if (d_bitmaps) {
            k_batch_bitmap<<<dim3((unsigned)std::min<uint64_t>(256, (nb + 255) / 256), (unsigned)grp.size()),
                             256, 0, st>>>(g.n, d_descs.as<QueryDesc>());
            RR_LAUNCHED();
        }
    }
    return RR_OK;
}

// bitmap of the union of `rows` witness rows (row-major, n each)
__global__ void k_union_bitmap(const uint64_t *__restrict__ W, uint32_t rows, uint32_t n,
                               uint8_t *__restrict__ bm)
{
    const uint32_t nb = (n + 7) / 8;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t i = 0; i < 8; ++i) {
            const uint32_t v = b * 8 + i;
            if (v >= n) break;
            for (uint32_t r = 0; r < rows; ++r)
                if (W[(size_t)r * n + v]) {
                    bits |= 1u << i;
                    break;
                }
        }
        bm[b] = (uint8_t)bits;
    }
}

// Lane j of the fan-out runs the query with k' = k - j of a call: the longest
// chain gets the highest stream priority. Lanes launch without programmatic
// dependencies (with several concurrent streams a waiting grid would hold SM
// slots the other lanes could use).
rr_status ensure_fan_lanes(const Graph &g, uint32_t lanes)
{
    FanOut &F = g.fan;
    if (!F.fork) RR_CUDA(cudaEventCreateWithFlags(&F.fork, cudaEventDisableTiming));
    int prio_least = 0, prio_greatest = 0;
    RR_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    while (F.ws.size() < lanes) {
        const int prio = std::min(prio_least, prio_greatest + (int)F.ws.size());
        cudaStream_t s2 = nullptr;
        cudaEvent_t e2 = nullptr;
        RR_CUDA(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio));
        F.st.push_back(s2);
        RR_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        F.done.push_back(e2);
        F.ws.emplace_back(new Workspace());
        F.ws.back()->pdl = false;
    }
    return RR_OK;
}

// Runs the persistent kernel's bounded wait on a counter that is never
// incremented (see k_wait_probe); synchronous.
rr_status debug_wait_probe(uint64_t timeout_ns, int abort_preset, int32_t *status,
                           uint64_t *elapsed_ns)
{
    if (!status || !elapsed_ns) return fail(RR_EINVAL, "rr_debug_wait_probe: NULL argument");
    if (timeout_ns > 10000000000ull) return fail(RR_EINVAL, "rr_debug_wait_probe: timeout above 10 s");
    DevBuf buf;
    RR_CUDA(buf.reserve(32));  // [0] counter, [1] next task, [2] abort flag, [4..7] out
    uint32_t *w = buf.as<uint32_t>();
    RR_CUDA(cudaMemset(buf.p, 0, 32));
    if (abort_preset) {
        const uint32_t one = 1;
        RR_CUDA(cudaMemcpy(w + 2, &one, 4, cudaMemcpyHostToDevice));
    }
    BatchArgs a{};
    a.ctl = w + 1;  // ctl[1] is the abort flag
    a.timeout_ns = timeout_ns;
    uint64_t *out = reinterpret_cast<uint64_t *>(w + 4);
    k_wait_probe<<<1, 32>>>(a, w, out);
    RR_LAUNCHED();
    uint64_t h[2] = {0, 0};
    RR_CUDA(cudaMemcpy(h, out, 16, cudaMemcpyDeviceToHost));
    *status = h[0] ? (int32_t)RR_ETIMEDOUT : (int32_t)RR_OK;
    *elapsed_ns = h[1];
    return RR_OK;
}

// at-most-k (Algorithm 2 stopped at k): the exact-k' queries for k' = 2..k,
// row k'-2 of d_witness each. For one seed the k'-vertex query's per-point
// layers agree with the k-vertex query's on the first 2^k' points, so on the
// reduced-state engine the k query also yields k' = atmost_first_branch..k-1
// (its per-point layer k'-2 as their tail: enqueue_query_v2's branches); the
// rest run concurrently, one lane (workspace and stream) each, largest k'
// first and on the stream of highest priority, forked from and joined back to
// `st`. If the scratch of all lanes does not fit 60% of free device memory the
// queries run in order on the graph's own workspace instead.
rr_status atmost_device(const Graph &g, uint32_t source, uint32_t k, uint64_t seed,
                        uint8_t *d_bitmap, uint64_t *d_witness, cudaStream_t st)
{
    const uint32_t lanes = k - 1;
    size_t free_b = 0, total_b = 0;
    RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t per_lane = (uint64_t)(0.6 * (double)(free_b + g.fan.bytes())) / lanes;
    uint64_t need = 0;
    for (uint32_t kk = 2; kk <= k; ++kk) {
        const uint64_t b = query_scratch_bytes(g, kk, per_lane);
        need = (b == UINT64_MAX || need == UINT64_MAX) ? UINT64_MAX : need + b;
    }
    if (need == UINT64_MAX) {
        for (uint32_t kk = 2; kk <= k; ++kk) {
            const rr_query q{source, kk, seed, nullptr};
            rr_status s = reach_on_stream(g, g.ws, &q, nullptr, d_witness + (size_t)(kk - 2) * g.n, 0, st);
            if (s != RR_OK) return s;
        }
    } else {
        FanOut &F = g.fan;
        rr_status ls = ensure_fan_lanes(g, lanes);
        if (ls != RR_OK) return ls;
        // k' = bfirst..k-1 come from the k query's own layers (lane 0), the
        // smaller k' run on their own lanes
        const uint32_t bfirst = atmost_branches(g, k);
        RR_CUDA(cudaEventRecord(F.fork, st));
        for (uint32_t kk = k; kk >= 2; --kk) {
            if (bfirst && kk >= bfirst && kk < k) continue;
            const uint32_t j = k - kk;  // lane
            const rr_query q{source, kk, seed, nullptr};
            RR_CUDA(cudaStreamWaitEvent(F.st[j], F.fork, 0));
            rr_status s;
            if (kk == k && bfirst) {
                uint64_t *bw = d_witness + (size_t)(bfirst - 2) * g.n;
                RR_CUDA(cudaMemsetAsync(bw, 0, (size_t)(k - bfirst) * g.n * 8, F.st[j]));
                s = reach_on_stream(g, *F.ws[j], &q, nullptr, d_witness + (size_t)(kk - 2) * g.n, per_lane,
                                    F.st[j], nullptr, nullptr, nullptr, PointRange(), bfirst, bw, nullptr);
            } else {
                s = reach_on_stream(g, *F.ws[j], &q, nullptr, d_witness + (size_t)(kk - 2) * g.n, per_lane,
                                    F.st[j]);
            }
            RR_CUDA(cudaEventRecord(F.done[j], F.st[j]));
            RR_CUDA(cudaStreamWaitEvent(st, F.done[j], 0));
            if (s != RR_OK) return s;
        }
    }
    if (d_bitmap) {
        const uint32_t nb = (g.n + 7) / 8;
        k_union_bitmap<<<std::max<uint32_t>(1, std::min<uint32_t>(1024, (nb + 255) / 256)), 256, 0, st>>>(
            d_witness, k - 1, g.n, d_bitmap);
        RR_LAUNCHED();
    }
    return RR_OK;
}

// Times each candidate (points per lane, points per chunk) on a plain query of
// size k from vertex 0 -- the best of interleaved rounds of about 2 ms of
// queries each -- and keeps the fastest.
// Times the persistent batch on `qs` for every shape candidate -- kernel
// variant (2, 4 or 6 blocks per SM), fine or coarse scheduling ranges, largest
// point chunk 256, 512 or 1024 -- best of two runs each after one untimed run, and
// keeps the fastest in the graph (every later batch on the graph, and the
// server's batch lanes, use it). Results do not depend on the shape.
rr_status autotune_batch(Graph &g, const rr_query *qs, uint32_t nq, uint32_t *minb,
                         uint32_t *ranges, uint32_t *max_chunk)
{
    DevBuf W;
    RR_CUDA(W.reserve((size_t)nq * g.n * 8));
    cudaEvent_t e0, e1;
    RR_CUDA(cudaEventCreate(&e0));
    RR_CUDA(cudaEventCreate(&e1));
    const uint32_t save[3] = {g.batch_minb, g.batch_ranges, g.batch_max_chunk};
    uint32_t best[3] = {0, 0, 0};
    float best_ms = 1e30f;
    rr_status st = RR_OK;
    for (uint32_t mb : {2u, 4u, 5u, 6u})
        for (uint32_t rg : {1u, 2u})
            for (uint32_t mc : {256u, 512u, 1024u}) {
                g.batch_minb = mb;
                g.batch_ranges = rg;
                g.batch_max_chunk = mc;
                float cand = 1e30f;
                for (int rep = 0; rep < 3 && st == RR_OK; ++rep) {
                    RR_CUDA(cudaEventRecord(e0, g.stream));
                    st = batch_device(g, qs, nq, nullptr, W.as<uint64_t>(), nullptr, g.stream);
                    RR_CUDA(cudaEventRecord(e1, g.stream));
                    RR_CUDA(cudaEventSynchronize(e1));
                    float ms = 0;
                    RR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0) cand = std::min(cand, ms);
                }
                if (st != RR_OK) break;
                if (cand < best_ms) {
                    best_ms = cand;
                    best[0] = mb;
                    best[1] = rg;
                    best[2] = mc;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RR_OK) {
        g.batch_minb = save[0];
        g.batch_ranges = save[1];
        g.batch_max_chunk = save[2];
        return st;
    }
    g.batch_minb = best[0];
    g.batch_ranges = best[1];
    g.batch_max_chunk = best[2];
    if (minb) *minb = best[0];
    if (ranges) *ranges = best[1];
    if (max_chunk) *max_chunk = best[2];
    return RR_OK;
}

rr_status autotune(Graph &g, uint32_t k, uint32_t *best_ppl, uint32_t *best_chunk)
{
    const uint64_t npts = 1ull << k;
    struct Cand { uint32_t ppl, chunk; };
    std::vector<Cand> cands;
    for (uint32_t ppl : {2u, 4u})
        for (uint32_t chunk : {64u, 128u, 256u, 512u, 1024u, 2048u}) {
            if (chunk % (32u * ppl)) continue;
            if (chunk > std::max<uint64_t>(npts, 32u * ppl)) continue;
            cands.push_back({ppl, chunk});
        }
    DevBuf S;
    RR_CUDA(S.reserve((size_t)g.n * 8));
    cudaEvent_t e0, e1;
    RR_CUDA(cudaEventCreate(&e0));
    RR_CUDA(cudaEventCreate(&e1));
    rr_query q{0, k, 0x7E57ull, nullptr};
    const uint32_t save_ppl = g.tune_ppl[k], save_chunk = g.tune_chunk[k];
    auto set_shape = [&](const Cand &c) {
        g.tune_ppl[k] = c.ppl;
        g.tune_chunk[k] = c.chunk;
        g.tune_gen++;
    };
    // keep the candidates the memory budget admits, warm each up (its first
    // call captures its launch graph) and time one call to size the repetitions
    std::vector<Cand> live;
    std::vector<float> one;
    for (const Cand &c : cands) {
        set_shape(c);
        size_t free_b = 0, total_b = 0;
        RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
        uint32_t ppl, chunk;
        const uint64_t budget = (uint64_t)(0.6 * (double)(free_b + g.ws.state.bytes));
        const bool ok = uses_v2(g, k) ? choose_shape_v2(g, k, budget, &ppl, &chunk)
                                      : choose_shape(g, k, budget, &ppl, &chunk);
        if (!ok || chunk != c.chunk || ppl != c.ppl) continue;
        rr_status s = reach_on_stream(g, g.ws, &q, nullptr, S.as<uint64_t>(), 0, g.stream);
        if (s != RR_OK) break;
        RR_CUDA(cudaEventRecord(e0, g.stream));
        s = reach_on_stream(g, g.ws, &q, nullptr, S.as<uint64_t>(), 0, g.stream);
        RR_CUDA(cudaEventRecord(e1, g.stream));
        RR_CUDA(cudaEventSynchronize(e1));
        if (s != RR_OK) break;
        float ms = 0;
        RR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        live.push_back(c);
        one.push_back(ms);
    }
    // best of interleaved rounds, each about 2 ms of queries per candidate
    // (one round when a query takes 5 ms or more)
    std::vector<float> bestv(live.size(), 1e30f);
    const float slowest = live.empty() ? 0.f : *std::max_element(one.begin(), one.end());
    const int rounds = slowest < 5.f ? 3 : 1;
    rr_status failed = RR_OK;
    for (int round = 0; round < rounds && failed == RR_OK; ++round)
        for (size_t i = 0; i < live.size() && failed == RR_OK; ++i) {
            set_shape(live[i]);
            const int reps = std::max(1, std::min(20, (int)(2.f / std::max(one[i], 1e-3f))));
            rr_status s = RR_OK;
            RR_CUDA(cudaEventRecord(e0, g.stream));
            for (int rep = 0; rep < reps && s == RR_OK; ++rep)
                s = reach_on_stream(g, g.ws, &q, nullptr, S.as<uint64_t>(), 0, g.stream);
            RR_CUDA(cudaEventRecord(e1, g.stream));
            RR_CUDA(cudaEventSynchronize(e1));
            if (s != RR_OK) {
                failed = s;
                break;
            }
            float ms = 0;
            RR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            bestv[i] = std::min(bestv[i], ms / (float)reps);
        }
    if (failed != RR_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        g.tune_ppl[k] = save_ppl;
        g.tune_chunk[k] = save_chunk;
        g.tune_gen++;
        return failed;
    }
    Cand win{0, 0};
    float best = 1e30f;
    for (size_t i = 0; i < live.size(); ++i)
        if (bestv[i] < best) {
            best = bestv[i];
            win = live[i];
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (win.ppl == 0) {
        g.tune_ppl[k] = save_ppl;
        g.tune_chunk[k] = save_chunk;
        g.tune_gen++;
        return fail(RR_ENOMEM, "rr_autotune: no candidate shape fits device memory");
    }
    g.tune_ppl[k] = win.ppl;
    g.tune_chunk[k] = win.chunk;
    g.tune_gen++;
    if (best_ppl) *best_ppl = win.ppl;
    if (best_chunk) *best_chunk = win.chunk;
    return RR_OK;
}

}  // namespace rr
