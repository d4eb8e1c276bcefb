// rr_v2_device.cuh -- per-warp bodies of the reduced-state engine's layers,
// shared by the one-query kernels (rr_sieve2.cu) and the persistent batched
// kernel (rr_batch.cu).
#pragma once
#include <cstdint>

#include "rr_device.cuh"
#include "rr_internal.h"

namespace rr {

// The multiply used by the per-warp layer code. Kernels that inline many task
// kinds (the persistent batch) define RR_OUTLINED_MUL before including this
// header and call one out-of-line copy: inlining ~300 integer instructions at
// every call site of every kind overflowed the instruction cache there. The
// one-query kernels, each a single variant, keep it inline.
#ifdef RR_OUTLINED_MUL
__device__ __noinline__ static uint64_t rr_mul(uint64_t a, uint64_t b)
{
    return gf64_mul(a, b);
}
#else
__device__ __forceinline__ static uint64_t rr_mul(uint64_t a, uint64_t b)
{
    return gf64_mul(a, b);
}
#endif
// An out-of-line multiply for the extra products of an otherwise inlined
// body: a call keeps only the caller's live values in registers, where
// inlining more products beside the body's own raised its register count
// (and cut the warps in flight) more than the call costs.
__device__ __noinline__ static uint64_t rr_mul_call(uint64_t a, uint64_t b)
{
    return gf64_mul(a, b);
}

constexpr int kW2 = 4;  // warps per block

// Layer 3 in pair-label space: a deep row holds the k(k+1)/2 values of a
// symmetric label pair matrix, value (i, j), i >= j, at i(i+1)/2 + j.
constexpr uint32_t kMaxPairs = 210;  // k = 20
__host__ __device__ __forceinline__ uint32_t pair_count(uint32_t k)
{
    return k * (k + 1) / 2;
}

// Pair tail: layer k-3 stores, per deep row and point group, the sums of its
// per-point state over the group's points that hold a given set A of at most
// two in-group labels (LG of them): slot 0 for A = {} (the group total), 1 + a
// for A = {a}, 1 + LG + b(b-1)/2 + a for A = {a < b}; 29 slots (LG = 7) or 22
// (LG = 6) of a 32-value block. Layer k-2 then keeps kLabelTailWidth values
// per deep row (LG label values and one per point group, at most 8 groups).
constexpr uint32_t kPairTailSlots = 32;
constexpr uint32_t kLabelTailWidth = 16;
constexpr uint32_t kPairTailMaxGroups = 8;
// Layer k-2 in label space costs 5 to 7 products per lane and row, the
// per-point layer it replaces chunk/32: the pair tail runs for chunks of at
// least this many points.
constexpr uint32_t kPairTailMinChunk = 256;
template <int LG>
__host__ __device__ __forceinline__ uint32_t pair_tail_slot(uint32_t A)
{
#ifdef __CUDA_ARCH__
    const int c = __popc(A);
    const uint32_t a = (uint32_t)__ffs((int)A) - 1u, b = 31u - (uint32_t)__clz((int)A);
#else
    const int c = __builtin_popcount(A);
    const uint32_t a = A ? (uint32_t)__builtin_ctz(A) : 0u, b = A ? 31u - (uint32_t)__builtin_clz(A) : 0u;
#endif
    if (c == 0) return 0u;
    if (c == 1) return 1u + a;
    return 1u + (uint32_t)LG + b * (b - 1u) / 2u + a;
}

struct V2Params {
    // list
    const uint32_t *head, *eid, *src, *ia, *ib;
    const uint2 *items;
    uint32_t nitems;
    // query
    const QueryDesc *qd;  // source, key_y and the witness pointer of the query
    const uint64_t *z;
    uint32_t n, k, layer;
    // chunk
    uint32_t chunk_base, chunk, ngroups, npoints;
    const uint64_t *py;     // scalar layer-1 prefix, indexed by producer rank
    const uint64_t *pr2;    // layer-2 label-space prefix, k values per state row
    const uint64_t *pr3;    // layer-3 pair-label prefix, pair_count(k) values per deep row
    const uint32_t *trank;  // per entry: rank of its tail among the deep rows' heads
    const uint32_t *dheads; // the deep rows' distinct heads
    uint32_t ndheads;
    uint64_t *tx;           // x_h^L x_s^L per deep-row head h (rank order) and point, stride chunk
    const uint64_t *st_in;  // full state, stride chunk
    uint64_t *st_out;       // full (stride chunk) or reduced (stride ngroups*(lg+1))
    // st_in's cut head segments carry lazily (one-query kernels): row r's true
    // prefix is st_in[r] ^ carry[row_carry[r]] (carry row 0 is zero); null:
    // st_in holds true prefixes
    const uint32_t *row_carry;
    const uint64_t *carry;
    // pair-sum blocks per stored row, for a last layer that reads the pair
    // tail's layer k-3 sums (at-most-k branch k-1)
    uint32_t blk_groups;
};

// z_{u,j}: from the table when the query has one (motif queries, Eq. 3), else
// drawn on the fly (plain queries: z_{u,j} = draw(key_z, 32u + j), the same
// value the table would hold).
__device__ __forceinline__ uint64_t zval(const V2Params &p, uint64_t u, uint32_t j)
{
    return p.z ? p.z[u * p.k + j] : sm_draw(p.qd->key_z, u * 32u + j);
}

// Programmatic dependent launch (sm_90 and later): wait until the previous
// kernel of the stream has completed and its writes are visible, then let the
// next kernel be scheduled once every block of this one has got here, so its
// launch overlaps this kernel's work while at most one waiting grid per stream
// holds SM slots. Called before a kernel touches memory; without a
// programmatic dependency both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The layer bodies of the one-query kernels call pdl_enter() late: after the
// loads and hashes that read only graph and query data (row metadata, y and z
// draws, per-head factors), before their first read of a previous kernel's
// results and before any write. When a kernel of the chain starts, the kernel
// two places before it has completed (its predecessor let it launch only after
// its own wait), so the query's z-table is ready; all writes wait.

__device__ __forceinline__ uint64_t shfl64b(uint64_t v, int src)
{
    return __shfl_sync(0xffffffffu, (unsigned long long)v, src);
}
__device__ __forceinline__ uint64_t shfl64x(uint64_t v, int mask)
{
    return __shfl_xor_sync(0xffffffffu, (unsigned long long)v, mask);
}

// Sum over j in L of the per-label values held by lanes first..first+k-1 (lane
// first+j holds label j+1's value), for the lane's PPL consecutive points
// pbits + i, i < PPL (pbits: the lane's first point, its low LOGP bits zero):
// label j+1 is in point L when bit j of L is set, so the labels above LOGP
// follow pbits and the lowest LOGP labels the point's offset i.
template <int PPL>
__device__ __forceinline__ void combine_labels(uint64_t lane_val, uint32_t k, uint32_t pbits,
                                               uint64_t (&out)[PPL], uint32_t first = 0)
{
    constexpr uint32_t LOGP = PPL == 4 ? 2 : 1;
    const uint64_t low0 = shfl64b(lane_val, (int)first);
    const uint64_t low1 = LOGP == 2 ? shfl64b(lane_val, (int)first + 1) : 0ull;
    uint64_t base = 0;
    for (uint32_t j = LOGP; j < k; ++j) {
        const uint64_t bj = shfl64b(lane_val, (int)(first + j));
        if ((pbits >> j) & 1u) base ^= bj;
    }
    out[0] = base;
    out[1] = base ^ low0;
    if constexpr (PPL == 4) {
        out[2] = base ^ low1;
        out[3] = base ^ low0 ^ low1;
    }
}

// Q^L = sum over i, j in L of the pair values sq(q) (value (i, j), i >= j, at
// q = i(i+1)/2 + j, the sum of both orders for i != j) for the lane's PPL
// points pbits + i: the labels above LOGP contribute the same base to all of
// them, the lowest LOGP labels their diagonal and their pairs with the base's
// labels. Every lane reads the same q at a time (broadcast loads).
template <int PPL, class Val>
__device__ __forceinline__ void pair_form(const Val &sq, uint32_t k, uint32_t pbits,
                                          uint64_t (&out)[PPL])
{
    constexpr uint32_t LOGP = PPL == 4 ? 2 : 1;
    uint64_t base = 0, t0 = sq(0), t1 = 0, s01 = 0;
    if constexpr (LOGP == 2) {
        t1 = sq(2);   // (1, 1)
        s01 = sq(1);  // (1, 0)
    }
    for (uint32_t i = LOGP; i < k; ++i) {
        const uint32_t r = i * (i + 1) / 2;
        uint64_t row = sq(r + i);
        for (uint32_t j = LOGP; j < i; ++j)
            if ((pbits >> j) & 1u) row ^= sq(r + j);
        if ((pbits >> i) & 1u) {
            base ^= row;
            t0 ^= sq(r);
            if constexpr (LOGP == 2) t1 ^= sq(r + 1);
        }
    }
    out[0] = base;
    out[1] = base ^ t0;
    if constexpr (PPL == 4) {
        out[2] = base ^ t1;
        out[3] = base ^ t0 ^ t1 ^ s01;
    }
}

// pair_form with the pair values spread over the warp: lane l holds value
// l + 32 s in d[s] (two slots: up to 64 values, k <= 10; with more values the
// layer reads them by broadcast loads, which measured faster there), read by
// shuffles that every lane executes (only the XORs depend on the lane's points;
// the slot of a value is warp-uniform, so exactly one shuffle runs per value).
template <int NS>
__device__ __forceinline__ uint64_t shfl_slot(const uint64_t (&d)[NS], uint32_t q)
{
    static_assert(NS == 2, "two slots (k <= 10)");
    const int l = (int)(q & 31u);
    return q < 32u ? shfl64b(d[0], l) : shfl64b(d[1], l);
}

template <int NS>
__device__ __forceinline__ void pair_window_regs(const uint64_t *__restrict__ pr3, uint32_t a, uint32_t b,
                                                 uint32_t np, int lane, uint64_t (&d)[NS])
{
    const uint64_t *pa = pr3 + (size_t)a * np, *pb = pr3 + (size_t)b * np;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const uint32_t q = 32u * s + (uint32_t)lane;
        d[s] = q < np ? (__ldg(pb + q) ^ __ldg(pa + q)) : 0ull;
    }
}

template <int PPL, int NS>
__device__ __forceinline__ void pair_form_shfl(const uint64_t (&d)[NS], uint32_t k, uint32_t pbits,
                                               uint64_t (&out)[PPL])
{
    constexpr uint32_t LOGP = PPL == 4 ? 2 : 1;
    auto sq = [&](uint32_t q) { return shfl_slot<NS>(d, q); };
    uint64_t base = 0, t0 = sq(0), t1 = 0, s01 = 0;
    if constexpr (LOGP == 2) {
        t1 = sq(2);
        s01 = sq(1);
    }
    for (uint32_t i = LOGP; i < k; ++i) {  // warp-uniform
        const uint32_t r = i * (i + 1) / 2;
        uint64_t row = sq(r + i);
        for (uint32_t j = LOGP; j < i; ++j) {  // warp-uniform
            const uint64_t v = sq(r + j);
            if ((pbits >> j) & 1u) row ^= v;
        }
        const uint64_t v0 = sq(r);
        const uint64_t v1 = LOGP == 2 ? sq(r + 1) : 0ull;
        if ((pbits >> i) & 1u) {
            base ^= row;
            t0 ^= v0;
            if constexpr (LOGP == 2) t1 ^= v1;
        }
    }
    out[0] = base;
    out[1] = base ^ t0;
    if constexpr (PPL == 4) {
        out[2] = base ^ t1;
        out[3] = base ^ t0 ^ t1 ^ s01;
    }
}

// x_h^L x_s^L for deep-row head rank r and the lane's PPL points of point
// group `group` of the chunk: the factor layer 4 applies to pair windows of
// h's rows (one table per chunk, one product per head and point).
template <int PPL>
__device__ __forceinline__ void head_factor_warp(const V2Params &p, uint32_t r, uint32_t group)
{
    const int lane = threadIdx.x & 31;
    const uint32_t k = p.k;
    const uint32_t col = group * (32u * PPL) + (uint32_t)lane * PPL;
    const uint32_t pbits = p.chunk_base + col;  // the lane's first point
    const uint32_t h = p.dheads[r];
    const uint64_t zs = (uint32_t)lane < k ? zval(p, p.qd->source, lane) : 0ull;
    const uint64_t zh = (uint32_t)lane < k ? zval(p, h, lane) : 0ull;
    uint64_t xs[PPL], xh[PPL], f[PPL];
    combine_labels<PPL>(zs, k, pbits, xs);
    combine_labels<PPL>(zh, k, pbits, xh);
#pragma unroll
    for (int i = 0; i < PPL; ++i) f[i] = rr_mul(xh[i], xs[i]);
    pdl_enter();  // the table is written from here on
    ulonglong2 *pt = reinterpret_cast<ulonglong2 *>(p.tx + (size_t)r * p.chunk + col);
    pt[0] = make_ulonglong2(f[0], f[1]);
    if constexpr (PPL == 4) pt[1] = make_ulonglong2(f[2], f[3]);
}

// ---------------------------------------------------------------------------
// Layer 1: PY[p+1] = XOR of [src == s] y_{f,1} over the producer-list entries
// of p's head segment up to p (segmented inclusive scan, 32 entries a step).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void first_scalar_warp(const V2Params &p, uint32_t task,
                                                  uint64_t *__restrict__ py)
{
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[task];
    const uint32_t source = p.qd->source;
    const uint64_t key_y = p.qd->key_y;
    uint64_t carry = 0;
    uint32_t carry_head = 0xFFFFFFFFu;
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t h = has ? p.head[ent] : 0xFFFFFFFEu;
        uint64_t q = 0;
        if (has && p.src[ent] == source)
            q = sm_draw(key_y, (uint64_t)p.eid[ent] * 32u);  // y_{f,1}
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t qq = __shfl_up_sync(0xffffffffu, (unsigned long long)q, d);
            const uint32_t hh = __shfl_up_sync(0xffffffffu, h, d);
            if (lane >= d && hh == h) q ^= qq;
        }
        if (h == carry_head) q ^= carry;
        if (has) py[(size_t)ent + 1] = q;
        const int last = (int)min(31u, it.y - 1 - base);
        carry = shfl64b(q, last);
        carry_head = __shfl_sync(0xffffffffu, h, last);
    }
}

// ---------------------------------------------------------------------------
// k = 2 without sieve points: layer 1 is the last layer, and summing
// y_{e,1} x_s^L x_v^L over all L leaves the 2x2 permanent, so every edge
// e = (s, v) adds y_{e,1} (z_{s,1} z_{v,2} + z_{s,2} z_{v,1}) to S[v]. One
// thread per CSR row r; only rows leaving the source look up their head v
// (the vertex with off[v] <= r < off[v+1], by bisection).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void first2_closed(const V2Params &p, const uint32_t *__restrict__ off,
                                              const uint32_t *__restrict__ row_src,
                                              const uint32_t *__restrict__ row_eid, uint32_t r)
{
    const uint32_t s = p.qd->source;
    if (row_src[r] != s) return;
    uint32_t lo = 0, hi = p.n;  // off[lo] <= r < off[hi]
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (off[mid] <= r) lo = mid;
        else hi = mid;
    }
    const uint32_t v = lo;
    const uint64_t perm = rr_mul(zval(p, s, 0), zval(p, v, 1)) ^ rr_mul(zval(p, s, 1), zval(p, v, 0));
    const uint32_t e = row_eid[r];
    const uint64_t val = rr_mul(sm_draw(p.qd->key_y, (uint64_t)e * 32u), perm);  // y_{e,1}
    if (val) atomicXor(reinterpret_cast<unsigned long long *>(p.qd->S + v), (unsigned long long)val);
    if (p.qd->E) p.qd->E[e] = val;  // one row per edge
}

// ---------------------------------------------------------------------------
// The last layer when k = 3, without sieve points. With the scalar layer-1
// prefix the layer-2 value of entry e (tail u, head v) at point L is
// y_{e,2} Y_e x_s^L x_u^L x_v^L, Y_e = PY[a0] ^ PY[b0]. Summed over all L, a
// product of k linear forms x_i^L = sum_{j in L} Z[i][j] gives the permanent
// of Z: each map i -> j_i is counted once for every L holding its image, i.e.
// 2^{k - |image|} times, which is odd only for the bijections. So entry e adds
//     y_{e,2} Y_e perm(z_s; z_u; z_v)
// to S[v], and only entries with Y_e != 0 (a source edge inside the window)
// do any multiplication. One thread per entry.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void last3_closed(const V2Params &p, uint32_t ent)
{
    const uint64_t Y = p.py[p.ia[ent]] ^ p.py[p.ib[ent]];
    if (!Y) return;
    const uint32_t s = p.qd->source, u = p.src[ent], v = p.head[ent];
    uint64_t a[3], b[3], c[3];
#pragma unroll
    for (uint32_t j = 0; j < 3; ++j) {
        a[j] = zval(p, s, j);
        b[j] = zval(p, u, j);
        c[j] = zval(p, v, j);
    }
    // expansion along z_s: 2x2 permanents of (z_u, z_v) without column j
    const uint64_t m0 = rr_mul(b[1], c[2]) ^ rr_mul(b[2], c[1]);
    const uint64_t m1 = rr_mul(b[0], c[2]) ^ rr_mul(b[2], c[0]);
    const uint64_t m2 = rr_mul(b[0], c[1]) ^ rr_mul(b[1], c[0]);
    const uint64_t perm = rr_mul(a[0], m0) ^ rr_mul(a[1], m1) ^ rr_mul(a[2], m2);
    const uint32_t e = p.eid[ent];
    const uint64_t y = sm_draw(p.qd->key_y, (uint64_t)e * 32u + 1u);  // y_{e,2}
    const uint64_t val = rr_mul(rr_mul(y, Y), perm);
    if (val) atomicXor(reinterpret_cast<unsigned long long *>(p.qd->S + v), (unsigned long long)val);
    if (p.qd->E) p.qd->E[e] = val;  // one entry per edge
}

// ---------------------------------------------------------------------------
// k = 4, last layer in closed form over the label-space layer 2. A state row
// f' of vertex v holds, over the points, P_2^L[f'] = x_v^L x_s^L
// sum_{j in L} (y_{f',2} Y_{f'}) z_{u_{f'},j}, so the window of entry e (tail
// v, head w) sums to x_v^L x_s^L D^L with D^L = sum_{j in L} dPR2_j, the
// window's difference of the label-space prefix. The last layer multiplies by
// y_{e,3} x_w^L, and summed over all L in [4] the product of the four linear
// forms x_s, x_v, x_w, D counts each choice of one label per form 2^{4 - #}
// times: only the bijections survive, so e adds
//     y_{e,3} perm(z_s; z_v; z_w; dPR2)
// to S[w]. A quad of lanes takes one entry, lane j owning label column j:
// with b = z_v, c = z_w, d = dPR2 and Q_{ab} = c_a d_b + c_b d_a (the 2x2
// permanents of the last two rows), lane j forms c_j d_{j^x} (x = 1, 2, 3),
// which with its partner j^x gives Q_{j,j^x}; then the expansion along z_v of
// the 3x3 minor without column j,
//     t_j = b_{j^1} Q_{j^2,j^3} + b_{j^2} Q_{j^1,j^3} + b_{j^3} Q_{j^1,j^2},
// and perm = sum_j z_{s,j} t_j over the quad: 8 products per lane. The tail
// list is grouped by head, so the quads of a warp XOR their values along runs
// of equal heads and the run's last quad adds the run's sum: one atomic per
// head and warp.
// ---------------------------------------------------------------------------
// Called by whole warps; ent = a warp-aligned base / 4 + quad (8 entries per warp).
__device__ __forceinline__ void last4_closed(const V2Params &p, uint32_t ent, uint32_t count, uint64_t zs_j)
{
    const int lane = threadIdx.x & 31;
    const int j = lane & 3, quad = lane >> 2;
    const bool has = ent < count;
    const uint32_t w = has ? p.head[ent] : 0xffffffffu;
    uint64_t d = 0;
    if (has) d = p.pr2[(size_t)p.ia[ent] * 4u + j] ^ p.pr2[(size_t)p.ib[ent] * 4u + j];
    uint64_t val = 0;
    if (__any_sync(0xffffffffu, d != 0)) {  // warp-uniform
        const uint32_t v = has ? p.src[ent] : 0u;
        const uint64_t b = has ? zval(p, v, (uint32_t)j) : 0ull;
        const uint64_t c = has ? zval(p, w, (uint32_t)j) : 0ull;
        // c_j d_{j^x}, then Q_{j,j^x} = c_j d_{j^x} + c_{j^x} d_j
        const uint64_t q1 = rr_mul(c, shfl64x(d, 1)), q2 = rr_mul(c, shfl64x(d, 2)), q3 = rr_mul(c, shfl64x(d, 3));
        const uint64_t Q1 = q1 ^ shfl64x(q1, 1), Q2 = q2 ^ shfl64x(q2, 2), Q3 = q3 ^ shfl64x(q3, 3);
        // Q_{j^2,j^3}: lane j^2's Q1; Q_{j^1,j^3}: lane j^1's Q2; Q_{j^1,j^2}: lane j^1's Q3
        const uint64_t t = rr_mul(shfl64x(b, 1), shfl64x(Q1, 2)) ^ rr_mul(shfl64x(b, 2), shfl64x(Q2, 1)) ^
                           rr_mul(shfl64x(b, 3), shfl64x(Q3, 1));
        uint64_t perm = rr_mul(zs_j, t);
        perm ^= shfl64x(perm, 1);
        perm ^= shfl64x(perm, 2);
        const uint32_t e = has ? p.eid[ent] : 0u;
        val = rr_mul(sm_draw(p.qd->key_y, (uint64_t)e * 32u + 2u), perm);  // y_{e,3}
        if (has && j == 0 && p.qd->E) p.qd->E[e] = val;  // one entry per edge
    }
    // XOR along the runs of equal heads (contiguous quads)
    const uint32_t prev = __shfl_sync(0xffffffffu, w, lane >= 4 ? lane - 4 : lane);
    const uint32_t starts = __ballot_sync(0xffffffffu, j == 0 && (quad == 0 || prev != w));
    const int run0 = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));  // first lane of the run
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        const uint64_t o = shfl64b(val, lane >= off ? lane - off : lane);
        if (lane - off >= run0) val ^= o;
    }
    const bool run_end = quad == 7 || ((starts >> (lane + 4 - j)) & 1u);
    if (has && j == 0 && run_end && val)
        atomicXor(reinterpret_cast<unsigned long long *>(p.qd->S + w), (unsigned long long)val);
}

// ---------------------------------------------------------------------------
// k = 5, last layer in closed form over the pair-label layer 3. The window of
// tail-list entry e (tail v, head w) over v's deep rows sums to
// x_v^L x_s^L sum_{i,j in L} dQ_ij (dQ the window's difference of the pair
// prefix), and the last layer multiplies by y_{e,4} x_w^L. Summed over all L in
// [5], a term w_a v_b s_c dQ_ij survives only when a, b, c, i, j are the five
// labels, so with S_{ij} = dQ_ij + dQ_ji (the stored off-diagonal value) and
// P_{bc} = v_b s_c + v_c s_b (2x2 permanents of z_v, z_s), e adds
//     y_{e,4} sum_a w_a X_a,   X_a = sum over the three ways to split [5] \ {a}
//                              into pairs {p, q} of S_p P_q + S_q P_p
// to S[w] (56 products). Eight lanes take one entry, lane c < 5 owning label
// c: it forms P over {c, c+1} and {c, c+2} (labels mod 5; the ten pairs once),
// gathers the four others it needs over shuffles, and adds w_c X_c; 12
// products a lane. The pair rows may belong to a larger query (at-most-k
// branch k' = 5 of a query with the pair-label layer 3): labels 0..4 are the
// first 15 values of their rows, np values apart. Runs of equal heads in a
// warp are XORed before one atomic per run.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pair_index(uint32_t x, uint32_t y)
{
    const uint32_t hi = max(x, y), lo = min(x, y);
    return hi * (hi + 1u) / 2u + lo;
}

// Called by whole warps; ent = a warp-aligned base / 8 + group (4 entries per
// warp). zs0, zs1, zs2: z_{s,c}, z_{s,c+1}, z_{s,c+2} (labels mod 5) of the
// lane's label c.
__device__ __forceinline__ void last5_closed(const V2Params &p, uint32_t ent, uint32_t count, uint32_t np,
                                             uint64_t zs0, uint64_t zs1, uint64_t zs2)
{
    const int lane = threadIdx.x & 31;
    const uint32_t c = (uint32_t)lane & 7u, gbase = (uint32_t)lane & ~7u, grp = (uint32_t)lane >> 3;
    const bool act = c < 5u;
    const bool has = ent < count;
    const uint32_t w = has ? p.head[ent] : 0xffffffffu;
    // the other four labels, and the six pairs among them in split order:
    // (o0,o1 | o2,o3), (o0,o2 | o1,o3), (o0,o3 | o1,o2)
    uint32_t o[4];
#pragma unroll
    for (uint32_t t = 0; t < 4; ++t) o[t] = t + (act && t >= c ? 1u : 0u);
    constexpr uint32_t PA[6] = {0, 2, 0, 1, 0, 1}, PB[6] = {1, 3, 2, 3, 3, 2};
    uint64_t S[6];
    bool nz = false;
#pragma unroll
    for (int t = 0; t < 6; ++t) S[t] = 0;
    if (has && act) {
        const uint64_t *ra = p.pr3 + (size_t)p.ia[ent] * np, *rb = p.pr3 + (size_t)p.ib[ent] * np;
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const uint32_t q = pair_index(o[PA[t]], o[PB[t]]);
            S[t] = ra[q] ^ rb[q];
            nz |= S[t] != 0;
        }
    }
    uint64_t val = 0;
    if (__any_sync(0xffffffffu, nz)) {  // warp-uniform
        const uint32_t v = has ? p.src[ent] : 0u;
        const uint64_t zv = has && act ? zval(p, v, c) : 0ull;
        const uint64_t zw = has && act ? zval(p, w, c) : 0ull;
        const uint32_t c1 = act ? (c + 1u) % 5u : c, c2 = act ? (c + 2u) % 5u : c;
        const uint64_t v1 = shfl64b(zv, (int)(gbase + c1)), v2 = shfl64b(zv, (int)(gbase + c2));
        uint64_t P1 = 0, P2 = 0;  // P over {c, c+1} and {c, c+2}
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const uint64_t Ph = rr_mul(zv, h ? zs2 : zs1) ^ rr_mul(h ? v2 : v1, zs0);
            if (h) P2 = Ph;
            else P1 = Ph;
        }
        // pair {x, y}: d = y - x mod 5; lane x holds it as its P_d for d = 1, 2,
        // else lane y as its P_{5-d}
        uint64_t P[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const uint32_t x = o[PA[t]], y = o[PB[t]], d = (y + 5u - x) % 5u;
            const uint32_t owner = d <= 2u ? x : y, slot = d <= 2u ? d : 5u - d;
            const uint64_t t1 = shfl64b(P1, (int)(gbase + owner)), t2 = shfl64b(P2, (int)(gbase + owner));
            P[t] = slot == 1u ? t1 : t2;
        }
        // one split at a time (operands by select): two products in flight
        uint64_t X = 0;
#pragma unroll 1
        for (int m = 0; m < 3; ++m) {
            const uint64_t sa = m == 0 ? S[0] : (m == 1 ? S[2] : S[4]);
            const uint64_t sb = m == 0 ? S[1] : (m == 1 ? S[3] : S[5]);
            const uint64_t pa = m == 0 ? P[0] : (m == 1 ? P[2] : P[4]);
            const uint64_t pb = m == 0 ? P[1] : (m == 1 ? P[3] : P[5]);
            X ^= rr_mul(sa, pb) ^ rr_mul(sb, pa);
        }
        uint64_t sum = rr_mul(zw, X);  // zero on lanes 5..7
        sum ^= shfl64x(sum, 1);
        sum ^= shfl64x(sum, 2);
        sum ^= shfl64x(sum, 4);
        const uint32_t e = has ? p.eid[ent] : 0u;
        val = rr_mul(sm_draw(p.qd->key_y, (uint64_t)e * 32u + 3u), sum);  // y_{e,4}
        if (has && c == 0u && p.qd->E) p.qd->E[e] = val;  // one entry per edge
    }
    // XOR along the runs of equal heads (contiguous groups of 8 lanes)
    const uint32_t prev = __shfl_sync(0xffffffffu, w, lane >= 8 ? lane - 8 : lane);
    const uint32_t starts = __ballot_sync(0xffffffffu, c == 0u && (grp == 0u || prev != w));
    const int run0 = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));  // first lane of the run
#pragma unroll
    for (int off = 8; off < 32; off <<= 1) {
        const uint64_t ov = shfl64b(val, lane >= off ? lane - off : lane);
        if (lane - off >= run0) val ^= ov;
    }
    const bool run_end = grp == 3u || ((starts >> (lane + 8 - (int)c)) & 1u);
    if (has && c == 0u && run_end && val)
        atomicXor(reinterpret_cast<unsigned long long *>(p.qd->S + w), (unsigned long long)val);
}

// Sums of a lane group's per-point values (acc, the lane's PPL points) over
// the group's 32*PPL points holding each in-group label: lane j < LG returns
// T_j -- the in-lane labels from U, the lane labels from the half-cube sums of
// V -- and lane LG the total V. Every lane takes part in the shuffles.
template <int PPL>
__device__ __forceinline__ uint64_t single_label_sums(const uint64_t (&acc)[PPL], int lane)
{
    constexpr int LOGP = PPL == 4 ? 2 : 1;
    constexpr int LG = LOGP + 5;
    uint64_t V = 0;
#pragma unroll
    for (int i = 0; i < PPL; ++i) V ^= acc[i];
    uint64_t U0 = acc[1] ^ (PPL == 4 ? acc[3] : 0ull);
    uint64_t U1 = PPL == 4 ? (acc[2] ^ acc[3]) : 0ull;
    uint64_t X = V, Y[5];
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        const uint64_t P = shfl64x(X, 1 << bb);
        Y[bb] = ((lane >> bb) & 1) ? X : P;
        X ^= P;
#pragma unroll
        for (int b2 = 0; b2 < bb; ++b2) Y[b2] ^= shfl64x(Y[b2], 1 << bb);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        U0 ^= shfl64x(U0, off);
        if constexpr (PPL == 4) U1 ^= shfl64x(U1, off);
    }
    // slot j < LG: T_j ; slot LG: V
    if (LOGP == 2 && lane == 1) return U1;
    if (lane == 0) return U0;
    if (lane < LG) {
        const int bb = lane - LOGP;
        return bb == 0 ? Y[0] : bb == 1 ? Y[1] : bb == 2 ? Y[2] : bb == 3 ? Y[3] : Y[4];
    }
    return X;
}

// At-most-k branch: the stored per-point rows of one layer, restricted to the
// points below p.npoints, as the sums over single labels of each point group
// -- what layer k'-2 of the k'-vertex query writes as its transformed state,
// since for the same seed the two queries' layers agree on those points. The
// lazy carries of cut hub segments are added first, so the rows are true
// prefixes. One warp per (32 consecutive deep rows, point group); p.st_out
// has p.ngroups groups of LG + 1 values per row.
template <int PPL>
__device__ __forceinline__ void transform_rows_warp(const V2Params &p, uint32_t task, uint32_t nrows)
{
    constexpr int LOGP = PPL == 4 ? 2 : 1;
    constexpr int LG = LOGP + 5;
    const int lane = threadIdx.x & 31;
    const uint32_t group = task % p.ngroups, rb = task / p.ngroups;
    const uint32_t col = group * (32u * PPL) + (uint32_t)lane * PPL;
    const uint32_t first = p.chunk_base + col;  // the lane's first point
    bool valid[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) valid[i] = first + i < p.npoints;
    const uint32_t r0 = 1 + rb * 32, r1 = min(nrows + 1, r0 + 32);  // deep rows 1..nrows
    const uint32_t m_slot = (p.carry && r0 + (uint32_t)lane < r1) ? p.row_carry[r0 + lane] : 0u;
    pdl_enter();  // the layer's rows and carries are read from here on
    for (uint32_t r = r0; r < r1; ++r) {
        const uint32_t slot = __shfl_sync(0xffffffffu, m_slot, (int)(r - r0));
        const ulonglong2 *pr = reinterpret_cast<const ulonglong2 *>(p.st_in + (size_t)r * p.chunk + col);
        uint64_t acc[PPL];
        const ulonglong2 a0 = __ldg(pr);
        acc[0] = a0.x;
        acc[1] = a0.y;
        if constexpr (PPL == 4) {
            const ulonglong2 a1 = __ldg(pr + 1);
            acc[2] = a1.x;
            acc[3] = a1.y;
        }
        if (slot) {  // warp-uniform
            const ulonglong2 *pc = reinterpret_cast<const ulonglong2 *>(p.carry + (size_t)slot * p.chunk + col);
            const ulonglong2 c0 = __ldg(pc);
            acc[0] ^= c0.x;
            acc[1] ^= c0.y;
            if constexpr (PPL == 4) {
                const ulonglong2 c1 = __ldg(pc + 1);
                acc[2] ^= c1.x;
                acc[3] ^= c1.y;
            }
        }
#pragma unroll
        for (int i = 0; i < PPL; ++i)
            if (!valid[i]) acc[i] = 0;
        const uint64_t val = single_label_sums<PPL>(acc, lane);
        if (lane <= LG) p.st_out[((size_t)r * p.ngroups + group) * (LG + 1) + lane] = val;
    }
}

// ---------------------------------------------------------------------------
// Layers 2..k-2.
//   FROM_Y: window sum W^L = Y_e x_s^L x_u^L (layer 2), Y_e = PY[a0] ^ PY[b0];
//   else  : W^L = state[a1] ^ state[b1] (layers >= 3).
//   OUT 0: write the per-point prefix to the state row of the entry;
//   OUT 1: write the group's transformed prefix (T_0..T_{lg-1}, V);
//   OUT 2: write its sums over label sets of at most two in-group labels
//          (the pair tail).
// One warp per (scheduling range, point group); lanes own PPL points each.
// ---------------------------------------------------------------------------
// COHERENT: state written earlier in the same launch is read through L2
// (ld.global.cg) instead of the non-coherent read-only path.
// FROM_R2: window sum of layer 2 from its label-space prefix (layer 3):
//   W^L = x_u^L x_s^L rho^L,  rho^L = sum_{j in L} (PR2[a1][j] ^ PR2[b1][j]).
// PAIR (layer 4 after layer 3 in pair-label space, PR3 from third_pair_row):
// the window sum is W^L = x_u^L x_s^L Q^L, Q^L = sum_{i,j in L} dQ_ij,
// dQ = PR3[b3] ^ PR3[a3] (the window's rows all lie in the tail u's segment,
// whose layer-3 rows share the factor x_u x_s); Q^L is evaluated per point
// from the pair values by XORs (pair_form).
template <int PPL, bool FROM_Y, int OUT, bool COHERENT, bool FROM_R2 = false, bool PAIR = false>
__device__ __forceinline__ void layer_warp(const V2Params &p, uint32_t item, uint32_t group)
{
    constexpr int LOGP = PPL == 4 ? 2 : 1;
    constexpr int LG = LOGP + 5;
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t k = p.k;
    const uint32_t source = p.qd->source;
    const uint64_t key_y = p.qd->key_y;
    const uint32_t col = group * (32u * PPL) + (uint32_t)lane * PPL;
    const uint32_t gbase = p.chunk_base + group * (32u * PPL);
    const uint32_t pbits = gbase + (uint32_t)lane * PPL;  // the lane's first point
    bool valid[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) valid[i] = gbase + (uint32_t)lane * PPL + i < p.npoints;

    uint64_t xs[PPL];
    if constexpr (FROM_Y || FROM_R2 || PAIR) {
        const uint64_t zs = (uint32_t)lane < k ? zval(p, source, lane) : 0ull;
        combine_labels<PPL>(zs, k, pbits, xs);
    }

    // FROM_Y: the prefix over the head v's entries factors as
    //   acc^L = (x_v^L x_s^L) * R^L,  R^L = sum_e (y_{e,2} Y_e) x_{u_e}^L,
    // and R needs no per-point multiplication (label values are multiplied
    // lane-parallel, then combined); x_v^L x_s^L is formed once per head.
    uint64_t acc[PPL], R[PPL], xvxs[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) acc[i] = R[i] = xvxs[i] = 0;
    uint32_t cur = p.head[it.x];
    uint64_t zv = 0;
    auto enter_head = [&](uint32_t v) {
        if constexpr (FROM_Y || FROM_R2) {
            zv = (uint32_t)lane < k ? zval(p, v, lane) : 0ull;
            uint64_t xv[PPL];
            combine_labels<PPL>(zv, k, pbits, xv);
#pragma unroll
            for (int i = 0; i < PPL; ++i) xvxs[i] = rr_mul(xv[i], xs[i]);
        }
    };
    enter_head(cur);
    // middle layers and layer 3: the label products of E = floor(32/k)
    // consecutive entries (y_e z_{v_e,j}, resp. y_e rho_{e,j}) are formed by
    // one multiplication per lane (lane i*k + j holds label j of the block's
    // i-th entry), not one per entry
    const uint32_t E = k <= 16 ? 32u / k : 1u;
    const uint32_t lane_e = (uint32_t)lane / k, lane_j = (uint32_t)lane % k;
    uint64_t lab = 0;

    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t m_head = has ? p.head[ent] : 0u;
        const uint32_t m_a = has ? p.ia[ent] : 0u;
        const uint32_t m_b = has ? p.ib[ent] : 0u;
        // carry slots of the window's end rows (lazily carried input state)
        uint32_t m_ca = 0, m_cb = 0;
        if constexpr (!FROM_Y && !FROM_R2 && !PAIR) {
            if (p.carry && has) {
                m_ca = p.row_carry[m_a];
                m_cb = p.row_carry[m_b];
            }
        }
        uint64_t m_coef = 0;
        uint32_t m_src = 0;
        if (has) {
            m_coef = sm_draw(key_y, (uint64_t)p.eid[ent] * 32u + (p.layer - 1u));
            if constexpr (FROM_Y || FROM_R2) m_src = p.src[ent];
            if constexpr (PAIR) m_src = p.tx ? p.trank[ent] : p.src[ent];  // head rank or vertex
        }
        if constexpr (!COHERENT) {
            if (base == it.x) pdl_enter();  // the previous layer's results are read from here on
        }
        if constexpr (FROM_Y) {
            if (has) m_coef = rr_mul(m_coef, p.py[m_a] ^ p.py[m_b]);  // y_{e,2} * Y_e
        }
        const uint32_t nb = min(32u, it.y - base);
        for (uint32_t t = 0; t < nb; ++t) {
            const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)t);
            if (h != cur) {
#pragma unroll
                for (int i = 0; i < PPL; ++i) acc[i] = R[i] = 0;
                cur = h;
                enter_head(cur);
            }
            const uint32_t a = __shfl_sync(0xffffffffu, m_a, (int)t);
            const uint32_t b = __shfl_sync(0xffffffffu, m_b, (int)t);
            if constexpr (FROM_Y) {
                const uint64_t coef = shfl64b(m_coef, (int)t);
                const uint32_t u = __shfl_sync(0xffffffffu, m_src, (int)t);
                const uint64_t zu = (uint32_t)lane < k ? zval(p, u, lane) : 0ull;
                uint64_t r[PPL];
                combine_labels<PPL>(rr_mul(coef, zu), k, pbits, r);
#pragma unroll
                for (int i = 0; i < PPL; ++i) R[i] ^= r[i];
#pragma unroll
                for (int i = 0; i < PPL; ++i) acc[i] = valid[i] ? rr_mul(xvxs[i], R[i]) : 0ull;
            } else if constexpr (FROM_R2) {
                // the same factoring one layer later: acc^L = (x_v^L x_s^L) * R^L with
                // R^L = sum_e x_{u_e}^L (y_{e,3} rho_e)^L; y is folded into the label
                // values lane-parallel, so each entry costs two products per point
                if (t % E == 0) {
                    // y rho_j of E consecutive entries, one multiplication per lane
                    const uint32_t src_lane = min(t + lane_e, 31u);
                    const uint32_t ae = __shfl_sync(0xffffffffu, m_a, (int)src_lane);
                    const uint32_t be = __shfl_sync(0xffffffffu, m_b, (int)src_lane);
                    const uint64_t ye = shfl64b(m_coef, (int)src_lane);
                    lab = 0;
                    if (lane_e < E && t + lane_e < nb && ae != be)
                        lab = rr_mul(ye, p.pr2[(size_t)ae * k + lane_j] ^ p.pr2[(size_t)be * k + lane_j]);
                }
                if (a != b) {
                    const uint32_t u = __shfl_sync(0xffffffffu, m_src, (int)t);
                    const uint64_t zu = (uint32_t)lane < k ? zval(p, u, lane) : 0ull;
                    uint64_t xu[PPL], yrho[PPL];
                    combine_labels<PPL>(zu, k, pbits, xu);
                    combine_labels<PPL>(lab, k, pbits, yrho, (t % E) * k);
#pragma unroll
                    for (int i = 0; i < PPL; ++i) R[i] ^= rr_mul(xu[i], yrho[i]);
#pragma unroll
                    for (int i = 0; i < PPL; ++i) acc[i] = valid[i] ? rr_mul(xvxs[i], R[i]) : 0ull;
                }
            } else {
              if (t % E == 0) {
                  const uint32_t src_lane = min(t + lane_e, 31u);
                  const uint32_t hv = __shfl_sync(0xffffffffu, m_head, (int)src_lane);
                  const uint64_t yv = shfl64b(m_coef, (int)src_lane);
                  lab = (lane_e < E && t + lane_e < nb) ? rr_mul(yv, zval(p, hv, lane_j)) : 0ull;
              }
              if (a != b) {
                uint64_t c[PPL], w[PPL];
                combine_labels<PPL>(lab, k, pbits, c, (t % E) * k);
                if constexpr (PAIR) {
                    // the window's pair values: rows b and a of u's segment
                    const uint32_t np = pair_count(k);
                    const uint64_t *pa = p.pr3 + (size_t)a * np, *pb = p.pr3 + (size_t)b * np;
                    if (np <= 64) {  // k <= 10
                        // the window's values spread over the warp by coalesced loads
                        uint64_t d[2];
                        pair_window_regs<2>(p.pr3, a, b, np, lane, d);
                        pair_form_shfl<PPL, 2>(d, k, pbits, w);
                    } else {
                        pair_form<PPL>([&](uint32_t q) { return __ldg(pb + q) ^ __ldg(pa + q); }, k, pbits, w);
                    }
                    // times x_u^L x_s^L: from the chunk's head-factor table, or
                    // formed here (u = the tail, m_src its vertex or head rank)
                    const uint32_t ut = __shfl_sync(0xffffffffu, m_src, (int)t);
                    if (p.tx) {
                        const ulonglong2 *pt =
                            reinterpret_cast<const ulonglong2 *>(p.tx + (size_t)ut * p.chunk + col);
                        uint64_t f[PPL];
                        const ulonglong2 f0 = __ldg(pt);
                        f[0] = f0.x;
                        f[1] = f0.y;
                        if constexpr (PPL == 4) {
                            const ulonglong2 f1 = __ldg(pt + 1);
                            f[2] = f1.x;
                            f[3] = f1.y;
                        }
#pragma unroll
                        for (int i = 0; i < PPL; ++i) w[i] = rr_mul_call(w[i], f[i]);
                    } else {
                        const uint64_t zu = (uint32_t)lane < k ? zval(p, ut, lane) : 0ull;
                        uint64_t xu[PPL];
                        combine_labels<PPL>(zu, k, pbits, xu);
#pragma unroll
                        for (int i = 0; i < PPL; ++i) w[i] = rr_mul_call(w[i], rr_mul_call(xu[i], xs[i]));
                    }
                } else {
                    const uint64_t *pa = p.st_in + (size_t)a * p.chunk + col;
                    const uint64_t *pb = p.st_in + (size_t)b * p.chunk + col;
                    const ulonglong2 *va = reinterpret_cast<const ulonglong2 *>(pa);
                    const ulonglong2 *vb = reinterpret_cast<const ulonglong2 *>(pb);
                    if constexpr (PPL == 4) {
                        const ulonglong2 a0 = COHERENT ? __ldcg(va) : __ldg(va);
                        const ulonglong2 a1 = COHERENT ? __ldcg(va + 1) : __ldg(va + 1);
                        const ulonglong2 b0 = COHERENT ? __ldcg(vb) : __ldg(vb);
                        const ulonglong2 b1 = COHERENT ? __ldcg(vb + 1) : __ldg(vb + 1);
                        w[0] = a0.x ^ b0.x; w[1] = a0.y ^ b0.y; w[2] = a1.x ^ b1.x; w[3] = a1.y ^ b1.y;
                    } else {
                        const ulonglong2 a0 = COHERENT ? __ldcg(va) : __ldg(va);
                        const ulonglong2 b0 = COHERENT ? __ldcg(vb) : __ldg(vb);
                        w[0] = a0.x ^ b0.x; w[1] = a0.y ^ b0.y;
                    }
                    if constexpr (!COHERENT) {
                        // window ends in different pieces of a cut head segment:
                        // their carries differ by the pieces' totals between them
                        const uint32_t ca = __shfl_sync(0xffffffffu, m_ca, (int)t);
                        const uint32_t cb = __shfl_sync(0xffffffffu, m_cb, (int)t);
                        if (ca != cb) {  // warp-uniform
                            const ulonglong2 *ka =
                                reinterpret_cast<const ulonglong2 *>(p.carry + (size_t)ca * p.chunk + col);
                            const ulonglong2 *kb =
                                reinterpret_cast<const ulonglong2 *>(p.carry + (size_t)cb * p.chunk + col);
                            const ulonglong2 x0 = __ldg(ka), y0 = __ldg(kb);
                            w[0] ^= x0.x ^ y0.x;
                            w[1] ^= x0.y ^ y0.y;
                            if constexpr (PPL == 4) {
                                const ulonglong2 x1 = __ldg(ka + 1), y1 = __ldg(kb + 1);
                                w[2] ^= x1.x ^ y1.x;
                                w[3] ^= x1.y ^ y1.y;
                            }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < PPL; ++i)
                    acc[i] ^= valid[i] ? rr_mul(c[i], w[i]) : 0ull;
              }
            }
            const size_t row = (size_t)base + t + 1;  // state row of this entry
            if constexpr (OUT == 0) {
                uint64_t *po = p.st_out + row * p.chunk + col;
                if constexpr (PPL == 4) {
                    reinterpret_cast<ulonglong2 *>(po)[0] = make_ulonglong2(acc[0], acc[1]);
                    reinterpret_cast<ulonglong2 *>(po)[1] = make_ulonglong2(acc[2], acc[3]);
                } else {
                    reinterpret_cast<ulonglong2 *>(po)[0] = make_ulonglong2(acc[0], acc[1]);
                }
            } else if constexpr (OUT == 1) {
                const uint64_t val = single_label_sums<PPL>(acc, lane);
                if (lane <= LG)
                    p.st_out[(row * p.ngroups + group) * (LG + 1) + lane] = val;
            } else if constexpr (OUT == 2) {
                // superset sums over the group's 32*PPL points: afterwards the
                // lane's value i (its point's in-group label set A = the lane
                // bits above the in-lane bits i) is the sum of acc over the
                // group's points containing A; the sets of at most two labels
                // are stored (slot pair_tail_slot(A))
                uint64_t v[PPL];
#pragma unroll
                for (int i = 0; i < PPL; ++i) v[i] = acc[i];
                v[0] ^= v[1];
                if constexpr (PPL == 4) {
                    v[2] ^= v[3];
                    v[0] ^= v[2];
                    v[1] ^= v[3];
                }
#pragma unroll
                for (int bb = 0; bb < 5; ++bb) {
                    const bool up = (lane >> bb) & 1;
#pragma unroll
                    for (int i = 0; i < PPL; ++i) {
                        const uint64_t o = shfl64x(v[i], 1 << bb);
                        if (!up) v[i] ^= o;
                    }
                }
                uint64_t *blk = p.st_out + (row * p.ngroups + group) * kPairTailSlots;
#pragma unroll
                for (int i = 0; i < PPL; ++i) {
                    const uint32_t A = ((uint32_t)lane << LOGP) | (uint32_t)i;
                    if (__popc(A) <= 2) blk[pair_tail_slot<LG>(A)] = v[i];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Layer 2 in label space (k >= 4): for every state row f of head v,
//   PR2[f][j] = XOR over v's state rows f' <= f of (y_{f',2} Y_{f'}) z_{u_{f'},j}
// so that P_2^L[f'] = x_v^L x_s^L sum_{j in L} (y Y)_{f'} z_{u_{f'},j}. Independent of
// the point chunk; lane j owns label j (one multiplication per lane and row).
// ---------------------------------------------------------------------------
template <bool LATE_WAIT>
__device__ __forceinline__ void second_label_warp(const V2Params &p, uint32_t item,
                                                  uint64_t *__restrict__ pr2)
{
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t k = p.k;
    const uint64_t key_y = p.qd->key_y;
    uint32_t cur = p.head[it.x];
    uint64_t acc = 0;
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t m_head = has ? p.head[ent] : 0u;
        const uint32_t m_src = has ? p.src[ent] : 0u;
        const uint64_t m_y = has ? sm_draw(key_y, (uint64_t)p.eid[ent] * 32u + 1u) : 0ull;  // y_{e,2}
        if constexpr (LATE_WAIT) {
            if (base == it.x) pdl_enter();  // the layer-1 prefix is read from here on
        }
        uint64_t m_coef = 0;
        if (has) m_coef = rr_mul(m_y, p.py[p.ia[ent]] ^ p.py[p.ib[ent]]);  // y_{e,2} Y_e
        const uint32_t nb = min(32u, it.y - base);
        for (uint32_t t = 0; t < nb; ++t) {
            const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)t);
            if (h != cur) {
                acc = 0;
                cur = h;
            }
            const uint64_t coef = shfl64b(m_coef, (int)t);
            const uint32_t u = __shfl_sync(0xffffffffu, m_src, (int)t);
            if ((uint32_t)lane < k) {
                acc ^= rr_mul(coef, zval(p, u, lane));
                pr2[((size_t)base + t + 1) * k + lane] = acc;
            }
        }
    }
}

// The same layer with the rows across the lanes (the one-query kernel): lane t
// takes row base + t and, label by label, its term c_t z_{u_t,j} (c_t =
// y_{e,2} Y_e); an XOR scan over the lanes along runs of equal heads, plus the
// prefix that the head's rows of the previous 32 left (lane j keeps label j's),
// gives PR2. k products per lane per 32 rows instead of 32 on k lanes.
template <bool LATE_WAIT>
__device__ __forceinline__ void second_label_scan_warp(const V2Params &p, uint32_t item,
                                                       uint64_t *__restrict__ pr2)
{
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t k = p.k;
    const uint64_t key_y = p.qd->key_y;
    uint64_t carry = 0;                // lane j < k: label j's prefix at the previous 32's last row
    uint32_t last_head = 0xffffffffu;  // the previous 32's last head (none yet)
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + (uint32_t)lane;
        const bool has = ent < it.y;
        const uint32_t h = has ? p.head[ent] : 0xfffffffeu;
        const uint32_t u = has ? p.src[ent] : 0u;
        const uint64_t y = has ? sm_draw(key_y, (uint64_t)p.eid[ent] * 32u + 1u) : 0ull;  // y_{e,2}
        const uint32_t ia = has ? p.ia[ent] : 0u, ib = has ? p.ib[ent] : 0u;
        if constexpr (LATE_WAIT) {
            if (base == it.x) pdl_enter();  // the layer-1 prefix is read from here on
        }
        const uint64_t coef = has ? rr_mul(y, p.py[ia] ^ p.py[ib]) : 0ull;  // y_{e,2} Y_e
        const bool any = __any_sync(0xffffffffu, coef != 0);
        const uint32_t hp = __shfl_up_sync(0xffffffffu, h, 1);
        const uint32_t starts = __ballot_sync(0xffffffffu, lane == 0 || hp != h);
        const int run0 = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));  // first lane of the run
        const bool cont = run0 == 0 && h == last_head;  // the run goes on from the previous 32
        last_head = __shfl_sync(0xffffffffu, h, 31);
        for (uint32_t j = 0; j < k; ++j) {
            uint64_t val = any ? rr_mul(coef, zval(p, u, j)) : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint64_t o = shfl64b(val, lane >= off ? lane - off : lane);
                if (lane - off >= run0) val ^= o;
            }
            const uint64_t cj = shfl64b(carry, (int)j);  // every lane takes part
            if (cont) val ^= cj;
            if (has) pr2[((size_t)ent + 1) * k + j] = val;
            const uint64_t v31 = shfl64b(val, 31);
            if ((uint32_t)lane == j) carry = v31;
        }
    }
}

// ---------------------------------------------------------------------------
// Layer 3 in pair-label space (6 <= k <= 20): the layer-3 value of deep row e
// (tail u, head v) at point L is x_v^L x_s^L x_u^L g_e^L with
// g_e^L = sum_{i in L} y_{e,3} (PR2[b1][i] ^ PR2[a1][i]), so the prefix over
// v's rows is x_v^L x_s^L Q^L, Q^L = sum_{i,j in L} Q_ij, with
//   Q_ij = XOR over v's rows f <= e of z_{u_f,i} g_{f,j}.
// PR3 stores Q symmetrised (pair_form): k(k+1)/2 values per row, independent
// of the point chunk; the factor x_v x_s is applied by the next layer's reads.
// Two passes: third_pair_rows writes every row's own term (rows in parallel),
// pair_prefix_warp turns them into the running XOR along each head's rows.
// ---------------------------------------------------------------------------
// The (i, j), i >= j, of pair value q = i(i+1)/2 + j.
__device__ __forceinline__ void pair_of(uint32_t q, uint32_t &i, uint32_t &j)
{
    i = (uint32_t)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    if ((i + 1) * (i + 2) / 2 <= q) ++i;  // exact integer correction of the estimate
    if (i * (i + 1) / 2 > q) --i;
    j = q - i * (i + 1) / 2;
}

// Row e (of the deep list's count rows) per warp: its own term
// z_{u_e,i} g_{e,j} (+ z_{u_e,j} g_{e,i}) at PR3 row e + 1. A lane owns pair
// values lane, lane+32, ...; label lanes i < k hold g_i and z_i.
__device__ __forceinline__ void third_pair_row(const V2Params &p, uint32_t e, uint64_t *__restrict__ pr3)
{
    const int lane = threadIdx.x & 31;
    const uint32_t k = p.k;
    const uint32_t np = pair_count(k);
    const uint32_t a = p.ia[e], b = p.ib[e], u = p.src[e];
    const uint64_t y = sm_draw(p.qd->key_y, (uint64_t)p.eid[e] * 32u + 2u);  // y_{e,3}
    uint64_t z = 0;
    if ((uint32_t)lane < k) z = zval(p, u, lane);
    pdl_enter();  // the layer-2 prefix is read from here on
    uint64_t g = 0;
    if ((uint32_t)lane < k && a != b)
        g = rr_mul(y, p.pr2[(size_t)a * k + lane] ^ p.pr2[(size_t)b * k + lane]);
    uint64_t *row = pr3 + ((size_t)e + 1) * np;
    for (uint32_t q0 = 0; q0 < np; q0 += 32) {  // warp-uniform
        const uint32_t q = q0 + (uint32_t)lane;
        uint32_t i = 0, j = 0;
        if (q < np) pair_of(q, i, j);
        const uint64_t gi = shfl64b(g, (int)i), gj = shfl64b(g, (int)j);
        const uint64_t zi = shfl64b(z, (int)i), zj = shfl64b(z, (int)j);
        if (q < np) row[q] = i == j ? rr_mul(zi, gi) : rr_mul(zi, gj) ^ rr_mul(zj, gi);
    }
}

// Both passes in one for a graph whose deep-row ranges are all short (a few
// rows): one warp per range, the running XOR kept in registers (lane owns pair
// values lane + 32 sl). Saves a launch where the launches dominate.
constexpr int kPairSlots = 7;  // ceil(kMaxPairs / 32)

__device__ __forceinline__ void third_pair_fused(const V2Params &p, uint32_t item,
                                                 uint64_t *__restrict__ pr3)
{
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t k = p.k;
    const uint32_t np = pair_count(k);
    const uint64_t key_y = p.qd->key_y;
    uint32_t pi[kPairSlots], pj[kPairSlots];
    uint64_t acc[kPairSlots];
#pragma unroll
    for (int sl = 0; sl < kPairSlots; ++sl) {
        const uint32_t q = (uint32_t)lane + 32u * sl;
        uint32_t i = 0, j = 0;
        if (q < np) pair_of(q, i, j);
        pi[sl] = i;
        pj[sl] = j;
        acc[sl] = 0;
    }
    uint32_t cur = p.head[it.x];
    bool waited = false;
    for (uint32_t e = it.x; e < it.y; ++e) {
        const uint32_t h = p.head[e];
        const uint32_t a = p.ia[e], b = p.ib[e], u = p.src[e];
        const uint64_t y = sm_draw(key_y, (uint64_t)p.eid[e] * 32u + 2u);  // y_{e,3}
        uint64_t z = 0;
        if ((uint32_t)lane < k) z = zval(p, u, lane);
        if (!waited) {
            pdl_enter();  // the layer-2 prefix is read from here on
            waited = true;
        }
        if (h != cur) {
#pragma unroll
            for (int sl = 0; sl < kPairSlots; ++sl) acc[sl] = 0;
            cur = h;
        }
        uint64_t g = 0;
        if ((uint32_t)lane < k && a != b)
            g = rr_mul(y, p.pr2[(size_t)a * k + lane] ^ p.pr2[(size_t)b * k + lane]);
        uint64_t *row = pr3 + ((size_t)e + 1) * np;
#pragma unroll
        for (int sl = 0; sl < kPairSlots; ++sl) {
            if (32u * sl >= np) break;  // warp-uniform
            const uint64_t gi = shfl64b(g, (int)pi[sl]), gj = shfl64b(g, (int)pj[sl]);
            const uint64_t zi = shfl64b(z, (int)pi[sl]), zj = shfl64b(z, (int)pj[sl]);
            if ((uint32_t)lane + 32u * sl < np) {
                acc[sl] ^= pi[sl] == pj[sl] ? rr_mul(zi, gi) : rr_mul(zi, gj) ^ rr_mul(zj, gi);
                row[lane + 32 * sl] = acc[sl];
            }
        }
    }
}

// The running XOR of the rows' terms along each head's rows of a scheduling
// range (in place; ranges cut inside a head are joined by the carry fix-up).
// One pass per 32 pair values; 8 rows' loads in flight at a time.
__device__ __forceinline__ void pair_prefix_warp(const V2Params &p, uint32_t item,
                                                 uint64_t *__restrict__ pr3)
{
    constexpr uint32_t R = 8;
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t np = pair_count(p.k);
    bool waited = false;
    for (uint32_t q0 = 0; q0 < np; q0 += 32) {  // warp-uniform
        const uint32_t q = q0 + (uint32_t)lane;
        const bool qv = q < np;
        uint64_t acc = 0;
        uint32_t cur = p.head[it.x];
        for (uint32_t base = it.x; base < it.y; base += 32) {
            const uint32_t ent = base + lane;
            const uint32_t m_head = ent < it.y ? p.head[ent] : 0u;
            if (!waited) {
                pdl_enter();  // the rows' terms are read from here on
                waited = true;
            }
            const uint32_t nb = min(32u, it.y - base);
            for (uint32_t t = 0; t < nb; t += R) {
                uint64_t v[R];
#pragma unroll
                for (uint32_t r = 0; r < R; ++r)
                    v[r] = (qv && t + r < nb) ? pr3[((size_t)base + t + r + 1) * np + q] : 0ull;
#pragma unroll
                for (uint32_t r = 0; r < R; ++r) {
                    if (t + r < nb) {  // warp-uniform
                        const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)(t + r));
                        if (h != cur) {
                            acc = 0;
                            cur = h;
                        }
                        acc ^= v[r];
                        if (qv) pr3[((size_t)base + t + r + 1) * np + q] = acc;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Carry fix-up of a cut head segment [b, e) of a row list whose prefix rows
// (entry + 1) hold `width` words each (1: scalar layer-1 prefix, k: label
// space, chunk: per-point, groups*(lg+1): transformed). Every piece of
// RowList::kMaxRun entries was computed from zero; the stored forms are all
// XOR-linear, so adding the full prefix at the previous piece's last row fixes
// a piece. Phase 1 walks the pieces' last rows in order (one thread per
// column); phase 2 (after phase 1 of the segment has finished) fixes the other
// rows, cut into tasks of kFixRows row slots. COHERENT reads state through L2
// when it was written earlier in the same launch.
// ---------------------------------------------------------------------------
constexpr uint32_t kFixRows = 64;

template <bool COHERENT>
__device__ __forceinline__ uint64_t ld_state(const uint64_t *q)
{
    return COHERENT ? __ldcg(q) : *q;
}

template <bool COHERENT>
__device__ __forceinline__ void fixup_phase1(uint64_t *__restrict__ buf, uint32_t width, uint32_t b,
                                             uint32_t e, uint32_t tid, uint32_t nthreads)
{
    constexpr uint32_t R = RowList::kMaxRun;
    constexpr uint32_t kAhead = 8;  // pieces whose last rows are loaded together
    for (uint32_t c = tid; c < width; c += nthreads) {
        uint64_t carry = ld_state<COHERENT>(buf + (size_t)(b + R) * width + c);  // piece 0's last row
        for (uint32_t ps0 = b + R; ps0 < e; ps0 += kAhead * R) {
            // the last rows of up to kAhead pieces [ps, pe) (rows ps+1 .. pe) are
            // independent loads; only the running XOR is a chain
            uint64_t v[kAhead];
#pragma unroll
            for (uint32_t i = 0; i < kAhead; ++i) {
                const uint32_t ps = ps0 + i * R;
                v[i] = ps < e ? ld_state<COHERENT>(buf + (size_t)min(e, ps + R) * width + c) : 0ull;
            }
#pragma unroll
            for (uint32_t i = 0; i < kAhead; ++i) {
                const uint32_t ps = ps0 + i * R;
                if (ps < e) {
                    carry ^= v[i];
                    buf[(size_t)min(e, ps + R) * width + c] = carry;
                }
            }
        }
    }
}

// Row slots of a cut segment: piece p >= 1 contributes slots for its rows
// ps+1 .. ps+R-1 (its last row is handled by phase 1), R-1 slots per piece.
__device__ __forceinline__ uint32_t fixup_slots(uint32_t b, uint32_t e)
{
    constexpr uint32_t R = RowList::kMaxRun;
    return ((e - b + R - 1) / R - 1) * (R - 1);
}

template <bool COHERENT>
__device__ __forceinline__ void fixup_phase2(uint64_t *__restrict__ buf, uint32_t width, uint32_t b,
                                             uint32_t e, uint32_t slot0, uint32_t tid, uint32_t nthreads)
{
    constexpr uint32_t R = RowList::kMaxRun;
    const uint32_t slots = min(kFixRows, fixup_slots(b, e) - slot0);
    const uint64_t total = (uint64_t)slots * width;
    for (uint64_t idx = tid; idx < total; idx += nthreads) {
        const uint32_t c = (uint32_t)(idx % width);
        const uint32_t slot = slot0 + (uint32_t)(idx / width);
        const uint32_t piece = 1 + slot / (R - 1);
        const uint32_t ps = b + piece * R;
        const uint32_t row = ps + 1 + slot % (R - 1);
        if (row >= min(e, ps + R)) continue;  // past a short last piece, or its last row
        buf[(size_t)row * width + c] ^= ld_state<COHERENT>(buf + (size_t)ps * width + c);
    }
}

// Lazy form of phase 1 for the one-query kernels' per-point state: instead of
// fixing rows in place, writes for every piece p >= 1 of the cut segment [b, e)
// the carry into it -- the XOR of the totals (last rows) of pieces 0..p-1 --
// to row slot0 + p - 1 of the carry table; readers add it (V2Params::carry).
__device__ __forceinline__ void carry_rows(const uint64_t *__restrict__ buf, uint64_t *__restrict__ carry,
                                           uint32_t width, uint32_t b, uint32_t e, uint32_t slot0,
                                           uint32_t tid, uint32_t nthreads)
{
    constexpr uint32_t R = RowList::kMaxRun;
    constexpr uint32_t kAhead = 8;  // pieces whose last rows are loaded together
    for (uint32_t c = tid; c < width; c += nthreads) {
        uint64_t acc = 0;
        uint32_t slot = slot0;
        // piece p-1 = entries [b + (p-1)R, b + pR): its last row is b + pR
        for (uint32_t ps0 = b + R; ps0 < e; ps0 += kAhead * R) {
            uint64_t v[kAhead];
#pragma unroll
            for (uint32_t i = 0; i < kAhead; ++i) {
                const uint32_t ps = ps0 + i * R;  // the start entry of piece p
                v[i] = ps < e ? buf[(size_t)ps * width + c] : 0ull;
            }
#pragma unroll
            for (uint32_t i = 0; i < kAhead; ++i) {
                if (ps0 + i * R < e) {
                    acc ^= v[i];
                    carry[(size_t)slot * width + c] = acc;
                    ++slot;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Last layer from the transformed state: lane (g, j) accumulates
// sum_e y_{e,k-1} T_{g,j}(W_e) over the rows e of one head vertex v, then
// multiplies once by z_{v,j} (j < lg) or by the XOR of z_{v,j'} over the
// group's fixed high labels j' (slot lg), and the warp XOR-reduces into S[v].
// PB: the state is the pair tail's sums of a larger query (p.blk_groups blocks
// of kPairTailSlots per row), whose slots 1 + j and 0 are T_{g,j} and the
// group total.
// ---------------------------------------------------------------------------
template <int LG, bool COHERENT, bool PB = false>
__device__ __forceinline__ void last_pass(const V2Params &p, uint32_t task, uint32_t g0, bool first)
{
    const int lane = threadIdx.x & 31;
    const uint2 it = p.items[task];
    const uint32_t k = p.k;
    const uint64_t key_y = p.qd->key_y;
    uint64_t *const S = p.qd->S;
    uint64_t *const E = p.qd->E;  // per-edge sums wanted (fine-grained output)
    constexpr uint32_t kGroupsPerPass = 32 / (LG + 1);
    // stored values per transformed row
    const uint32_t row_slots = PB ? p.blk_groups * kPairTailSlots : p.ngroups * (LG + 1);
    const uint32_t slots = min(kGroupsPerPass, p.ngroups - g0) * (LG + 1);  // this pass's
    const bool active = (uint32_t)lane < slots;
    const uint32_t g = g0 + (uint32_t)lane / (LG + 1);
    const uint32_t j = (uint32_t)lane % (LG + 1);
    const uint32_t gbase = p.chunk_base + g * (1u << LG);
    const uint32_t col = PB ? g * kPairTailSlots + (j < (uint32_t)LG ? 1u + j : 0u) : g0 * (LG + 1) + (uint32_t)lane;

    auto zsel_of = [&](uint32_t v) -> uint64_t {
        if (!active) return 0ull;
        if (j < (uint32_t)LG) return j < k ? zval(p, v, j) : 0ull;
        uint64_t zz = 0;
        for (uint32_t jj = LG; jj < k; ++jj)
            if ((gbase >> jj) & 1u) zz ^= zval(p, v, jj);
        return zz;
    };

    uint32_t cur = p.head[it.x];
    uint64_t zsel = zsel_of(cur);
    uint64_t acc = 0;
    auto flush = [&](uint32_t v) {
        uint64_t t = active ? rr_mul(zsel, acc) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t ^= shfl64x(t, off);
        if (lane == 0 && t) atomicXor(reinterpret_cast<unsigned long long *>(S + v),
                                      (unsigned long long)t);
    };
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t m_head = has ? p.head[ent] : 0u;
        const uint32_t m_a = has ? p.ia[ent] : 0u;
        const uint32_t m_b = has ? p.ib[ent] : 0u;
        const uint32_t m_eid = has ? p.eid[ent] : 0u;
        const uint64_t m_y = has ? sm_draw(key_y, (uint64_t)m_eid * 32u + (p.layer - 1u)) : 0ull;
        if constexpr (!COHERENT) {
            if (first && base == it.x) pdl_enter();  // the transformed state is read from here on
        }
        const uint32_t nb = min(32u, it.y - base);
        for (uint32_t t = 0; t < nb; ++t) {
            const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)t);
            if (h != cur) {
                flush(cur);
                acc = 0;
                cur = h;
                zsel = zsel_of(cur);
            }
            const uint32_t a = __shfl_sync(0xffffffffu, m_a, (int)t);
            const uint32_t b = __shfl_sync(0xffffffffu, m_b, (int)t);
            const uint64_t y = shfl64b(m_y, (int)t);
            uint64_t yt = 0;
            if (active) {
                const uint64_t *sa = p.st_in + (size_t)a * row_slots + col;
                const uint64_t *sb = p.st_in + (size_t)b * row_slots + col;
                const uint64_t tv = COHERENT ? (__ldcg(sa) ^ __ldcg(sb)) : (*sa ^ *sb);
                yt = rr_mul(y, tv);
                acc ^= yt;
            }
            if (E) {
                // this entry's own sum over the pass's points: the flush's
                // product taken per entry instead of per head
                uint64_t c = active ? rr_mul(zsel, yt) : 0ull;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) c ^= shfl64x(c, off);
                const uint32_t e = __shfl_sync(0xffffffffu, m_eid, (int)t);
                if (lane == 0 && c) atomicXor(reinterpret_cast<unsigned long long *>(E + e),
                                              (unsigned long long)c);
            }
        }
    }
    flush(cur);
}

// A warp covers 32 / (LG + 1) point groups at a time (one lane per stored
// value); a chunk with more groups takes several passes over the rows.
template <int LG, bool COHERENT, bool PB = false>
__device__ __forceinline__ void last_warp(const V2Params &p, uint32_t task)
{
    constexpr uint32_t kGroupsPerPass = 32 / (LG + 1);
#pragma unroll 1
    for (uint32_t g0 = 0; g0 < p.ngroups; g0 += kGroupsPerPass)
        last_pass<LG, COHERENT, PB>(p, task, g0, g0 == 0);
}

// ---------------------------------------------------------------------------
// Pair tail, layer k-2 in label space. The last layer uses layer k-2 only
// through sum over a group g's points of x_w^L P^L(f), and with
// P^L = y x_v^L W^L (a row of head v, W its window of layer k-3) that sum is a
// bilinear form in the z values of w and v over the pair sums of W: writing
// x^L = sum_{i in I, i in L} z_i + A_g (I = the LG in-group labels, A_g = sum
// of z_j over the labels above them that every point of g holds),
//   sum_{L in g} x_w^L x_v^L W^L = sum_{i,j in I} zw_i zv_j T_g{i,j}
//       + sum_i zw_i A_{v,g} T_g{i} + A_{w,g} sum_j zv_j T_g{j} + A_{w,g} A_{v,g} V_g,
// T_g{i,j} the sum of W^L over g's points holding labels i and j (T_g{i,i} =
// T_g{i}), V_g over all of g's points. Grouped by w's factors, a row adds
//   G_i     = y (sum_{j in I} zv_j sum_g T_g{i,j} + sum_g A_{v,g} T_g{i})   (i in I)
//   G_{g,*} = y (sum_{j in I} zv_j T_g{j} + A_{v,g} V_g)                     (g < ng)
// and the last layer takes sum_i zw_i dR_i + sum_g A_{w,g} dR_{g,*} from the
// windows of R, the prefix of G over v's rows (stride kLabelTailWidth).
// One warp per scheduling range of the deep rows. Per row with a non-empty
// window: lane l forms the y-scaled multiplier m_l (y zv_l for l < LG,
// y A_{v,l-LG} above); lane s of the slot pass sums slot s of the window over
// the groups and multiplies it by the multipliers its label pair or single
// label needs; lane q of each group pass takes (group q/8, slot q%8) of the
// singles and totals. The products meet their targets in `sm` (192 values).
// COHERENT: the pair sums were written earlier in the same launch (read
// through L2).
// ---------------------------------------------------------------------------
template <int LG, bool COHERENT>
__device__ __forceinline__ void label_tail_warp(const V2Params &p, uint32_t item, uint64_t *sm)
{
    constexpr uint32_t NS = 1u + LG + LG * (LG - 1) / 2;  // used slots of a group block
    constexpr uint32_t kPB = 64;                          // group-pass products at sm[kPB..]
    const uint32_t lane = threadIdx.x & 31;
    const uint2 it = p.items[item];
    const uint32_t k = p.k;
    const uint32_t ng = p.ngroups;
    const uint64_t key_y = p.qd->key_y;
    const uint32_t blk_w = ng * kPairTailSlots;            // values per input row
    const uint32_t rb_passes = (ng * 8u + 31u) / 32u;      // group passes (ng <= 8: at most 2)
    const uint32_t ntarget = LG + ng;
    auto ld = [](const uint64_t *q) { return COHERENT ? __ldcg(q) : __ldg(q); };

    // slot pass: what lane s computes (s < NS). single i: P0 = m_i T -> R_i;
    // pair (i < j): P0 = m_j T -> R_i and P1 = m_i T -> R_j; s = 0 (total):
    // nothing. Packed: bits 0-4 the lane of P0's multiplier, 5-9 P1's, bit 10
    // / 11 set when P0 / P1 is used.
    uint32_t dec = 0;
    if (lane >= 1 && lane <= (uint32_t)LG) {
        dec = (lane - 1) | (1u << 10);
    } else if (lane > (uint32_t)LG && lane < NS) {
        const uint32_t idx = lane - 1 - LG;
        uint32_t j = 1;
        while ((j + 1) * j / 2 <= idx) ++j;  // largest j with j(j-1)/2 <= idx
        const uint32_t i = idx - j * (j - 1) / 2;
        dec = j | (i << 5) | (3u << 10);
    }
    // target lane t: the smem positions it sums (see the gather below)
    uint32_t cur = p.head[it.x];
    uint64_t M = 0;  // lane l < LG: zv_l; lane LG+g: A_{v,g}
    auto enter_head = [&](uint32_t v) {
        const uint64_t zv = lane < k ? zval(p, v, lane) : 0ull;
        const uint32_t gbase = p.chunk_base + (lane - (uint32_t)LG) * (1u << LG);
        uint64_t a = 0;
        for (uint32_t j = LG; j < k; ++j) {  // warp-uniform
            const uint64_t zj = shfl64b(zv, (int)j);
            if ((gbase >> j) & 1u) a ^= zj;
        }
        M = lane < (uint32_t)LG ? zv : (lane < ntarget ? a : 0ull);
    };
    enter_head(cur);
    uint64_t R = 0;
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t m_head = has ? p.head[ent] : 0u;
        const uint32_t m_a = has ? p.ia[ent] : 0u;
        const uint32_t m_b = has ? p.ib[ent] : 0u;
        const uint64_t m_coef = has ? sm_draw(key_y, (uint64_t)p.eid[ent] * 32u + (p.layer - 1u)) : 0ull;
        if (base == it.x) pdl_enter();  // the pair sums are read, and R written, from here on
        const uint32_t nb = min(32u, it.y - base);
        for (uint32_t t = 0; t < nb; ++t) {
            const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)t);
            if (h != cur) {
                R = 0;
                cur = h;
                enter_head(cur);
            }
            const uint32_t a = __shfl_sync(0xffffffffu, m_a, (int)t);
            const uint32_t b = __shfl_sync(0xffffffffu, m_b, (int)t);
            const uint64_t y = shfl64b(m_coef, (int)t);
            if (a != b) {  // warp-uniform
                const uint64_t m = rr_mul(y, M);
                const uint64_t *ra = p.st_in + (size_t)a * blk_w;
                const uint64_t *rb = p.st_in + (size_t)b * blk_w;
                // slot pass
                uint64_t ts = 0;
                if (lane < NS)
                    for (uint32_t g = 0; g < ng; ++g)
                        ts ^= ld(rb + g * kPairTailSlots + lane) ^ ld(ra + g * kPairTailSlots + lane);
                const uint64_t mA = shfl64b(m, (int)(dec & 31u)), mB = shfl64b(m, (int)((dec >> 5) & 31u));
                sm[2 * lane] = rr_mul((dec >> 10) & 1u ? mA : 0ull, ts);
                sm[2 * lane + 1] = rr_mul((dec >> 11) & 1u ? mB : 0ull, ts);
                // group passes: (g, s) = (q / 8, q % 8); s = 0 the total V_g,
                // s = 1 + i the single T_g{i}: P0 = A'_g T -> R_i (s > 0) or
                // R_{g,*} (s = 0), P1 = m_i T -> R_{g,*} (s > 0)
                for (uint32_t r = 0; r < rb_passes; ++r) {
                    const uint32_t q = lane + 32u * r;
                    const uint32_t g = q >> 3, s = q & 7u;
                    const bool ok = g < ng && s <= (uint32_t)LG;
                    const uint64_t tv = ok ? (ld(rb + g * kPairTailSlots + s) ^
                                              ld(ra + g * kPairTailSlots + s)) : 0ull;
                    const uint64_t mg = shfl64b(m, (int)min((uint32_t)LG + g, 31u));
                    const uint64_t mi = shfl64b(m, (int)(s == 0 ? 0u : s - 1u));
                    sm[kPB + 2 * q] = rr_mul(ok ? mg : 0ull, tv);
                    sm[kPB + 2 * q + 1] = rr_mul(ok && s > 0 ? mi : 0ull, tv);
                }
                __syncwarp();
                uint64_t G = 0;
                if (lane < (uint32_t)LG) {
                    const uint32_t i = lane;
                    for (uint32_t o = 0; o < (uint32_t)LG; ++o) {
                        const uint32_t lo = min(i, o), hi = max(i, o);
                        const uint32_t slot = lo == hi ? 1u + i : 1u + LG + hi * (hi - 1) / 2 + lo;
                        G ^= sm[2 * slot + (i > o ? 1u : 0u)];
                    }
                    for (uint32_t g = 0; g < ng; ++g) G ^= sm[kPB + 2 * (g * 8u + 1u + i)];
                } else if (lane < ntarget) {
                    const uint32_t g = lane - LG;
                    G = sm[kPB + 2 * (g * 8u)];
                    for (uint32_t i = 0; i < (uint32_t)LG; ++i) G ^= sm[kPB + 2 * (g * 8u + 1u + i) + 1];
                }
                __syncwarp();
                R ^= G;
            }
            const size_t row = (size_t)base + t + 1;  // deep row of this entry
            if (lane < kLabelTailWidth) p.st_out[row * kLabelTailWidth + lane] = R;
        }
    }
}

// Last layer of the pair tail: lane t < LG + ng accumulates sum_f y_f dR_t over
// the rows f of one head vertex w (dR = the window of R), then multiplies once
// by zw_t (t < LG) or A_{w,t-LG}, and the warp XOR-reduces into S[w].
template <int LG, bool COHERENT>
__device__ __forceinline__ void last_label_warp(const V2Params &p, uint32_t task)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint2 it = p.items[task];
    const uint32_t k = p.k;
    const uint64_t key_y = p.qd->key_y;
    uint64_t *const S = p.qd->S;
    uint64_t *const E = p.qd->E;  // per-edge sums wanted (fine-grained output)
    const bool active = lane < (uint32_t)LG + p.ngroups;
    const uint32_t gbase = p.chunk_base + (lane - (uint32_t)LG) * (1u << LG);  // lanes >= LG

    auto zsel_of = [&](uint32_t v) -> uint64_t {
        if (!active) return 0ull;
        if (lane < (uint32_t)LG) return lane < k ? zval(p, v, lane) : 0ull;
        uint64_t zz = 0;
        for (uint32_t j = LG; j < k; ++j)
            if ((gbase >> j) & 1u) zz ^= zval(p, v, j);
        return zz;
    };

    uint32_t cur = p.head[it.x];
    uint64_t zsel = zsel_of(cur);
    uint64_t acc = 0;
    auto flush = [&](uint32_t v) {
        uint64_t t = active ? rr_mul(zsel, acc) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t ^= shfl64x(t, off);
        if (lane == 0 && t) atomicXor(reinterpret_cast<unsigned long long *>(S + v),
                                      (unsigned long long)t);
    };
    for (uint32_t base = it.x; base < it.y; base += 32) {
        const uint32_t ent = base + lane;
        const bool has = ent < it.y;
        const uint32_t m_head = has ? p.head[ent] : 0u;
        const uint32_t m_a = has ? p.ia[ent] : 0u;
        const uint32_t m_b = has ? p.ib[ent] : 0u;
        const uint32_t m_eid = has ? p.eid[ent] : 0u;
        const uint64_t m_y = has ? sm_draw(key_y, (uint64_t)m_eid * 32u + (p.layer - 1u)) : 0ull;
        if (base == it.x) pdl_enter();  // R is read from here on
        const uint32_t nb = min(32u, it.y - base);
        for (uint32_t t = 0; t < nb; ++t) {
            const uint32_t h = __shfl_sync(0xffffffffu, m_head, (int)t);
            if (h != cur) {
                flush(cur);
                acc = 0;
                cur = h;
                zsel = zsel_of(cur);
            }
            const uint32_t a = __shfl_sync(0xffffffffu, m_a, (int)t);
            const uint32_t b = __shfl_sync(0xffffffffu, m_b, (int)t);
            const uint64_t y = shfl64b(m_y, (int)t);
            uint64_t yt = 0;
            if (active && a != b) {
                const uint64_t *ra = p.st_in + (size_t)a * kLabelTailWidth + lane;
                const uint64_t *rb = p.st_in + (size_t)b * kLabelTailWidth + lane;
                const uint64_t dr = COHERENT ? (__ldcg(ra) ^ __ldcg(rb)) : (__ldg(ra) ^ __ldg(rb));
                yt = rr_mul(y, dr);
                acc ^= yt;
            }
            if (E) {
                // this entry's own sum: the flush's product taken per entry
                uint64_t c = active ? rr_mul(zsel, yt) : 0ull;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) c ^= shfl64x(c, off);
                const uint32_t e = __shfl_sync(0xffffffffu, m_eid, (int)t);
                if (lane == 0 && c) atomicXor(reinterpret_cast<unsigned long long *>(E + e),
                                              (unsigned long long)c);
            }
        }
    }
    flush(cur);
}

}  // namespace rr
