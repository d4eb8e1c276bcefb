// rr_graph.cu -- graph load: in-edge CSR sorted by (head, time, edge index),
// restless windows and the windowed-prefix state layout.
//
// Window of an edge e = (u, v, t_e) (Eq. (1): the walk may continue along e
// from any walk that arrived at u by an edge f with t_f <= t_e <= t_f +
// delta(u); restless-walk definition): the rows f of u's in-segment with
// t_e - delta(u) <= t_f <= t_e, a contiguous range [lo, hi) because the
// segment is sorted by time.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstring>
#include <numeric>

#include "rr_internal.h"

namespace rr {
namespace {

constexpr uint32_t kItemRows = 64;      // target rows per scheduling range
constexpr uint32_t kItemMaxVerts = 512; // cap on vertices per range

__global__ void k_make_keys(const uint32_t *__restrict__ dst, const uint32_t *__restrict__ t,
                            uint64_t m, uint64_t *__restrict__ key, uint32_t *__restrict__ val)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        key[e] = ((uint64_t)dst[e] << 32) | t[e];
        val[e] = (uint32_t)e;
    }
}

// Unpacks the sorted keys and gathers each row's tail vertex.
__global__ void k_unpack_rows(const uint64_t *__restrict__ key, const uint32_t *__restrict__ eid,
                              const uint32_t *__restrict__ src, uint64_t m,
                              uint32_t *__restrict__ row_t, uint32_t *__restrict__ row_dst,
                              uint32_t *__restrict__ row_src)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[r];
        row_t[r] = (uint32_t)k;
        row_dst[r] = (uint32_t)(k >> 32);
        row_src[r] = src[eid[r]];
    }
}

// off[v] = number of rows whose head is < v, for v = 0..n. Row r closes the
// vertices (head(r-1), head(r)] (head(-1) = -1, head(m) = n), so every v is
// written exactly once.
__global__ void k_offsets(const uint32_t *__restrict__ row_dst, uint64_t m, uint32_t n,
                          uint32_t *__restrict__ off)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        int64_t hp = (r == 0) ? -1 : (int64_t)row_dst[r - 1];
        int64_t hc = (r == m) ? (int64_t)n : (int64_t)row_dst[r];
        for (int64_t v = hp + 1; v <= hc; ++v) off[v] = (uint32_t)r;
    }
}

__device__ __forceinline__ uint32_t lower_bound_t(const uint32_t *__restrict__ row_t, uint32_t lo,
                                                  uint32_t hi, int64_t key)
{
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)row_t[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Window [lo, hi) of every row (absolute rows of the tail's in-segment) and,
// in compact mode, a +1/-1 difference array marking rows covered by some window.
__global__ void k_windows(const uint32_t *__restrict__ row_t, const uint32_t *__restrict__ row_src,
                          const uint32_t *__restrict__ off, const uint32_t *__restrict__ delta,
                          uint64_t m, uint32_t *__restrict__ lo_out, uint32_t *__restrict__ hi_out,
                          int32_t *__restrict__ diff, unsigned long long *__restrict__ nonempty)
{
    uint32_t local = 0;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = row_src[r];
        int64_t te = row_t[r];
        int64_t first = te - (int64_t)delta[u];
        uint32_t s0 = off[u], s1 = off[u + 1];
        uint32_t lo = lower_bound_t(row_t, s0, s1, first);
        uint32_t hi = lower_bound_t(row_t, lo, s1, te + 1);
        lo_out[r] = lo;
        hi_out[r] = hi;
        if (hi > lo) {
            ++local;
            if (diff) {
                atomicAdd(&diff[lo], 1);
                atomicAdd(&diff[hi], -1);
            }
        }
    }
    if (local) atomicAdd(nonempty, (unsigned long long)local);
}

__global__ void k_dense_flags(uint64_t m, uint32_t *__restrict__ prod)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x)
        prod[r] = 1u;
}

__global__ void k_cover_to_flags(const int32_t *__restrict__ cover, uint64_t m,
                                 uint32_t *__restrict__ prod)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x)
        prod[r] = cover[r] > 0 ? 1u : 0u;
}

// rank[r] = number of producer rows in [0, r] (inclusive scan of the flags).
// Producer r owns state row rank[r]; a window [lo, hi) reads
// state[rank[hi-1]] ^ state[rank of the last producer before lo in the same
// segment, or 0].
__global__ void k_state_index(const uint32_t *__restrict__ rank, const uint32_t *__restrict__ prod,
                              const uint32_t *__restrict__ lo_in, const uint32_t *__restrict__ hi_in,
                              const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ off,
                              uint64_t m, uint32_t *__restrict__ row_a, uint32_t *__restrict__ row_b,
                              uint32_t *__restrict__ row_s,
                              unsigned long long *__restrict__ prod_window)
{
    uint32_t local = 0;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        row_s[r] = prod[r] ? rank[r] : 0u;
        if (prod[r] && hi_in[r] > lo_in[r]) ++local;
        uint32_t lo = lo_in[r], hi = hi_in[r];
        if (hi > lo) {
            row_a[r] = rank[hi - 1];
            uint32_t s0 = off[row_src[r]];
            uint32_t before_seg = s0 ? rank[s0 - 1] : 0u;
            uint32_t before_lo = lo ? rank[lo - 1] : 0u;
            row_b[r] = (lo > s0 && before_lo > before_seg) ? before_lo : 0u;
        } else {
            row_a[r] = 0u;
            row_b[r] = 0u;
        }
    }
    if (local) atomicAdd(prod_window, (unsigned long long)local);
}

__global__ void k_v2_flags(const uint32_t *__restrict__ lo_in, const uint32_t *__restrict__ hi_in,
                           const uint32_t *__restrict__ tprod, uint64_t m,
                           uint32_t *__restrict__ c0, uint32_t *__restrict__ c1)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = hi_in[r] > lo_in[r] ? 1u : 0u;
        c0[r] = w;
        c1[r] = w & tprod[r];
    }
}

// Last entry of an inclusive rank array at or before row x inside the segment
// that starts at s0: rank[x] if it counts a flagged row of the segment, else 0.
__device__ __forceinline__ uint32_t rank_in_segment(const uint32_t *__restrict__ rank, int64_t x,
                                                    uint32_t s0)
{
    if (x < (int64_t)s0) return 0u;
    const uint32_t before = s0 ? rank[s0 - 1] : 0u;
    const uint32_t at = rank[x];
    return at > before ? at : 0u;
}

__global__ void k_v2_index(const uint32_t *__restrict__ lo_in, const uint32_t *__restrict__ hi_in,
                           const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ off,
                           const uint32_t *__restrict__ rank_p, const uint32_t *__restrict__ rank1,
                           uint64_t m, uint32_t *__restrict__ a0, uint32_t *__restrict__ b0,
                           uint32_t *__restrict__ a1, uint32_t *__restrict__ b1,
                           uint32_t *__restrict__ c2)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t lo = lo_in[r], hi = hi_in[r];
        if (hi > lo) {
            const uint32_t s0 = off[row_src[r]];
            a0[r] = rank_in_segment(rank_p, (int64_t)hi - 1, s0);
            b0[r] = rank_in_segment(rank_p, (int64_t)lo - 1, s0);
            a1[r] = rank_in_segment(rank1, (int64_t)hi - 1, s0);
            b1[r] = rank_in_segment(rank1, (int64_t)lo - 1, s0);
            c2[r] = a1[r] != b1[r] ? 1u : 0u;
        } else {
            a0[r] = b0[r] = a1[r] = b1[r] = 0u;
            c2[r] = 0u;
        }
    }
}

struct ListOut {
    uint32_t *head, *eid, *src, *a0, *b0, *a1, *b1, *a3, *b3;
};

// deep rows: state rows (c1) whose window holds a state row (a1 != b1)
__global__ void k_v2_deep(const uint32_t *__restrict__ c1, const uint32_t *__restrict__ a1,
                          const uint32_t *__restrict__ b1, uint64_t m, uint32_t *__restrict__ d)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x)
        d[r] = (c1[r] && a1[r] != b1[r]) ? 1u : 0u;
}

// window of every row in deep-row indices, and the flag "window holds a deep row"
__global__ void k_v2_index3(const uint32_t *__restrict__ lo_in, const uint32_t *__restrict__ hi_in,
                            const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ off,
                            const uint32_t *__restrict__ rank_d, uint64_t m,
                            uint32_t *__restrict__ a3, uint32_t *__restrict__ b3,
                            uint32_t *__restrict__ c4)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t lo = lo_in[r], hi = hi_in[r];
        if (hi > lo) {
            const uint32_t s0 = off[row_src[r]];
            a3[r] = rank_in_segment(rank_d, (int64_t)hi - 1, s0);
            b3[r] = rank_in_segment(rank_d, (int64_t)lo - 1, s0);
        } else {
            a3[r] = b3[r] = 0u;
        }
        c4[r] = a3[r] != b3[r] ? 1u : 0u;
    }
}

// entries of the deep list and of the k >= 5 last-layer list
__global__ void k_v2_scatter3(const uint32_t *__restrict__ row_dst, const uint32_t *__restrict__ row_eid,
                              const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ a1,
                              const uint32_t *__restrict__ b1, const uint32_t *__restrict__ a3,
                              const uint32_t *__restrict__ b3, const uint32_t *__restrict__ d,
                              const uint32_t *__restrict__ rank_d, const uint32_t *__restrict__ c4,
                              const uint32_t *__restrict__ rank4, uint64_t m, ListOut D, ListOut T)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        if (d[r]) {
            const uint32_t i = rank_d[r] - 1;
            D.head[i] = row_dst[r]; D.eid[i] = row_eid[r]; D.src[i] = row_src[r];
            D.a1[i] = a1[r]; D.b1[i] = b1[r]; D.a3[i] = a3[r]; D.b3[i] = b3[r];
        }
        if (c4[r]) {
            const uint32_t i = rank4[r] - 1;
            T.head[i] = row_dst[r]; T.eid[i] = row_eid[r]; T.src[i] = row_src[r];
            T.a3[i] = a3[r]; T.b3[i] = b3[r];
        }
    }
}

__global__ void k_v2_scatter(const uint32_t *__restrict__ row_dst, const uint32_t *__restrict__ row_eid,
                             const uint32_t *__restrict__ row_src, const uint32_t *__restrict__ a0,
                             const uint32_t *__restrict__ b0, const uint32_t *__restrict__ a1,
                             const uint32_t *__restrict__ b1, const uint32_t *__restrict__ tprod,
                             const uint32_t *__restrict__ rank_p, const uint32_t *__restrict__ c1,
                             const uint32_t *__restrict__ rank1, const uint32_t *__restrict__ c0,
                             const uint32_t *__restrict__ rank0, const uint32_t *__restrict__ c2,
                             const uint32_t *__restrict__ rank2, uint64_t m, ListOut P, ListOut S,
                             ListOut W, ListOut T)
{
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t h = row_dst[r], e = row_eid[r], u = row_src[r];
        if (tprod[r]) {
            const uint32_t i = rank_p[r] - 1;
            P.head[i] = h; P.eid[i] = e; P.src[i] = u;
        }
        if (c1[r]) {
            const uint32_t i = rank1[r] - 1;
            S.head[i] = h; S.eid[i] = e; S.src[i] = u;
            S.a0[i] = a0[r]; S.b0[i] = b0[r]; S.a1[i] = a1[r]; S.b1[i] = b1[r];
        }
        if (c0[r]) {
            const uint32_t i = rank0[r] - 1;
            W.head[i] = h; W.eid[i] = e; W.src[i] = u; W.a0[i] = a0[r]; W.b0[i] = b0[r];
        }
        if (c2[r]) {
            const uint32_t i = rank2[r] - 1;
            T.head[i] = h; T.eid[i] = e; T.src[i] = u; T.a1[i] = a1[r]; T.b1[i] = b1[r];
        }
    }
}

inline unsigned grid_for(uint64_t count, unsigned block)
{
    uint64_t g = (count + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535ull * 8) g = 65535ull * 8;
    return (unsigned)g;
}

}  // namespace

// Builds the (v0, v1) scheduling ranges from the host copy of off: consecutive
// vertices until about kItemRows rows; a vertex with more rows forms its own
// range. Ranges are ordered largest first so big segments start early.
static void build_items(const std::vector<uint32_t> &off, uint32_t n,
                        std::vector<uint32_t> &v0, std::vector<uint32_t> &v1,
                        std::vector<uint32_t> &rows, uint32_t *max_deg)
{
    uint32_t start = 0, acc = 0, nv = 0;
    *max_deg = 0;
    auto flush = [&](uint32_t end) {
        if (acc > 0) {
            v0.push_back(start);
            v1.push_back(end);
            rows.push_back(acc);
        }
        start = end;
        acc = 0;
        nv = 0;
    };
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t d = off[v + 1] - off[v];
        *max_deg = std::max(*max_deg, d);
        if (d >= kItemRows) {
            flush(v);
            acc = d;
            flush(v + 1);
            continue;
        }
        acc += d;
        ++nv;
        if (acc >= kItemRows || nv >= kItemMaxVerts) flush(v + 1);
    }
    flush(n);
}

// Head-aligned scheduling ranges over a row list: consecutive head runs are
// packed until `target` entries; a run of `target` entries or more forms its
// own range(s), cut into pieces of at most RowList::kMaxRun entries (the cut
// runs are returned in `chains`). Ranges are ordered largest first.
static void build_entry_items(const std::vector<uint32_t> &head, uint32_t target,
                              std::vector<uint2> &items, std::vector<uint2> *chains)
{
    std::vector<uint2> tmp;
    const uint32_t maxrun = RowList::kMaxRun;
    const uint64_t cnt = head.size();
    uint64_t start = 0, i = 0;
    while (i < cnt) {
        uint64_t j = i + 1;
        while (j < cnt && head[j] == head[i]) ++j;  // run [i, j)
        if (j - i >= target) {
            if (i > start) tmp.push_back(make_uint2((uint32_t)start, (uint32_t)i));
            for (uint64_t b = i; b < j; b += maxrun)
                tmp.push_back(make_uint2((uint32_t)b, (uint32_t)std::min<uint64_t>(j, b + maxrun)));
            if (chains && j - i > maxrun) chains->push_back(make_uint2((uint32_t)i, (uint32_t)j));
            start = j;
        } else if (j - start >= target) {
            tmp.push_back(make_uint2((uint32_t)start, (uint32_t)j));
            start = j;
        }
        i = j;
    }
    if (cnt > start) tmp.push_back(make_uint2((uint32_t)start, (uint32_t)cnt));
    std::stable_sort(tmp.begin(), tmp.end(),
                     [](const uint2 &a, const uint2 &b) { return (a.y - a.x) > (b.y - b.x); });
    items.swap(tmp);
}

static rr_status scan_u32(const uint32_t *in, uint32_t *out, uint64_t m, DevBuf &tmp,
                          cudaStream_t st)
{
    size_t tb = 0;
    RR_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb, in, out, (int64_t)m, st));
    RR_CUDA(tmp.reserve(tb));
    RR_CUDA(cub::DeviceScan::InclusiveSum(tmp.p, tb, in, out, (int64_t)m, st));
    return RR_OK;
}

// Builds the reduced-state engine's row lists (rr_internal.h, RowList) from
// the windows [row_lo, row_hi), the head of every row and the true producer
// flags (rows inside some window).
rr_status build_lists_v2(Graph &g, const uint32_t *row_dst, const uint32_t *tprod, cudaStream_t st)
{
    const uint64_t m = g.m;
    DevBuf c0, c1, c2, rank_p, rank0, rank1, rank2, a0, b0, a1, b1, tmp;
    for (DevBuf *b : {&c0, &c1, &c2, &rank_p, &rank0, &rank1, &rank2, &a0, &b0, &a1, &b1})
        RR_CUDA(b->reserve(m * 4));
    k_v2_flags<<<grid_for(m, 256), 256, 0, st>>>(g.row_lo.as<uint32_t>(), g.row_hi.as<uint32_t>(),
                                                 tprod, m, c0.as<uint32_t>(), c1.as<uint32_t>());
    RR_LAUNCHED();
    rr_status s;
    if ((s = scan_u32(tprod, rank_p.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
    if ((s = scan_u32(c0.as<uint32_t>(), rank0.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
    if ((s = scan_u32(c1.as<uint32_t>(), rank1.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
    k_v2_index<<<grid_for(m, 256), 256, 0, st>>>(
        g.row_lo.as<uint32_t>(), g.row_hi.as<uint32_t>(), g.row_src.as<uint32_t>(),
        g.off.as<uint32_t>(), rank_p.as<uint32_t>(), rank1.as<uint32_t>(), m, a0.as<uint32_t>(),
        b0.as<uint32_t>(), a1.as<uint32_t>(), b1.as<uint32_t>(), c2.as<uint32_t>());
    RR_LAUNCHED();
    if ((s = scan_u32(c2.as<uint32_t>(), rank2.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
    uint32_t counts[4] = {0, 0, 0, 0};
    RR_CUDA(cudaMemcpyAsync(&counts[0], rank_p.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(&counts[1], rank1.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(&counts[2], rank0.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(&counts[3], rank2.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    RowList *L[4] = {&g.prod_list, &g.state_list, &g.win_list, &g.tail_list};
    ListOut out[4];
    for (int i = 0; i < 4; ++i) {
        RowList &R = *L[i];
        R.count = counts[i];
        const size_t bytes = (size_t)std::max<uint32_t>(1, counts[i]) * 4;
        RR_CUDA(R.head.reserve(bytes));
        RR_CUDA(R.eid.reserve(bytes));
        RR_CUDA(R.src.reserve(bytes));  // the tail list's: the k = 4 closed form's z_v
        if (i == 1 || i == 2) {
            RR_CUDA(R.a0.reserve(bytes));
            RR_CUDA(R.b0.reserve(bytes));
        }
        if (i == 1 || i == 3) {
            RR_CUDA(R.a1.reserve(bytes));
            RR_CUDA(R.b1.reserve(bytes));
        }
        out[i] = ListOut{R.head.as<uint32_t>(), R.eid.as<uint32_t>(), R.src.as<uint32_t>(),
                         R.a0.as<uint32_t>(), R.b0.as<uint32_t>(), R.a1.as<uint32_t>(),
                         R.b1.as<uint32_t>(), nullptr, nullptr};
    }
    k_v2_scatter<<<grid_for(m, 256), 256, 0, st>>>(
        row_dst, g.row_eid.as<uint32_t>(), g.row_src.as<uint32_t>(), a0.as<uint32_t>(),
        b0.as<uint32_t>(), a1.as<uint32_t>(), b1.as<uint32_t>(), tprod, rank_p.as<uint32_t>(),
        c1.as<uint32_t>(), rank1.as<uint32_t>(), c0.as<uint32_t>(), rank0.as<uint32_t>(),
        c2.as<uint32_t>(), rank2.as<uint32_t>(), m, out[0], out[1], out[2], out[3]);
    RR_LAUNCHED();

    // deep rows (layers >= 3) and the last-layer rows that read them
    {
        DevBuf d, rank_d, a3, b3, c4, rank4;
        for (DevBuf *b : {&d, &rank_d, &a3, &b3, &c4, &rank4}) RR_CUDA(b->reserve(m * 4));
        k_v2_deep<<<grid_for(m, 256), 256, 0, st>>>(c1.as<uint32_t>(), a1.as<uint32_t>(),
                                                    b1.as<uint32_t>(), m, d.as<uint32_t>());
        RR_LAUNCHED();
        if ((s = scan_u32(d.as<uint32_t>(), rank_d.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
        k_v2_index3<<<grid_for(m, 256), 256, 0, st>>>(
            g.row_lo.as<uint32_t>(), g.row_hi.as<uint32_t>(), g.row_src.as<uint32_t>(),
            g.off.as<uint32_t>(), rank_d.as<uint32_t>(), m, a3.as<uint32_t>(), b3.as<uint32_t>(),
            c4.as<uint32_t>());
        RR_LAUNCHED();
        if ((s = scan_u32(c4.as<uint32_t>(), rank4.as<uint32_t>(), m, tmp, st)) != RR_OK) return s;
        uint32_t c3[2] = {0, 0};
        RR_CUDA(cudaMemcpyAsync(&c3[0], rank_d.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaMemcpyAsync(&c3[1], rank4.as<uint32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        RowList &D = g.deep_list, &T = g.tail3_list;
        D.count = c3[0];
        T.count = c3[1];
        const size_t db = (size_t)std::max<uint32_t>(1, c3[0]) * 4;
        const size_t tb = (size_t)std::max<uint32_t>(1, c3[1]) * 4;
        for (DevBuf *b : {&D.head, &D.eid, &D.src, &D.a1, &D.b1, &D.a3, &D.b3}) RR_CUDA(b->reserve(db));
        for (DevBuf *b : {&T.head, &T.eid, &T.src, &T.a3, &T.b3}) RR_CUDA(b->reserve(tb));
        ListOut od{D.head.as<uint32_t>(), D.eid.as<uint32_t>(), D.src.as<uint32_t>(), nullptr, nullptr,
                   D.a1.as<uint32_t>(), D.b1.as<uint32_t>(), D.a3.as<uint32_t>(), D.b3.as<uint32_t>()};
        ListOut ot{T.head.as<uint32_t>(), T.eid.as<uint32_t>(), T.src.as<uint32_t>(), nullptr, nullptr,
                   nullptr, nullptr, T.a3.as<uint32_t>(), T.b3.as<uint32_t>()};
        k_v2_scatter3<<<grid_for(m, 256), 256, 0, st>>>(
            row_dst, g.row_eid.as<uint32_t>(), g.row_src.as<uint32_t>(), a1.as<uint32_t>(),
            b1.as<uint32_t>(), a3.as<uint32_t>(), b3.as<uint32_t>(), d.as<uint32_t>(),
            rank_d.as<uint32_t>(), c4.as<uint32_t>(), rank4.as<uint32_t>(), m, od, ot);
        RR_LAUNCHED();
        RR_CUDA(cudaStreamSynchronize(st));
    }
    g.state_compute_rows = g.deep_list.count;
    {
        std::vector<uint32_t> ha(g.deep_list.count), hb(g.deep_list.count);
        if (g.deep_list.count) {
            RR_CUDA(cudaMemcpyAsync(ha.data(), g.deep_list.a3.p, ha.size() * 4, cudaMemcpyDeviceToHost, st));
            RR_CUDA(cudaMemcpyAsync(hb.data(), g.deep_list.b3.p, hb.size() * 4, cudaMemcpyDeviceToHost, st));
        }
        RR_CUDA(cudaStreamSynchronize(st));
        uint64_t cnt = 0;
        for (size_t i = 0; i < ha.size(); ++i) cnt += ha[i] != hb[i];
        g.deep_compute_rows = cnt;
    }
    // scheduling ranges of every list
    RowList *LL[6] = {&g.prod_list, &g.state_list, &g.win_list, &g.tail_list, &g.deep_list,
                      &g.tail3_list};
    for (int i = 0; i < 6; ++i) {
        RowList &R = *LL[i];
        std::vector<uint32_t> heads(R.count);
        if (R.count)
            RR_CUDA(cudaMemcpyAsync(heads.data(), R.head.p, R.count * 4, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        // fine ranges: enough warps for about 32 per SM even with one point
        // group -- about what the layer kernels keep resident, so that one
        // wave covers a small list (under programmatic dependent launch a
        // kernel's successor can start only once its last wave runs); coarse
        // ranges for the persistent batch, whose parallelism comes from many
        // queries at once
        const uint32_t target =
            (uint32_t)std::min<uint64_t>(128, std::max<uint64_t>(1, R.count / (152 * 32)));
        // runs longer than kMaxRun are cut at the same places in both range
        // sets, so one chain table serves both
        std::vector<uint2> items, coarse, chains;
        build_entry_items(heads, std::min<uint32_t>(target, RowList::kMaxRun), items, &chains);
        build_entry_items(heads, 32, coarse, nullptr);
        R.nchains = (uint32_t)chains.size();
        RR_CUDA(R.chains.reserve(std::max<size_t>(1, chains.size()) * sizeof(uint2)));
        if (!chains.empty())
            RR_CUDA(cudaMemcpyAsync(R.chains.p, chains.data(), chains.size() * sizeof(uint2),
                                    cudaMemcpyHostToDevice, st));
        std::vector<uint2> fix2;
        for (size_t c = 0; c < chains.size(); ++c) {
            const uint32_t R_ = RowList::kMaxRun;
            const uint32_t len = chains[c].y - chains[c].x;
            const uint32_t slots = ((len + R_ - 1) / R_ - 1) * (R_ - 1);
            for (uint32_t s0 = 0; s0 < slots; s0 += 64) fix2.push_back(make_uint2((uint32_t)c, s0));
        }
        R.nfix2 = (uint32_t)fix2.size();
        RR_CUDA(R.fix2.reserve(std::max<size_t>(1, fix2.size()) * sizeof(uint2)));
        if (!fix2.empty())
            RR_CUDA(cudaMemcpyAsync(R.fix2.p, fix2.data(), fix2.size() * sizeof(uint2),
                                    cudaMemcpyHostToDevice, st));
        if (&R == &g.deep_list) {
            // carry slots of the pieces after the first of every cut segment
            std::vector<uint32_t> row_carry(R.count + 1, 0u), slot0(std::max<size_t>(1, chains.size()), 0u);
            uint32_t next = 1;  // slot 0: the zero row
            for (size_t c = 0; c < chains.size(); ++c) {
                const uint32_t R_ = RowList::kMaxRun;
                slot0[c] = next;
                for (uint32_t b = chains[c].x + R_, piece = 0; b < chains[c].y; b += R_, ++piece) {
                    const uint32_t e = std::min(chains[c].y, b + R_);
                    for (uint32_t ent = b; ent < e; ++ent) row_carry[ent + 1] = next + piece;
                }
                next += (chains[c].y - chains[c].x + R_ - 1) / R_ - 1;
            }
            R.ncarry = next;
            RR_CUDA(R.row_carry.reserve(row_carry.size() * 4));
            RR_CUDA(cudaMemcpyAsync(R.row_carry.p, row_carry.data(), row_carry.size() * 4,
                                    cudaMemcpyHostToDevice, st));
            RR_CUDA(R.chain_slot0.reserve(slot0.size() * 4));
            RR_CUDA(cudaMemcpyAsync(R.chain_slot0.p, slot0.data(), slot0.size() * 4,
                                    cudaMemcpyHostToDevice, st));
            RR_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
        }
        R.nitems = (uint32_t)items.size();
        R.nitems_coarse = (uint32_t)coarse.size();
        if (&R == &g.deep_list) {
            // head runs over the fine ranges (the per-point layer 3 forms
            // x_v x_s once per run)
            uint64_t runs = 0;
            for (const uint2 &it : items)
                for (uint32_t r = it.x; r < it.y; ++r) runs += r == it.x || heads[r] != heads[r - 1];
            g.deep_head_runs = runs;
            uint32_t longest = 0;
            for (const uint2 &it : items) longest = std::max(longest, it.y - it.x);
            g.deep_max_item = longest;
            // distinct heads (rows are grouped by head, heads ascending) and the
            // rank among them of every entry's tail
            std::vector<uint32_t> dh;
            for (size_t r = 0; r < heads.size(); ++r)
                if (r == 0 || heads[r] != heads[r - 1]) dh.push_back(heads[r]);
            std::vector<uint32_t> tails(R.count), trank(R.count);
            if (R.count)
                RR_CUDA(cudaMemcpyAsync(tails.data(), R.src.p, R.count * 4, cudaMemcpyDeviceToHost, st));
            RR_CUDA(cudaStreamSynchronize(st));
            for (size_t r = 0; r < tails.size(); ++r) {
                auto f = std::lower_bound(dh.begin(), dh.end(), tails[r]);
                trank[r] = (f != dh.end() && *f == tails[r]) ? (uint32_t)(f - dh.begin()) : UINT32_MAX;
            }
            R.nheads = (uint32_t)dh.size();
            RR_CUDA(R.heads.reserve(std::max<size_t>(1, dh.size()) * 4));
            RR_CUDA(R.trank.reserve(std::max<size_t>(1, trank.size()) * 4));
            if (!dh.empty())
                RR_CUDA(cudaMemcpyAsync(R.heads.p, dh.data(), dh.size() * 4, cudaMemcpyHostToDevice, st));
            if (!trank.empty())
                RR_CUDA(cudaMemcpyAsync(R.trank.p, trank.data(), trank.size() * 4, cudaMemcpyHostToDevice, st));
        }
        RR_CUDA(R.items.reserve(std::max<size_t>(1, items.size()) * sizeof(uint2)));
        RR_CUDA(R.items_coarse.reserve(std::max<size_t>(1, coarse.size()) * sizeof(uint2)));
        if (!items.empty())
            RR_CUDA(cudaMemcpyAsync(R.items.p, items.data(), items.size() * sizeof(uint2),
                                    cudaMemcpyHostToDevice, st));
        if (!coarse.empty())
            RR_CUDA(cudaMemcpyAsync(R.items_coarse.p, coarse.data(), coarse.size() * sizeof(uint2),
                                    cudaMemcpyHostToDevice, st));
        RR_CUDA(cudaStreamSynchronize(st));
    }
    return RR_OK;
}

rr_status graph_load(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                     const uint32_t *t, const uint32_t *delta, const uint8_t *color,
                     uint32_t flags, rr_graph **out)
{
    if (!out) return fail(RR_EINVAL, "rr_graph_load: out is NULL");
    *out = nullptr;
    if (n == 0) return fail(RR_EINVAL, "rr_graph_load: n must be >= 1");
    if (m >= (1ull << 31)) return fail(RR_EINVAL, "rr_graph_load: m must be < 2^31");
    if (m && (!src || !dst || !t)) return fail(RR_EINVAL, "rr_graph_load: NULL edge array");
    if (!delta) return fail(RR_EINVAL, "rr_graph_load: NULL delta");
    for (uint64_t e = 0; e < m; ++e) {
        if (src[e] >= n || dst[e] >= n)
            return fail(RR_EINVAL, "rr_graph_load: endpoint >= n at edge " + std::to_string(e));
        if (src[e] == dst[e])
            return fail(RR_EINVAL, "rr_graph_load: self-loop at edge " + std::to_string(e));
    }

    rr_graph *g = new rr_graph();
    std::unique_ptr<rr_graph> guard(g);
    RR_CUDA(cudaGetDevice(&g->dev));
    g->n = n;
    g->m = m;
    g->has_colors = color != nullptr;
    g->compact = !(flags & 1u);
    if ((flags & 6u) == 6u) return fail(RR_EINVAL, "rr_graph_load: flags turn the pair-label layer 3 both on and off");
    g->pair_force = (flags & 2u) ? 2u : ((flags & 4u) ? 1u : 0u);
    if ((flags & 24u) == 24u) return fail(RR_EINVAL, "rr_graph_load: flags turn the head-factor table both on and off");
    g->head_table_force = (flags & 8u) ? 2u : ((flags & 16u) ? 1u : 0u);
    g->pair_tail_off = (flags & 32u) != 0;
    g->k4_per_point = (flags & 256u) != 0;
    g->k5_closed = (flags & 512u) != 0;
    if ((flags & 192u) == 192u) return fail(RR_EINVAL, "rr_graph_load: flags turn the at-most-k branches both on and off");
    g->atmost_branches = (flags & 128u) ? 2u : ((flags & 64u) ? 1u : 0u);
    RR_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    cudaStream_t st = g->stream;

    RR_CUDA(g->off.reserve((size_t)(n + 1) * 4));
    if (color) {
        RR_CUDA(g->color.reserve(n));
        RR_CUDA(cudaMemcpyAsync(g->color.p, color, n, cudaMemcpyHostToDevice, st));
        // counting sort of the vertices by colour
        std::vector<uint32_t> start(257, 0), order(n);
        for (uint32_t v = 0; v < n; ++v) ++start[color[v] + 1u];
        for (int c = 0; c < 256; ++c) start[c + 1] += start[c];
        for (uint32_t v = 0; v < n; ++v) order[start[color[v]]++] = v;
        RR_CUDA(g->color_order.reserve((size_t)n * 4));
        RR_CUDA(cudaMemcpy(g->color_order.p, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    }
    const size_t mb = (size_t)(m ? m : 1);
    for (DevBuf *b : {&g->row_a, &g->row_b, &g->row_s, &g->row_eid, &g->row_src, &g->row_lo,
                      &g->row_hi})
        RR_CUDA(b->reserve(mb * 4));

    DevBuf d_delta;
    RR_CUDA(d_delta.reserve((size_t)n * 4));
    RR_CUDA(cudaMemcpyAsync(d_delta.p, delta, (size_t)n * 4, cudaMemcpyHostToDevice, st));

    if (m == 0) {
        RR_CUDA(cudaMemsetAsync(g->off.p, 0, (size_t)(n + 1) * 4, st));
    } else {
        DevBuf d_src, d_dst, d_t, key_in, key_out, val_in, tmp;
        RR_CUDA(d_src.reserve(mb * 4));
        RR_CUDA(d_dst.reserve(mb * 4));
        RR_CUDA(d_t.reserve(mb * 4));
        RR_CUDA(cudaMemcpyAsync(d_src.p, src, m * 4, cudaMemcpyHostToDevice, st));
        RR_CUDA(cudaMemcpyAsync(d_dst.p, dst, m * 4, cudaMemcpyHostToDevice, st));
        RR_CUDA(cudaMemcpyAsync(d_t.p, t, m * 4, cudaMemcpyHostToDevice, st));
        RR_CUDA(key_in.reserve(mb * 8));
        RR_CUDA(key_out.reserve(mb * 8));
        RR_CUDA(val_in.reserve(mb * 4));
        k_make_keys<<<grid_for(m, 256), 256, 0, st>>>(d_dst.as<uint32_t>(), d_t.as<uint32_t>(), m,
                                                      key_in.as<uint64_t>(), val_in.as<uint32_t>());
        RR_LAUNCHED();
        int head_bits = 0;
        while (head_bits < 32 && ((uint64_t)(n - 1) >> head_bits)) ++head_bits;
        size_t tmp_bytes = 0;
        RR_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key_in.as<uint64_t>(),
                                                key_out.as<uint64_t>(), val_in.as<uint32_t>(),
                                                g->row_eid.as<uint32_t>(), (int64_t)m, 0,
                                                32 + head_bits, st));
        RR_CUDA(tmp.reserve(tmp_bytes));
        RR_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, key_in.as<uint64_t>(),
                                                key_out.as<uint64_t>(), val_in.as<uint32_t>(),
                                                g->row_eid.as<uint32_t>(), (int64_t)m, 0,
                                                32 + head_bits, st));
        key_in.release();
        val_in.release();
        d_dst.release();
        d_t.release();
        RR_CUDA(g->row_t.reserve(mb * 4));
        RR_CUDA(g->row_head.reserve(mb * 4));
        k_unpack_rows<<<grid_for(m, 256), 256, 0, st>>>(
            key_out.as<uint64_t>(), g->row_eid.as<uint32_t>(), d_src.as<uint32_t>(), m,
            g->row_t.as<uint32_t>(), g->row_head.as<uint32_t>(), g->row_src.as<uint32_t>());
        RR_LAUNCHED();
        key_out.release();
        d_src.release();
        k_offsets<<<grid_for(m + 1, 256), 256, 0, st>>>(g->row_head.as<uint32_t>(), m, n,
                                                        g->off.as<uint32_t>());
        RR_LAUNCHED();

        DevBuf diff, cover, prod, tprod, rank, counter;
        RR_CUDA(counter.reserve(16));
        RR_CUDA(cudaMemsetAsync(counter.p, 0, 16, st));
        RR_CUDA(diff.reserve((mb + 1) * 4));
        RR_CUDA(cudaMemsetAsync(diff.p, 0, (mb + 1) * 4, st));
        k_windows<<<grid_for(m, 256), 256, 0, st>>>(
            g->row_t.as<uint32_t>(), g->row_src.as<uint32_t>(), g->off.as<uint32_t>(),
            d_delta.as<uint32_t>(), m, g->row_lo.as<uint32_t>(), g->row_hi.as<uint32_t>(),
            diff.as<int32_t>(), counter.as<unsigned long long>());
        RR_LAUNCHED();
        RR_CUDA(prod.reserve(mb * 4));
        RR_CUDA(tprod.reserve(mb * 4));
        RR_CUDA(cover.reserve(mb * 4));
        tmp_bytes = 0;
        RR_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, diff.as<int32_t>(),
                                              cover.as<int32_t>(), (int64_t)m, st));
        RR_CUDA(tmp.reserve(tmp_bytes));
        RR_CUDA(cub::DeviceScan::InclusiveSum(tmp.p, tmp_bytes, diff.as<int32_t>(),
                                              cover.as<int32_t>(), (int64_t)m, st));
        k_cover_to_flags<<<grid_for(m, 256), 256, 0, st>>>(cover.as<int32_t>(), m,
                                                           tprod.as<uint32_t>());
        RR_LAUNCHED();
        if (g->compact) {
            RR_CUDA(cudaMemcpyAsync(prod.p, tprod.p, m * 4, cudaMemcpyDeviceToDevice, st));
        } else {
            k_dense_flags<<<grid_for(m, 256), 256, 0, st>>>(m, prod.as<uint32_t>());
            RR_LAUNCHED();
        }
        RR_CUDA(rank.reserve(mb * 4));
        tmp_bytes = 0;
        RR_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, prod.as<uint32_t>(),
                                              rank.as<uint32_t>(), (int64_t)m, st));
        RR_CUDA(tmp.reserve(tmp_bytes));
        RR_CUDA(cub::DeviceScan::InclusiveSum(tmp.p, tmp_bytes, prod.as<uint32_t>(),
                                              rank.as<uint32_t>(), (int64_t)m, st));
        k_state_index<<<grid_for(m, 256), 256, 0, st>>>(
            rank.as<uint32_t>(), prod.as<uint32_t>(), g->row_lo.as<uint32_t>(),
            g->row_hi.as<uint32_t>(), g->row_src.as<uint32_t>(), g->off.as<uint32_t>(), m,
            g->row_a.as<uint32_t>(), g->row_b.as<uint32_t>(), g->row_s.as<uint32_t>(),
            counter.as<unsigned long long>() + 1);
        RR_LAUNCHED();
        uint32_t last_rank = 0;
        unsigned long long nonempty = 0, prod_window = 0;
        RR_CUDA(cudaMemcpyAsync(&last_rank, rank.as<uint32_t>() + (m - 1), 4,
                                cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaMemcpyAsync(&nonempty, counter.p, 8, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaMemcpyAsync(&prod_window, counter.as<unsigned long long>() + 1, 8,
                                cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        g->state_rows = 1ull + last_rank;
        g->window_rows = nonempty;
        g->producer_window_rows = prod_window;
        rr_status ls = build_lists_v2(*g, g->row_head.as<uint32_t>(), tprod.as<uint32_t>(), st);
        if (ls != RR_OK) return ls;
    }

    std::vector<uint32_t> h_off(n + 1);
    RR_CUDA(cudaMemcpyAsync(h_off.data(), g->off.p, (size_t)(n + 1) * 4, cudaMemcpyDeviceToHost,
                            st));
    RR_CUDA(cudaStreamSynchronize(st));
    std::vector<uint32_t> v0, v1, rows;
    build_items(h_off, n, v0, v1, rows, &g->max_in_degree);
    std::vector<uint32_t> order(v0.size());
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return rows[a] > rows[b]; });
    std::vector<uint2> items(order.size());
    g->h_item_rows.resize(order.size());
    for (size_t i = 0; i < order.size(); ++i) {
        items[i] = make_uint2(v0[order[i]], v1[order[i]]);
        g->h_item_rows[i] = rows[order[i]];
    }
    g->nitems = (uint32_t)items.size();
    RR_CUDA(g->items.reserve(std::max<size_t>(1, items.size()) * sizeof(uint2)));
    if (!items.empty())
        RR_CUDA(cudaMemcpyAsync(g->items.p, items.data(), items.size() * sizeof(uint2),
                                cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaStreamSynchronize(st));
    *out = guard.release();
    return RR_OK;
}

}  // namespace rr
