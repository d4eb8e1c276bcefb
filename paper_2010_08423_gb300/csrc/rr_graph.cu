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
    RR_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    cudaStream_t st = g->stream;

    RR_CUDA(g->off.reserve((size_t)(n + 1) * 4));
    if (color) {
        RR_CUDA(g->color.reserve(n));
        RR_CUDA(cudaMemcpyAsync(g->color.p, color, n, cudaMemcpyHostToDevice, st));
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
        DevBuf d_src, d_dst, d_t, key_in, key_out, val_in, row_t, row_dst, tmp;
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
        RR_CUDA(row_t.reserve(mb * 4));
        RR_CUDA(row_dst.reserve(mb * 4));
        k_unpack_rows<<<grid_for(m, 256), 256, 0, st>>>(
            key_out.as<uint64_t>(), g->row_eid.as<uint32_t>(), d_src.as<uint32_t>(), m,
            row_t.as<uint32_t>(), row_dst.as<uint32_t>(), g->row_src.as<uint32_t>());
        RR_LAUNCHED();
        key_out.release();
        d_src.release();
        k_offsets<<<grid_for(m + 1, 256), 256, 0, st>>>(row_dst.as<uint32_t>(), m, n,
                                                        g->off.as<uint32_t>());
        RR_LAUNCHED();

        DevBuf diff, cover, prod, rank, counter;
        RR_CUDA(counter.reserve(16));
        RR_CUDA(cudaMemsetAsync(counter.p, 0, 16, st));
        if (g->compact) {
            RR_CUDA(diff.reserve((mb + 1) * 4));
            RR_CUDA(cudaMemsetAsync(diff.p, 0, (mb + 1) * 4, st));
        }
        k_windows<<<grid_for(m, 256), 256, 0, st>>>(
            row_t.as<uint32_t>(), g->row_src.as<uint32_t>(), g->off.as<uint32_t>(),
            d_delta.as<uint32_t>(), m, g->row_lo.as<uint32_t>(), g->row_hi.as<uint32_t>(),
            g->compact ? diff.as<int32_t>() : nullptr,
            counter.as<unsigned long long>());
        RR_LAUNCHED();
        RR_CUDA(prod.reserve(mb * 4));
        if (g->compact) {
            RR_CUDA(cover.reserve(mb * 4));
            tmp_bytes = 0;
            RR_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, diff.as<int32_t>(),
                                                  cover.as<int32_t>(), (int64_t)m, st));
            RR_CUDA(tmp.reserve(tmp_bytes));
            RR_CUDA(cub::DeviceScan::InclusiveSum(tmp.p, tmp_bytes, diff.as<int32_t>(),
                                                  cover.as<int32_t>(), (int64_t)m, st));
            k_cover_to_flags<<<grid_for(m, 256), 256, 0, st>>>(cover.as<int32_t>(), m,
                                                               prod.as<uint32_t>());
        } else {
            k_dense_flags<<<grid_for(m, 256), 256, 0, st>>>(m, prod.as<uint32_t>());
        }
        RR_LAUNCHED();
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
