// rr_fine.cu -- the fine-grained oracle's per-time outputs (Algorithm 1; Sec.
// "A fine-grained decision oracle").
//
// Algorithm 1 keeps one polynomial per (vertex u, time i): the walks of k
// vertices that end at u with a last edge at time i. In the edge-layer form
// that polynomial is the XOR, over the edges e into u with t_e = i, of E[e] =
// the sum over all sieve points of e's last-layer value. The query kernels
// write E when the query descriptor asks for it; here the in-edge rows of
// every vertex, sorted by time, are cut into runs of equal time, each run's E
// values are XOR-ed, and R_u is the smallest time of a run with a non-zero
// sum (UINT32_MAX when there is none). D = {u : R_u < UINT32_MAX}.
#include <algorithm>

#include "rr_internal.h"

namespace rr {

namespace {

// One thread per CSR row; the first row of every (head, time) run sums the
// run and lowers R of its head if the sum is non-zero. Rows are sorted by
// (head, time, edge), so a run is a contiguous range.
__global__ void k_arrival(uint32_t m, const uint32_t *__restrict__ row_head,
                          const uint32_t *__restrict__ row_t, const uint32_t *__restrict__ row_eid,
                          const uint64_t *__restrict__ E, uint32_t *__restrict__ R)
{
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const uint32_t v = row_head[r], t = row_t[r];
        if (r > 0 && row_head[r - 1] == v && row_t[r - 1] == t) continue;  // not a run start
        uint64_t sum = 0;
        for (uint32_t q = r; q < m && row_head[q] == v && row_t[q] == t; ++q) sum ^= E[row_eid[q]];
        if (sum) atomicMin(R + v, t);
    }
}

__global__ void k_arrival_bitmap(uint32_t n, const uint32_t *__restrict__ R, uint8_t *__restrict__ bm)
{
    const uint32_t nb = (n + 7) / 8;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t i = 0; i < 8; ++i) {
            const uint32_t v = b * 8 + i;
            if (v < n && R[v] != 0xFFFFFFFFu) bits |= 1u << i;
        }
        bm[b] = (uint8_t)bits;
    }
}

unsigned grid_for(uint64_t count, unsigned block)
{
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(152ull * 32, (count + block - 1) / block));
}

}  // namespace

rr_status arrival_device(const Graph &g, const rr_query *q, uint64_t *d_witness, uint64_t *d_E,
                         uint32_t *d_R, uint8_t *d_bitmap, cudaStream_t st)
{
    Workspace &ws = g.ws;
    if (!d_E) {
        RR_CUDA(ws.edges.reserve((size_t)std::max<uint64_t>(1, g.m) * 8));
        d_E = ws.edges.as<uint64_t>();
    }
    if (g.m) RR_CUDA(cudaMemsetAsync(d_E, 0, (size_t)g.m * 8, st));
    RR_CUDA(cudaMemsetAsync(d_R, 0xFF, (size_t)g.n * 4, st));
    rr_status s = reach_on_stream(g, ws, q, nullptr, d_witness, 0, st, d_E);
    if (s != RR_OK) return s;
    if (g.m) {
        k_arrival<<<grid_for(g.m, 256), 256, 0, st>>>((uint32_t)g.m, g.row_head.as<uint32_t>(),
                                                       g.row_t.as<uint32_t>(), g.row_eid.as<uint32_t>(),
                                                       d_E, d_R);
        RR_LAUNCHED();
    }
    if (d_bitmap) {
        k_arrival_bitmap<<<grid_for((g.n + 7) / 8, 256), 256, 0, st>>>(g.n, d_R, d_bitmap);
        RR_LAUNCHED();
    }
    return RR_OK;
}

}  // namespace rr
