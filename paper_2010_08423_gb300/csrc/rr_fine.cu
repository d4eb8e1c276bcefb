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

// One extraction step (Sec. "Extracting an optimal solution using k queries").
// Among the rows r of `cur`'s segment with time tc whose tail u is not
// deleted, find the earliest time i inside r's restless window at which u's
// (u, i) polynomial -- the XOR of E over u's rows at time i -- is non-zero;
// best = min over such rows of (i << 32 | r). Rows of one (head, time) run are
// in input-edge order, so the smallest r is the smallest edge index. With
// `first` set, the candidates are instead the rows from `source` (the path's
// first edge) and best = min r.
__global__ void k_extract_step(uint32_t cur, uint32_t tc, const uint32_t *__restrict__ off,
                               const uint32_t *__restrict__ row_t, const uint32_t *__restrict__ row_src,
                               const uint32_t *__restrict__ row_lo, const uint32_t *__restrict__ row_hi,
                               const uint32_t *__restrict__ row_eid, const uint64_t *__restrict__ E,
                               const uint8_t *__restrict__ vmask, uint32_t source, int first,
                               unsigned long long *best)
{
    const uint32_t r0 = off[cur], r1 = off[cur + 1];
    for (uint32_t r = r0 + blockIdx.x * blockDim.x + threadIdx.x; r < r1; r += gridDim.x * blockDim.x) {
        if (row_t[r] != tc) continue;
        const uint32_t u = row_src[r];
        if (first) {
            if (u == source) atomicMin(best, (unsigned long long)r);
            continue;
        }
        if (vmask[u]) continue;
        uint32_t f = row_lo[r];
        const uint32_t hi = row_hi[r];
        while (f < hi) {  // the window's rows, one time group at a time
            const uint32_t t = row_t[f];
            uint64_t x = 0;
            for (; f < hi && row_t[f] == t; ++f) x ^= E[row_eid[f]];
            if (x) {
                atomicMin(best, ((unsigned long long)t << 32) | r);
                break;
            }
        }
    }
}

unsigned grid_for(uint64_t count, unsigned block)
{
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(152ull * 32, (count + block - 1) / block));
}

}  // namespace

// Folds one k' into the bounded-reach outputs (callers go through k' in
// increasing order): R = min(R, R_k'), L = k' where L is still 0 and k'
// reaches the vertex.
__global__ void k_merge_arrival(uint32_t n, const uint32_t *__restrict__ Rk, uint32_t kk,
                                uint32_t *__restrict__ R, uint8_t *__restrict__ L)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t r = Rk[v];
        if (r == 0xFFFFFFFFu) continue;
        if (r < R[v]) R[v] = r;
        if (L && L[v] == 0) L[v] = (uint8_t)kk;
    }
}

rr_status arrival_device(const Graph &g, const rr_query *q, uint64_t *d_witness, uint64_t *d_E,
                         uint32_t *d_R, uint8_t *d_bitmap, cudaStream_t st, const uint8_t *d_vmask)
{
    return arrival_on(g, g.ws, q, d_witness, d_E, d_R, d_bitmap, st, d_vmask, 0);
}

rr_status arrival_on(const Graph &g, Workspace &ws, const rr_query *q, uint64_t *d_witness,
                     uint64_t *d_E, uint32_t *d_R, uint8_t *d_bitmap, cudaStream_t st,
                     const uint8_t *d_vmask, uint64_t budget, uint32_t bfirst)
{
    if (!d_E) {
        RR_CUDA(ws.edges.reserve((size_t)std::max<uint64_t>(1, g.m) * 8));
        d_E = ws.edges.as<uint64_t>();
    }
    const uint32_t nb = bfirst ? q->k - bfirst : 0;  // at-most-k branches k' = bfirst..k-1
    const size_t mw = (size_t)std::max<uint64_t>(1, g.m);
    if (nb) {
        RR_CUDA(ws.bS.reserve((size_t)nb * g.n * 8));
        RR_CUDA(ws.bE.reserve((size_t)nb * mw * 8));
        RR_CUDA(ws.bR.reserve((size_t)nb * g.n * 4));
        RR_CUDA(cudaMemsetAsync(ws.bS.p, 0, (size_t)nb * g.n * 8, st));
        RR_CUDA(cudaMemsetAsync(ws.bE.p, 0, (size_t)nb * mw * 8, st));
        RR_CUDA(cudaMemsetAsync(ws.bR.p, 0xFF, (size_t)nb * g.n * 4, st));
    }
    if (g.m) RR_CUDA(cudaMemsetAsync(d_E, 0, (size_t)g.m * 8, st));
    RR_CUDA(cudaMemsetAsync(d_R, 0xFF, (size_t)g.n * 4, st));
    rr_status s = reach_on_stream(g, ws, q, nullptr, d_witness, budget, st, d_E, d_vmask, nullptr,
                                  PointRange(), bfirst, nb ? ws.bS.as<uint64_t>() : nullptr,
                                  nb ? ws.bE.as<uint64_t>() : nullptr);
    if (s != RR_OK) return s;
    for (uint32_t b = 0; g.m && b <= nb; ++b) {  // the query's own arrivals, then each branch's
        const uint64_t *E = b == 0 ? d_E : ws.bE.as<uint64_t>() + (size_t)(b - 1) * mw;
        uint32_t *R = b == 0 ? d_R : ws.bR.as<uint32_t>() + (size_t)(b - 1) * g.n;
        k_arrival<<<grid_for(g.m, 256), 256, 0, st>>>((uint32_t)g.m, g.row_head.as<uint32_t>(),
                                                       g.row_t.as<uint32_t>(), g.row_eid.as<uint32_t>(),
                                                       E, R);
        RR_LAUNCHED();
    }
    if (d_bitmap) {
        k_arrival_bitmap<<<grid_for((g.n + 7) / 8, 256), 256, 0, st>>>(g.n, d_R, d_bitmap);
        RR_LAUNCHED();
    }
    return RR_OK;
}

// One optimal restless path (Sec. "Extracting an optimal solution using k
// queries"): the fine-grained query for k vertices gives the target's minimum
// arrival time; each further query, for one vertex fewer on the graph without
// the chosen vertices (and, for motif queries, without their colours in M),
// certifies the next vertex back. Synchronous on the graph's stream.
rr_status extract_path(const Graph &g, const rr_query *q, uint32_t target, uint32_t *vertices,
                       uint32_t *edges, uint32_t *times)
{
    const uint32_t k = q->k;
    cudaStream_t st = g.stream;
    Workspace &ws = g.ws;
    RR_CUDA(ws.S.reserve((size_t)g.n * 8));
    RR_CUDA(ws.arrival.reserve((size_t)g.n * 4));
    RR_CUDA(ws.vmask.reserve(g.n));
    RR_CUDA(ws.pick.reserve(8));
    RR_CUDA(ws.edges.reserve((size_t)std::max<uint64_t>(1, g.m) * 8));
    uint8_t *vm = ws.vmask.as<uint8_t>();
    RR_CUDA(cudaMemsetAsync(vm, 0, g.n, st));
    std::vector<uint8_t> M;
    if (q->motif) M.assign(q->motif, q->motif + k);
    auto drop_colour = [&](uint32_t v) -> rr_status {
        if (!q->motif) return RR_OK;
        uint8_t c = 0;
        RR_CUDA(cudaMemcpyAsync(&c, g.color.as<uint8_t>() + v, 1, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        auto it = std::find(M.begin(), M.end(), c);
        if (it == M.end()) return fail(RR_ECUDA, "rr_extract_path: chosen vertex colour not in M");
        M.erase(it);
        return RR_OK;
    };
    auto run = [&](uint32_t kk, const uint8_t *mask) -> rr_status {
        rr_query qq{q->source, kk, q->seed, q->motif ? M.data() : nullptr};
        return arrival_device(g, &qq, ws.S.as<uint64_t>(), ws.edges.as<uint64_t>(),
                              ws.arrival.as<uint32_t>(), nullptr, st, mask);
    };
    auto pick = [&](uint32_t cur, uint32_t tc, int first, uint64_t *out) -> rr_status {
        RR_CUDA(cudaMemsetAsync(ws.pick.p, 0xFF, 8, st));
        k_extract_step<<<152, 256, 0, st>>>(cur, tc, g.off.as<uint32_t>(), g.row_t.as<uint32_t>(),
                                            g.row_src.as<uint32_t>(), g.row_lo.as<uint32_t>(),
                                            g.row_hi.as<uint32_t>(), g.row_eid.as<uint32_t>(),
                                            ws.edges.as<uint64_t>(), vm, q->source, first,
                                            ws.pick.as<unsigned long long>());
        RR_LAUNCHED();
        RR_CUDA(cudaMemcpyAsync(out, ws.pick.p, 8, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        return RR_OK;
    };
    auto row_field = [&](const DevBuf &b, uint32_t r, uint32_t *out) -> rr_status {
        RR_CUDA(cudaMemcpyAsync(out, b.as<uint32_t>() + r, 4, cudaMemcpyDeviceToHost, st));
        RR_CUDA(cudaStreamSynchronize(st));
        return RR_OK;
    };

    // the target's minimum arrival time
    rr_status s = run(k, nullptr);
    if (s != RR_OK) return s;
    uint32_t tc = 0;
    RR_CUDA(cudaMemcpyAsync(&tc, ws.arrival.as<uint32_t>() + target, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (tc == 0xFFFFFFFFu) return fail(RR_ENOPATH, "rr_extract_path: the target has no arrival");
    uint32_t cur = target;
    vertices[k - 1] = target;
    times[k - 2] = tc;
    for (uint32_t ell = k - 1; ell >= 2; --ell) {
        RR_CUDA(cudaMemsetAsync(vm + cur, 1, 1, st));  // delete the vertex chosen last
        if ((s = drop_colour(cur)) != RR_OK) return s;
        if ((s = run(ell, vm)) != RR_OK) return s;
        uint64_t best = 0;
        if ((s = pick(cur, tc, 0, &best)) != RR_OK) return s;
        if (best == ~0ull)
            return fail(RR_ENOPATH, "rr_extract_path: a step's polynomials vanished (probability <= (3k-1)/2^64)");
        const uint32_t r = (uint32_t)best, i = (uint32_t)(best >> 32);
        uint32_t u = 0, e = 0;
        if ((s = row_field(g.row_src, r, &u)) != RR_OK) return s;
        if ((s = row_field(g.row_eid, r, &e)) != RR_OK) return s;
        vertices[ell - 1] = u;
        edges[ell - 1] = e;
        times[ell - 2] = i;
        cur = u;
        tc = i;
    }
    // the first edge: from the source into vertices[1] at its chosen time
    uint64_t best = 0;
    if ((s = pick(cur, tc, 1, &best)) != RR_OK) return s;
    if (best == ~0ull) return fail(RR_ECUDA, "rr_extract_path: no source edge at the chosen time");
    uint32_t e0 = 0;
    if ((s = row_field(g.row_eid, (uint32_t)best, &e0)) != RR_OK) return s;
    vertices[0] = q->source;
    edges[0] = e0;
    return RR_OK;
}

// k-RestlessReach from a set of sources, optionally avoiding separators (Sec.
// "Discussion": the multi-source variant; the case study's separators). Walks
// start at every edge leaving a source; the sums are the XOR of the
// single-source sums. One source runs the reduced-state engine, a larger set
// the per-point engine with a source mask.
rr_status sources_device(const Graph &g, const uint32_t *sources, uint32_t nsources, uint32_t k,
                         uint64_t seed, const uint8_t *motif, const uint8_t *d_separators,
                         uint8_t *d_bitmap, uint64_t *d_witness, cudaStream_t st)
{
    const rr_query q{sources[0], k, seed, motif};
    if (nsources == 1)
        return reach_on_stream(g, g.ws, &q, d_bitmap, d_witness, 0, st, nullptr, d_separators);
    std::vector<uint8_t> flags(g.n, 0);
    for (uint32_t i = 0; i < nsources; ++i) flags[sources[i]] = 1;
    Workspace &ws = g.ws;
    RR_CUDA(ws.srcmask.reserve(g.n));
    // pageable source: the copy is staged before the call returns
    RR_CUDA(cudaMemcpyAsync(ws.srcmask.p, flags.data(), g.n, cudaMemcpyHostToDevice, st));
    return reach_on_stream(g, ws, &q, d_bitmap, d_witness, 0, st, nullptr, d_separators,
                           ws.srcmask.as<uint8_t>());
}

// Bounded RestlessReach (Algorithm 2 with its loop over k' stopped at k):
// the fine-grained query for every k' = 2..k, concurrently on the graph's
// lanes (largest k' first) when their scratch fits 60% of free device memory
// together, else one after another on the graph's workspace; then R = the
// minimum arrival over k', L = the smallest k' reaching each vertex, and the
// bitmap of D = {v : R_v defined}.
rr_status atmost_arrival_device(const Graph &g, uint32_t source, uint32_t k, uint64_t seed,
                                uint32_t *d_R, uint8_t *d_L, uint8_t *d_bitmap, cudaStream_t st)
{
    const uint32_t lanes = k - 1;
    const size_t mb = (size_t)std::max<uint64_t>(1, g.m) * 8;
    size_t free_b = 0, total_b = 0;
    RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t per_lane = (uint64_t)(0.6 * (double)(free_b + g.fan.bytes())) / lanes;
    const uint64_t extra = mb + (uint64_t)g.n * 12;  // per-edge sums, arrival, witness
    uint64_t need = 0;
    for (uint32_t kk = 2; kk <= k; ++kk) {
        const uint64_t b = per_lane > extra ? query_scratch_bytes(g, kk, per_lane - extra) : UINT64_MAX;
        need = (b == UINT64_MAX || need == UINT64_MAX) ? UINT64_MAX : need + b + extra;
    }
    RR_CUDA(cudaMemsetAsync(d_R, 0xFF, (size_t)g.n * 4, st));
    if (d_L) RR_CUDA(cudaMemsetAsync(d_L, 0, g.n, st));
    const unsigned grid = grid_for(g.n, 256);
    if (need == UINT64_MAX) {
        Workspace &ws = g.ws;
        RR_CUDA(ws.S.reserve((size_t)g.n * 8));
        RR_CUDA(ws.arrival.reserve((size_t)g.n * 4));
        RR_CUDA(ws.edges.reserve(mb));
        for (uint32_t kk = 2; kk <= k; ++kk) {
            const rr_query q{source, kk, seed, nullptr};
            rr_status s = arrival_on(g, ws, &q, ws.S.as<uint64_t>(), ws.edges.as<uint64_t>(),
                                     ws.arrival.as<uint32_t>(), nullptr, st, nullptr, 0);
            if (s != RR_OK) return s;
            k_merge_arrival<<<grid, 256, 0, st>>>(g.n, ws.arrival.as<uint32_t>(), kk, d_R, d_L);
            RR_LAUNCHED();
        }
    } else {
        rr_status s = ensure_fan_lanes(g, lanes);
        if (s != RR_OK) return s;
        FanOut &F = g.fan;
        // k' = bfirst..k-1 come from the k query's own layers (lane 0)
        const uint32_t bfirst = atmost_branches(g, k);
        RR_CUDA(cudaEventRecord(F.fork, st));
        for (uint32_t kk = k; kk >= 2; --kk) {
            if (bfirst && kk >= bfirst && kk < k) continue;
            const uint32_t j = k - kk;  // lane
            Workspace &ws = *F.ws[j];
            RR_CUDA(ws.S.reserve((size_t)g.n * 8));
            RR_CUDA(ws.arrival.reserve((size_t)g.n * 4));
            RR_CUDA(ws.edges.reserve(mb));
            const rr_query q{source, kk, seed, nullptr};
            RR_CUDA(cudaStreamWaitEvent(F.st[j], F.fork, 0));
            s = arrival_on(g, ws, &q, ws.S.as<uint64_t>(), ws.edges.as<uint64_t>(),
                           ws.arrival.as<uint32_t>(), nullptr, F.st[j], nullptr, per_lane - extra,
                           kk == k ? bfirst : 0u);
            RR_CUDA(cudaEventRecord(F.done[j], F.st[j]));
            RR_CUDA(cudaStreamWaitEvent(st, F.done[j], 0));
            if (s != RR_OK) return s;
        }
        for (uint32_t kk = 2; kk <= k; ++kk) {
            const uint32_t *R = bfirst && kk >= bfirst && kk < k
                                    ? F.ws[0]->bR.as<uint32_t>() + (size_t)(kk - bfirst) * g.n
                                    : F.ws[k - kk]->arrival.as<uint32_t>();
            k_merge_arrival<<<grid, 256, 0, st>>>(g.n, R, kk, d_R, d_L);
            RR_LAUNCHED();
        }
    }
    if (d_bitmap) {
        k_arrival_bitmap<<<grid_for((g.n + 7) / 8, 256), 256, 0, st>>>(g.n, d_R, d_bitmap);
        RR_LAUNCHED();
    }
    return RR_OK;
}

}  // namespace rr
