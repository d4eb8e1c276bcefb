// rr_batch.cu -- many queries in one call, and the shape autotuner.
#include <algorithm>
#include <cstring>

#include "rr_internal.h"

namespace rr {

rr_status batch_device(const Graph &g, const rr_query *qs, uint32_t nq, uint8_t *d_bitmaps,
                       uint64_t *d_witness, int32_t *d_status, cudaStream_t st)
{
    const size_t nb = (g.n + 7) / 8;
    for (uint32_t i = 0; i < nq; ++i) {
        rr_status s = reach_on_stream(g, g.ws, &qs[i], d_bitmaps ? d_bitmaps + i * nb : nullptr,
                                      d_witness + (size_t)i * g.n, 0, st);
        if (s != RR_OK) return s;
    }
    if (d_status && nq) RR_CUDA(cudaMemsetAsync(d_status, 0, (size_t)nq * 4, st));
    return RR_OK;
}

// Times each candidate (points per lane, points per chunk) on a plain query of
// size k from the vertex with the most out-rows and keeps the fastest.
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
    float best = 1e30f;
    Cand win{0, 0};
    const uint32_t save_ppl = g.tune_ppl[k], save_chunk = g.tune_chunk[k];
    for (const Cand &c : cands) {
        g.tune_ppl[k] = c.ppl;
        g.tune_chunk[k] = c.chunk;
        size_t free_b = 0, total_b = 0;
        RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
        uint32_t ppl, chunk;
        if (!choose_shape(g, k, (uint64_t)(0.6 * (double)(free_b + g.ws.state.bytes)), &ppl, &chunk) ||
            chunk != c.chunk)
            continue;
        rr_status s = reach_on_stream(g, g.ws, &q, nullptr, S.as<uint64_t>(), 0, g.stream);  // warm-up
        if (s != RR_OK) break;
        RR_CUDA(cudaEventRecord(e0, g.stream));
        for (int rep = 0; rep < 3 && s == RR_OK; ++rep)
            s = reach_on_stream(g, g.ws, &q, nullptr, S.as<uint64_t>(), 0, g.stream);
        RR_CUDA(cudaEventRecord(e1, g.stream));
        RR_CUDA(cudaEventSynchronize(e1));
        if (s != RR_OK) break;
        float ms = 0;
        RR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (win.ppl == 0) {
        g.tune_ppl[k] = save_ppl;
        g.tune_chunk[k] = save_chunk;
        return fail(RR_ENOMEM, "rr_autotune: no candidate shape fits device memory");
    }
    g.tune_ppl[k] = win.ppl;
    g.tune_chunk[k] = win.chunk;
    if (best_ppl) *best_ppl = win.ppl;
    if (best_chunk) *best_chunk = win.chunk;
    return RR_OK;
}

}  // namespace rr
