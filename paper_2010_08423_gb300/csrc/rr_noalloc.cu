// rr_noalloc.cu -- rr_reach_device_noalloc: one query of the sieve whose
// scratch lives in a fixed, statically sized device array instead of memory
// obtained from cudaMalloc.
//
// Who needs this: callers that must not allocate device memory while serving a
// query -- for example a host process whose device memory is already handed
// out to another allocator's pool (so a cudaMalloc here would fail or fight
// that pool), or a latency-sensitive loop where a cudaMalloc/cudaFree would
// synchronise the device and stall the other streams. Such callers load the
// graph once up front and then run queries through this entry point, which
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The scratch is the file-scope array below (kNoAllocScratchBytes = 256 MiB).
// It is resident on every device where this library's device code is loaded,
// for the life of the process: under CUDA's default lazy module loading from
// the first use of this file's device code on that device, under eager loading
// (CUDA_MODULE_LOADING=EAGER) on every device where the process creates a
// context. Device-memory budgets computed from cudaMemGetInfo see it as used.
// The array is shared by every call: a call reuses what the previous call left
// there and clears what must start at zero itself (the zero state row of both
// prefix buffers; the witness output is cleared too), so calls whose work
// overlaps on the GPU -- for instance calls issued on different streams without
// ordering between them -- race on the array and give wrong results. Order such
// calls on one stream.
#include <mutex>

#include "rr_internal.h"

namespace rr {

constexpr size_t kNoAllocScratchBytes = size_t(256) << 20;
constexpr int kNoAllocMaxDevices = 64;

// The array. In host code this name is only a host-side stand-in for the
// symbol: its device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchBytes / 8];

static std::mutex g_noalloc_mu;
static uint64_t *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on device `dev`, looked up once per
// device with that device current.
static rr_status noalloc_scratch(int dev, uint64_t **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(RR_EINVAL, "rr_reach_device_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return RR_OK;
}

// Copies a motif's shade table (a kernel argument, so no host memory is read
// by a copy) into its place in the scratch array.
__global__ void k_put_shades(const ShadeTable sh, uint32_t *__restrict__ dst)
{
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) {
        dst[i] = sh.first[i];
        dst[256 + i] = sh.mu[i];
    }
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_reach_device_noalloc(const rr_graph *g, const rr_query *q,
                                             uint8_t *d_bitmap, uint64_t *d_witness,
                                             void *stream)
{
    clear_error();
    if (!g) return fail(RR_EINVAL, "rr_reach_device_noalloc: NULL graph");
    if (!d_witness) return fail(RR_EINVAL, "rr_reach_device_noalloc: d_witness is required");
    rr_status vs = validate_query(*g, q);
    if (vs != RR_OK) return vs;
    int dev = -1;
    RR_CUDA(cudaGetDevice(&dev));
    if (dev != g->dev)
        return fail(RR_EINVAL, "rr_reach_device_noalloc: call with the graph's device current");
    uint64_t *scratch = nullptr;
    rr_status s = noalloc_scratch(dev, &scratch);
    if (s != RR_OK) return s;

    // Layout of the array: z-table (n*k words), shade table (512 uint32), then
    // the two prefix-state buffers (state_rows * chunk words each).
    const uint32_t k = q->k;
    const size_t z_words = ((size_t)g->n * k + 31) / 32 * 32;
    const size_t shade_words = sizeof(ShadeTable) / 8;
    const size_t fixed_bytes = (z_words + shade_words) * 8;
    if (fixed_bytes >= kNoAllocScratchBytes)
        return fail(RR_ENOMEM, "rr_reach_device_noalloc: the z-table of this query (" +
                                   std::to_string(fixed_bytes) + " bytes) exceeds the " +
                                   std::to_string(kNoAllocScratchBytes) + "-byte static scratch");
    // the graph's tuning for k, read under its lock (rr_autotune and
    // rr_set_tuning change it there)
    uint32_t tune_ppl = 0, tune_chunk = 0;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        tune_ppl = g->tune_ppl[k];
        tune_chunk = g->tune_chunk[k];
    }
    uint32_t ppl = 0, chunk = 0;
    if (!choose_shape_tuned(*g, k, kNoAllocScratchBytes - fixed_bytes, tune_ppl, tune_chunk, &ppl,
                            &chunk)) {
        const uint64_t unit = 32ull * shape_ppl(k, tune_ppl);  // the smallest point chunk
        return fail(RR_ENOMEM,
                    "rr_reach_device_noalloc: this graph needs " +
                        std::to_string(fixed_bytes + 2ull * g->state_rows * unit * 8) +
                        " bytes of scratch for the smallest point chunk (" + std::to_string(unit) +
                        " points), more than the " + std::to_string(kNoAllocScratchBytes) +
                        "-byte static scratch");
    }
    uint64_t *d_z = scratch;
    uint32_t *d_shades = reinterpret_cast<uint32_t *>(scratch + z_words);
    uint64_t *d_state = scratch + z_words + shade_words;

    cudaStream_t st = (cudaStream_t)stream;
    if (q->motif) {
        ShadeTable sh;
        make_shades(q->motif, k, &sh);
        k_put_shades<<<1, 256, 0, st>>>(sh, d_shades);
        RR_LAUNCHED();
    }
    s = launch_ztable(*g, k, make_keys(q->seed), q->motif != nullptr, d_shades, d_z, st);
    if (s != RR_OK) return s;
    RR_CUDA(cudaMemsetAsync(d_witness, 0, (size_t)g->n * 8, st));
    // run_query_layers clears state row 0 of both buffers before the first layer
    s = run_query_layers(*g, q, d_z, d_state, ppl, chunk, d_witness, nullptr, 0, nullptr, st);
    if (s != RR_OK) return s;
    if (d_bitmap) return launch_bitmap(d_witness, g->n, d_bitmap, st);
    return RR_OK;
}
