// rr_sieve.cu -- the sieve's device path for one query: z-table (Eq. (2)/(3)),
// the layer kernel (Eq. (1) in edge form, all sieve points of a chunk at once)
// with the per-vertex XOR reduce fused into the last layer (Algorithm 1's
// per-vertex sums), and the reach bitmap.
//
// Layer l value of edge e at sieve point L (e = (u, v, t_e)):
//   P_1^L[e] = [u = s] y_{e,1} x_s^L x_v^L
//   P_l^L[e] = y_{e,l} x_v^L W_l^L[e],  W_l^L[e] = sum of P_{l-1}^L[f] over the
//              rows f of u's in-segment inside e's restless window.
// The window sum is the XOR of two entries of a per-segment prefix-XOR state
// (so the paper's loop over j in {0..delta} disappears), and
// y_{e,l} x_v^L = sum_{j in L} b_j with b_j = y_{e,l} z_{v,j}: the k products
// b_j are formed once per edge (one per lane) and each point needs a single
// general multiplication P = W * c^L.
#include <algorithm>
#include <cstring>

#include "rr_device.cuh"
#include "rr_internal.h"

namespace rr {

struct LayerParams {
    const uint32_t *off;
    const uint32_t *row_a;
    const uint32_t *row_b;
    const uint32_t *row_s;
    const uint32_t *row_eid;
    const uint32_t *row_src;
    const uint2 *items;
    uint32_t nitems;
    const uint64_t *z;  // n x k
    uint32_t n, k, source, layer;
    uint64_t key_y;
    uint32_t chunk_base;  // first point of this chunk
    uint32_t chunk;       // points per chunk = state row stride
    uint32_t ngroups;     // chunk / (32 * PPL)
    uint32_t npoints;     // number of valid points (2^k or number of masks)
    const uint64_t *st_in;
    uint64_t *st_out;
    uint64_t *S;                // last layer: per-vertex XOR target
    uint64_t *E;                // last layer: per-edge XOR target (m, by input edge) or null
    const uint8_t *src_mask;    // layer 1: a set of sources (n flags) instead of `source`
    const uint32_t *masks;      // mask-list mode: point p is masks[p]
    uint64_t *dbg_out;          // mask-list mode, last layer: out[p * n + v]
};

enum : int { kFirst = 1, kLast = 2 };
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src)
{
    return __shfl_sync(0xffffffffu, (unsigned long long)v, src);
}

template <int PPL>
__device__ __forceinline__ void load_pts(const uint64_t *__restrict__ p, uint64_t (&v)[PPL])
{
    if constexpr (PPL == 4) {
        const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        v[0] = a.x; v[1] = a.y;
    }
}

template <int PPL>
__device__ __forceinline__ void store_pts(uint64_t *__restrict__ p, const uint64_t (&v)[PPL])
{
    if constexpr (PPL == 4) {
        reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(v[0], v[1]);
        reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(v[2], v[3]);
    } else {
        reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(v[0], v[1]);
    }
}

// One warp processes one (vertex range, point group): lane `lane` owns the
// PPL consecutive points lane*PPL .. lane*PPL+PPL-1 of the group, so every
// state row slice a warp touches is 32*PPL*8 contiguous bytes.
template <int PPL, int MODE, bool MASKLIST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_layer(const LayerParams p)
{
    constexpr int LOGP = PPL == 4 ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const uint32_t task = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (task >= p.nitems * p.ngroups) return;
    const uint32_t item = task / p.ngroups;
    const uint32_t group = task - item * p.ngroups;
    const uint2 range = p.items[item];
    const uint32_t k = p.k;

    const uint32_t col = group * (32u * PPL) + (uint32_t)lane * PPL;  // column within the chunk
    uint32_t L[PPL];
    bool valid[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
        const uint32_t idx = p.chunk_base + col + i;
        valid[i] = idx < p.npoints;
        L[i] = MASKLIST ? (valid[i] ? p.masks[idx] : 0u) : idx;
    }
    const uint32_t hi_bits = (p.chunk_base + group * (32u * PPL)) >> (LOGP + 5);

    uint64_t xs[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) xs[i] = 0;
    if constexpr ((MODE & kFirst) != 0) {
        for (uint32_t j = 0; j < k; ++j) {
            const uint64_t zsj = p.z[(size_t)p.source * k + j];
#pragma unroll
            for (int i = 0; i < PPL; ++i)
                if ((L[i] >> j) & 1u) xs[i] ^= zsj;
        }
    }

    for (uint32_t v = range.x; v < range.y; ++v) {
        const uint32_t r0 = p.off[v], r1 = p.off[v + 1];
        if (r0 == r1) continue;
        const uint64_t zv = (uint32_t)lane < k ? p.z[(size_t)v * k + lane] : 0ull;
        uint64_t acc[PPL];
#pragma unroll
        for (int i = 0; i < PPL; ++i) acc[i] = 0;
        bool any = false;
        for (uint32_t r = r0; r < r1; ++r) {
            const uint32_t ra = p.row_a[r];
            const uint32_t rs = ((MODE & kLast) != 0) ? 0u : p.row_s[r];
            const bool compute = ((MODE & kFirst) != 0)
                                     ? (p.src_mask ? p.src_mask[p.row_src[r]] != 0 : p.row_src[r] == p.source)
                                     : (ra != 0u);
            if constexpr ((MODE & kLast) != 0) {
                if (!compute) continue;
            } else {
                if (rs == 0u) continue;  // not inside any window: nobody reads its prefix
            }
            if (compute) {
                const uint32_t eid = p.row_eid[r];
                const uint64_t y = sm_draw(p.key_y, (uint64_t)eid * 32u + (p.layer - 1u));
                const uint64_t b = gf64_mul(y, zv);  // lane j holds b_{j+1} = y z_{v,j+1}
                uint64_t c[PPL];
                if constexpr (MASKLIST) {
#pragma unroll
                    for (int i = 0; i < PPL; ++i) c[i] = 0;
                    for (uint32_t j = 0; j < k; ++j) {
                        const uint64_t bj = shfl64(b, (int)j);
#pragma unroll
                        for (int i = 0; i < PPL; ++i)
                            if ((L[i] >> j) & 1u) c[i] ^= bj;
                    }
                } else {
                    uint64_t base = 0, low0 = 0, low1 = 0;
                    for (uint32_t j = 0; j < k; ++j) {
                        const uint64_t bj = shfl64(b, (int)j);
                        if (j == 0) low0 = bj;
                        else if (LOGP == 2 && j == 1) low1 = bj;
                        else if (j < (uint32_t)LOGP + 5u) {
                            if (((uint32_t)lane >> (j - LOGP)) & 1u) base ^= bj;
                        } else if ((hi_bits >> (j - LOGP - 5u)) & 1u) {
                            base ^= bj;
                        }
                    }
                    c[0] = base;
                    c[1] = base ^ low0;
                    if constexpr (PPL == 4) {
                        c[2] = base ^ low1;
                        c[3] = base ^ low0 ^ low1;
                    }
                }
                uint64_t w[PPL];
                if constexpr ((MODE & kFirst) != 0) {
                    if (p.src_mask) {
                        // x_u of this row's tail u (one of the sources)
                        const size_t u = p.row_src[r];
#pragma unroll
                        for (int i = 0; i < PPL; ++i) w[i] = 0;
                        for (uint32_t j = 0; j < k; ++j) {
                            const uint64_t zuj = p.z[u * k + j];
#pragma unroll
                            for (int i = 0; i < PPL; ++i)
                                if ((L[i] >> j) & 1u) w[i] ^= zuj;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < PPL; ++i) w[i] = xs[i];
                    }
                } else {
                    const uint32_t rb = p.row_b[r];
                    uint64_t wa[PPL], wb[PPL];
                    load_pts<PPL>(p.st_in + (size_t)ra * p.chunk + col, wa);
                    load_pts<PPL>(p.st_in + (size_t)rb * p.chunk + col, wb);
#pragma unroll
                    for (int i = 0; i < PPL; ++i) w[i] = wa[i] ^ wb[i];
                }
                uint64_t dsum = 0;  // this row's own sum over the lane's points
#pragma unroll
                for (int i = 0; i < PPL; ++i) {
                    const uint64_t inc = valid[i] ? gf64_mul(w[i], c[i]) : 0ull;
                    acc[i] ^= inc;
                    dsum ^= inc;
                }
                any = true;
                if constexpr ((MODE & kLast) != 0 && !MASKLIST) {
                    if (p.E) {
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            dsum ^= __shfl_xor_sync(0xffffffffu, (unsigned long long)dsum, off);
                        if (lane == 0 && dsum)
                            atomicXor(reinterpret_cast<unsigned long long *>(p.E + eid),
                                      (unsigned long long)dsum);
                    }
                }
            }
            if constexpr ((MODE & kLast) == 0) store_pts<PPL>(p.st_out + (size_t)rs * p.chunk + col, acc);
        }
        if constexpr ((MODE & kLast) != 0) {
            if (!any) continue;
            if constexpr (MASKLIST) {
#pragma unroll
                for (int i = 0; i < PPL; ++i)
                    if (valid[i] && acc[i])
                        p.dbg_out[(size_t)(p.chunk_base + col + i) * p.n + v] = acc[i];
            } else {
                uint64_t t = 0;
#pragma unroll
                for (int i = 0; i < PPL; ++i) t ^= acc[i];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    t ^= __shfl_xor_sync(0xffffffffu, (unsigned long long)t, off);
                if (lane == 0 && t) atomicXor(reinterpret_cast<unsigned long long *>(p.S + v),
                                              (unsigned long long)t);
            }
        }
    }
}

// z_{u,j} (j = 0..k-1 stored at u*k + j): plain iid draws or Eq. (3).
__global__ void k_ztable(uint32_t n, uint32_t k, uint64_t key_z, uint64_t key_g, uint64_t key_o,
                         const uint8_t *__restrict__ color, const uint32_t *__restrict__ shades,
                         uint64_t *__restrict__ z, const uint8_t *__restrict__ vmask)
{
    const uint64_t total = (uint64_t)n * k;
    for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t u = idx / k;
        const uint32_t j = (uint32_t)(idx - u * k);
        uint64_t val;
        if (shades == nullptr) {
            val = sm_draw(key_z, u * 32u + j);
        } else {
            const uint32_t c = color[u];
            const uint32_t d0 = shades[c], mu = shades[256 + c];
            val = 0;
            for (uint32_t d = d0; d < d0 + mu; ++d)
                val ^= gf64_mul(sm_draw(key_g, u * 32u + d), sm_draw(key_o, (uint64_t)d * 32u + j));
        }
        if (vmask && vmask[u]) val = 0;  // deleted vertex
        z[idx] = val;
    }
}

__global__ void k_bitmap(const uint64_t *__restrict__ S, uint32_t n, uint8_t *__restrict__ bm)
{
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

__global__ void k_gf_mul(const uint64_t *a, const uint64_t *b, uint64_t *o, uint64_t count)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        o[i] = gf64_mul(a[i], b[i]);
}

__global__ void k_draw(uint64_t key, uint64_t first, uint64_t count, uint64_t *o)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        o[i] = sm_draw(key, first + i);
}

static unsigned grid_1d(uint64_t count, unsigned block)
{
    uint64_t g = (count + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535ull * 16) g = 65535ull * 16;
    return (unsigned)g;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
QueryKeys make_keys(uint64_t seed)
{
    return QueryKeys{family_key(seed, kTagY), family_key(seed, kTagZ),
                     family_key(seed, kTagGamma), family_key(seed, kTagOmega)};
}

void make_shades(const uint8_t *motif, uint32_t k, ShadeTable *out)
{
    std::memset(out, 0, sizeof *out);
    for (uint32_t i = 0; i < k; ++i) out->mu[motif[i]]++;
    uint32_t next = 0;
    for (uint32_t c = 0; c < 256; ++c) {
        out->first[c] = next;
        next += out->mu[c];
    }
}

rr_status validate_query(const Graph &g, const rr_query *q)
{
    if (!q) return fail(RR_EINVAL, "query is NULL");
    if (q->k < 2 || q->k > 20) return fail(RR_EINVAL, "k must be in [2, 20]");
    if (q->source >= g.n) return fail(RR_EINVAL, "source >= n");
    if (q->motif && !g.has_colors) return fail(RR_EINVAL, "motif query on a graph without colours");
    return RR_OK;
}

bool choose_shape(const Graph &g, uint32_t k, uint64_t budget, uint32_t *ppl_out,
                  uint32_t *chunk_out)
{
    return choose_shape_tuned(g, k, budget, g.tune_ppl[k], g.tune_chunk[k], ppl_out, chunk_out);
}

uint32_t shape_ppl(uint32_t k, uint32_t tune_ppl)
{
    return tune_ppl ? tune_ppl : ((1ull << k) >= 128 ? 4u : 2u);
}

bool choose_shape_tuned(const Graph &g, uint32_t k, uint64_t budget, uint32_t tune_ppl,
                        uint32_t tune_chunk, uint32_t *ppl_out, uint32_t *chunk_out)
{
    const uint64_t npts = 1ull << k;
    uint32_t ppl = shape_ppl(k, tune_ppl);
    uint64_t unit = 32ull * ppl;
    uint64_t want = tune_chunk ? tune_chunk : npts;
    if (want < unit) want = unit;
    if (want > 2048) want = 2048;
    want = (want + unit - 1) / unit * unit;
    while (want > unit && 2ull * g.state_rows * want * 8ull > budget) want -= unit;
    if (2ull * g.state_rows * want * 8ull > budget) return false;
    *ppl_out = ppl;
    *chunk_out = (uint32_t)want;
    return true;
}

rr_status launch_ztable(const Graph &g, uint32_t k, const QueryKeys &keys, bool colored,
                        const uint32_t *d_shades, uint64_t *d_z, cudaStream_t st,
                        const uint8_t *d_vmask)
{
    const int tslot = timing_begin(st);
    k_ztable<<<grid_1d((uint64_t)g.n * k, 256), 256, 0, st>>>(
        g.n, k, keys.key_z, keys.key_gamma, keys.key_omega,
        colored ? g.color.as<uint8_t>() : nullptr, colored ? d_shades : nullptr, d_z, d_vmask);
    timing_end(tslot, kTimeZ, st);
    RR_LAUNCHED();
    return RR_OK;
}

rr_status launch_bitmap(const uint64_t *d_S, uint32_t n, uint8_t *d_bitmap, cudaStream_t st)
{
    k_bitmap<<<grid_1d((n + 7) / 8, 256), 256, 0, st>>>(d_S, n, d_bitmap);
    RR_LAUNCHED();
    return RR_OK;
}

template <int PPL>
static rr_status launch_layer_ppl(const LayerParams &lp, int mode, bool masklist, cudaStream_t st)
{
    const uint64_t tasks = (uint64_t)lp.nitems * lp.ngroups;
    if (tasks == 0) return RR_OK;
    const unsigned blocks = (unsigned)((tasks + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const unsigned threads = kWarpsPerBlock * 32;
    const int tslot = timing_begin(st);
#define RR_LAYER_CASE(M, ML) k_layer<PPL, M, ML><<<blocks, threads, 0, st>>>(lp)
    if (masklist) {
        switch (mode) {
        case 0: RR_LAYER_CASE(0, true); break;
        case kFirst: RR_LAYER_CASE(kFirst, true); break;
        case kLast: RR_LAYER_CASE(kLast, true); break;
        default: RR_LAYER_CASE(kFirst | kLast, true); break;
        }
    } else {
        switch (mode) {
        case 0: RR_LAYER_CASE(0, false); break;
        case kFirst: RR_LAYER_CASE(kFirst, false); break;
        case kLast: RR_LAYER_CASE(kLast, false); break;
        default: RR_LAYER_CASE(kFirst | kLast, false); break;
        }
    }
#undef RR_LAYER_CASE
    timing_end(tslot, (mode & kFirst) ? kTimeFirst : ((mode & kLast) ? kTimeLast : kTimeMid), st);
    RR_LAUNCHED();
    return RR_OK;
}

rr_status run_query_layers(const Graph &g, const rr_query *q, const uint64_t *d_z,
                           uint64_t *d_state, uint32_t ppl, uint32_t chunk, uint64_t *d_S,
                           const uint32_t *d_masks, uint32_t nmasks, uint64_t *d_debug_out,
                           cudaStream_t st, uint64_t *d_E, const uint8_t *d_srcmask,
                           PointRange range)
{
    const uint32_t k = q->k;
    const bool masklist = d_masks != nullptr;
    if (masklist) range = PointRange();
    if (range.first % kRangeAlign || range.first > range.stop(k) || range.stop(k) > (1u << k))
        return fail(RR_EINVAL, "bad sieve-point range");
    // points [first, npoints): all 2^k, a range of them, or the mask list's entries
    const uint64_t first = range.first;
    const uint64_t npoints = masklist ? nmasks : range.stop(k);
    const uint64_t nchunks = (npoints - first + chunk - 1) / chunk;
    uint64_t *buf[2] = {d_state, d_state + (size_t)g.state_rows * chunk};
    // state row 0 is the zero row of both buffers (never written by a layer)
    RR_CUDA(cudaMemsetAsync(buf[0], 0, (size_t)chunk * 8, st));
    RR_CUDA(cudaMemsetAsync(buf[1], 0, (size_t)chunk * 8, st));

    LayerParams lp{};
    lp.off = g.off.as<uint32_t>();
    lp.row_a = g.row_a.as<uint32_t>();
    lp.row_b = g.row_b.as<uint32_t>();
    lp.row_s = g.row_s.as<uint32_t>();
    lp.row_eid = g.row_eid.as<uint32_t>();
    lp.row_src = g.row_src.as<uint32_t>();
    lp.items = g.items.as<uint2>();
    lp.nitems = g.nitems;
    lp.z = d_z;
    lp.n = g.n;
    lp.k = k;
    lp.source = q->source;
    lp.key_y = make_keys(q->seed).key_y;
    lp.chunk = chunk;
    lp.ngroups = chunk / (32u * ppl);
    lp.npoints = (uint32_t)npoints;
    lp.S = d_S;
    lp.E = d_E;
    lp.src_mask = d_srcmask;
    lp.masks = d_masks;
    lp.dbg_out = d_debug_out;
    for (uint64_t c = 0; c < nchunks; ++c) {
        lp.chunk_base = (uint32_t)(first + c * chunk);
        for (uint32_t l = 1; l <= k - 1; ++l) {
            lp.layer = l;
            // layer l reads buf[(l-1)&1] (written by layer l-1) and writes buf[l&1]
            lp.st_in = buf[(l - 1) & 1u];
            lp.st_out = buf[l & 1u];
            int mode = (l == 1 ? kFirst : 0) | (l == k - 1 ? kLast : 0);
            rr_status s = (ppl == 4) ? launch_layer_ppl<4>(lp, mode, masklist, st)
                                     : launch_layer_ppl<2>(lp, mode, masklist, st);
            if (s != RR_OK) return s;
        }
    }
    return RR_OK;
}

bool uses_v2(const Graph &g, uint32_t k)
{
    return g.compact && k >= 2;
}

bool choose_shape_v2(const Graph &g, uint32_t k, uint64_t budget, uint32_t *ppl_out,
                     uint32_t *chunk_out)
{
    const uint64_t npts = 1ull << k;
    const uint32_t ppl = g.tune_ppl[k] ? g.tune_ppl[k] : (npts >= 128 ? 4u : 2u);
    const uint64_t unit = 32ull * ppl;
    uint64_t want = g.tune_chunk[k] ? g.tune_chunk[k] : npts;
    want = std::max<uint64_t>(unit, std::min<uint64_t>(want, 8 * unit));  // <= 8 groups
    want = (want + unit - 1) / unit * unit;
    while (want > unit && v2_scratch_bytes(g, ppl, (uint32_t)want, k) > budget) want -= unit;
    if (v2_scratch_bytes(g, ppl, (uint32_t)want, k) > budget) return false;
    *ppl_out = ppl;
    *chunk_out = (uint32_t)want;
    return true;
}

uint64_t query_scratch_bytes(const Graph &g, uint32_t k, uint64_t budget)
{
    uint32_t ppl = 0, chunk = 0;
    const uint64_t z = (uint64_t)g.n * k * 8ull + 2048;
    if (uses_v2(g, k)) {
        if (!choose_shape_v2(g, k, budget, &ppl, &chunk)) return UINT64_MAX;
        return v2_scratch_bytes(g, ppl, chunk, k) + z;
    }
    if (!choose_shape(g, k, budget, &ppl, &chunk)) return UINT64_MAX;
    return 2ull * g.state_rows * chunk * 8ull + z;
}

rr_status reach_on_stream(const Graph &g, Workspace &ws, const rr_query *q, uint8_t *d_bitmap,
                          uint64_t *d_witness, uint64_t budget, cudaStream_t st, uint64_t *d_E,
                          const uint8_t *d_vmask, const uint8_t *d_srcmask, PointRange range,
                          uint32_t bfirst, uint64_t *b_witness, uint64_t *b_edges)
{
    rr_status vs = validate_query(g, q);
    if (vs != RR_OK) return vs;
    const uint32_t k = q->k;
    if (!range.full(k) && (k <= 3 || d_bitmap))
        return fail(RR_EINVAL, "a part of the sieve points needs k >= 4 and gives no bitmap");
    // a set of sources runs on the per-point engine (the reduced-state engine
    // factors x_s out of layer 1); its shape is never cached per k
    const bool v2 = uses_v2(g, k) && !d_srcmask;
    if (bfirst && (!v2 || q->motif || d_vmask || !range.full(k) || bfirst < atmost_first_branch(g, k) ||
                   k - bfirst > Workspace::kMaxBranches))
        return fail(RR_EINVAL, "internal: at-most-k branches need a plain whole query on the reduced-state engine");
    if (d_srcmask && budget == 0) {
        size_t free_b = 0, total_b = 0;
        RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
        budget = (uint64_t)(0.6 * (double)(free_b + ws.state.bytes));
    }
    uint32_t ppl = 0, chunk = 0;
    if (budget == 0 && ws.shape_ppl[k] && ws.shape_gen[k] == g.tune_gen) {
        // shape already chosen for this k on this workspace: no device query
        ppl = ws.shape_ppl[k];
        chunk = ws.shape_chunk[k];
    } else {
        const bool remember = budget == 0;
        if (budget == 0) {
            size_t free_b = 0, total_b = 0;
            RR_CUDA(cudaMemGetInfo(&free_b, &total_b));
            budget = (uint64_t)(0.6 * (double)(free_b + ws.state.bytes));
        }
        if (v2 ? !choose_shape_v2(g, k, budget, &ppl, &chunk)
               : !choose_shape(g, k, budget, &ppl, &chunk))
            return fail(RR_ENOMEM, "state for one point chunk does not fit device memory");
        if (remember) {
            ws.shape_ppl[k] = ppl;
            ws.shape_chunk[k] = chunk;
            ws.shape_gen[k] = g.tune_gen;
        }
    }
    RR_CUDA(ws.state.reserve(v2 ? v2_scratch_bytes(g, ppl, chunk, k, bfirst != 0)
                                : 2ull * g.state_rows * chunk * 8ull));
    RR_CUDA(ws.z.reserve((size_t)g.n * k * 8));
    if (v2)
        return reach_v2(g, ws, q, d_bitmap, d_witness, ppl, chunk, st, d_E, d_vmask, range, bfirst,
                        b_witness, b_edges);
    const QueryKeys keys = make_keys(q->seed);
    const uint32_t *d_shades = nullptr;
    if (q->motif) {
        ShadeTable sh;
        make_shades(q->motif, k, &sh);
        RR_CUDA(ws.shade.reserve(sizeof sh));
        RR_CUDA(cudaMemcpyAsync(ws.shade.p, &sh, sizeof sh, cudaMemcpyHostToDevice, st));
        d_shades = ws.shade.as<uint32_t>();
    }
    rr_status s = launch_ztable(g, k, keys, q->motif != nullptr, d_shades, ws.z.as<uint64_t>(), st,
                                d_vmask);
    if (s != RR_OK) return s;
    RR_CUDA(cudaMemsetAsync(d_witness, 0, (size_t)g.n * 8, st));
    s = run_query_layers(g, q, ws.z.as<uint64_t>(), ws.state.as<uint64_t>(), ppl, chunk, d_witness,
                         nullptr, 0, nullptr, st, d_E, d_srcmask, range);
    if (s != RR_OK) return s;
    if (d_bitmap) return launch_bitmap(d_witness, g.n, d_bitmap, st);
    return RR_OK;
}

rr_status debug_point_sums(const Graph &g, const rr_query *q, const uint32_t *masks,
                           uint32_t nmasks, uint64_t *out)
{
    rr_status vs = validate_query(g, q);
    if (vs != RR_OK) return vs;
    if (!out || (!masks && nmasks)) return fail(RR_EINVAL, "NULL masks/out");
    for (uint32_t i = 0; i < nmasks; ++i)
        if (masks[i] >> q->k) return fail(RR_EINVAL, "mask has bits at or above k");
    std::lock_guard<std::mutex> lk(g.mu);
    cudaStream_t st = g.stream;
    const uint32_t k = q->k;
    if (nmasks == 0) return RR_OK;
    uint32_t ppl = 2, chunk = 64;
    RR_CUDA(g.ws.state.reserve(2ull * g.state_rows * chunk * 8ull));
    RR_CUDA(g.ws.z.reserve((size_t)g.n * k * 8));
    DevBuf d_masks, d_out;
    RR_CUDA(d_masks.reserve((size_t)nmasks * 4));
    RR_CUDA(d_out.reserve((size_t)nmasks * g.n * 8));
    RR_CUDA(cudaMemcpyAsync(d_masks.p, masks, (size_t)nmasks * 4, cudaMemcpyHostToDevice, st));
    RR_CUDA(cudaMemsetAsync(d_out.p, 0, (size_t)nmasks * g.n * 8, st));
    const QueryKeys keys = make_keys(q->seed);
    const uint32_t *d_shades = nullptr;
    ShadeTable sh;
    if (q->motif) {
        make_shades(q->motif, k, &sh);
        RR_CUDA(g.ws.shade.reserve(sizeof sh));
        RR_CUDA(cudaMemcpyAsync(g.ws.shade.p, &sh, sizeof sh, cudaMemcpyHostToDevice, st));
        d_shades = g.ws.shade.as<uint32_t>();
    }
    rr_status s = launch_ztable(g, k, keys, q->motif != nullptr, d_shades, g.ws.z.as<uint64_t>(), st);
    if (s != RR_OK) return s;
    s = run_query_layers(g, q, g.ws.z.as<uint64_t>(), g.ws.state.as<uint64_t>(), ppl, chunk,
                         nullptr, d_masks.as<uint32_t>(), nmasks, d_out.as<uint64_t>(), st);
    if (s != RR_OK) return s;
    RR_CUDA(cudaMemcpyAsync(out, d_out.p, (size_t)nmasks * g.n * 8, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    return RR_OK;
}

rr_status debug_ztable(const Graph &g, const rr_query *q, uint64_t *out)
{
    rr_status vs = validate_query(g, q);
    if (vs != RR_OK) return vs;
    std::lock_guard<std::mutex> lk(g.mu);
    cudaStream_t st = g.stream;
    RR_CUDA(g.ws.z.reserve((size_t)g.n * q->k * 8));
    const uint32_t *d_shades = nullptr;
    ShadeTable sh;
    if (q->motif) {
        make_shades(q->motif, q->k, &sh);
        RR_CUDA(g.ws.shade.reserve(sizeof sh));
        RR_CUDA(cudaMemcpyAsync(g.ws.shade.p, &sh, sizeof sh, cudaMemcpyHostToDevice, st));
        d_shades = g.ws.shade.as<uint32_t>();
    }
    rr_status s = launch_ztable(g, q->k, make_keys(q->seed), q->motif != nullptr, d_shades,
                                g.ws.z.as<uint64_t>(), st);
    if (s != RR_OK) return s;
    RR_CUDA(cudaMemcpyAsync(out, g.ws.z.p, (size_t)g.n * q->k * 8, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    return RR_OK;
}

// Multiply-rate microbenchmark: four dependent chains per thread, each step
// multiplying two values that both change every iteration (so nothing about an
// operand can be hoisted out of the loop), and nothing read from memory.
__global__ void k_gf_mul_rate(uint32_t iters, uint64_t *sink)
{
    const uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t a = sm_mix(id + 1), b = sm_mix(id + 2), c = sm_mix(id + 3), d = sm_mix(id + 4);
    uint64_t e = sm_mix(id + 5), f = sm_mix(id + 6), g = sm_mix(id + 7), h = sm_mix(id + 8);
    // four independent products a step; every operand value enters exactly one
    // product, as in the layer kernels (no value is multiplied twice there), so
    // the compiler cannot share an operand's split into bit classes and
    // Karatsuba sums between two products
    for (uint32_t i = 0; i < iters; ++i) {
        const uint64_t p0 = gf64_mul(a, b), p1 = gf64_mul(c, d), p2 = gf64_mul(e, f), p3 = gf64_mul(g, h);
        a = p0;
        b ^= p1;
        c = p2;
        d ^= p3;
        e = p1;
        f ^= p0;
        g = p3;
        h ^= p2;
    }
    // keeps the chains live; practically never taken
    if ((a ^ b ^ c ^ d ^ e ^ f ^ g ^ h) == 0x5EEDull) sink[0] = a;
}

rr_status bench_gf_mul(uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t *d_sink,
                       uint64_t *mults, cudaStream_t st)
{
    if (!blocks || !threads || threads > 1024 || !d_sink || !mults)
        return fail(RR_EINVAL, "rr_bench_gf_mul: bad launch shape or NULL argument");
    k_gf_mul_rate<<<blocks, threads, 0, st>>>(iters, d_sink);
    RR_LAUNCHED();
    *mults = (uint64_t)blocks * threads * iters * 4ull;
    return RR_OK;
}

rr_status debug_gf_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t count)
{
    if (count == 0) return RR_OK;
    if (!a || !b || !out) return fail(RR_EINVAL, "NULL array");
    DevBuf da, db, dout;
    RR_CUDA(da.reserve(count * 8));
    RR_CUDA(db.reserve(count * 8));
    RR_CUDA(dout.reserve(count * 8));
    RR_CUDA(cudaMemcpy(da.p, a, count * 8, cudaMemcpyHostToDevice));
    RR_CUDA(cudaMemcpy(db.p, b, count * 8, cudaMemcpyHostToDevice));
    k_gf_mul<<<grid_1d(count, 256), 256>>>(da.as<uint64_t>(), db.as<uint64_t>(),
                                           dout.as<uint64_t>(), count);
    RR_LAUNCHED();
    RR_CUDA(cudaMemcpy(out, dout.p, count * 8, cudaMemcpyDeviceToHost));
    return RR_OK;
}

rr_status debug_draw(uint64_t key, uint64_t first, uint64_t count, uint64_t *out)
{
    if (count == 0) return RR_OK;
    if (!out) return fail(RR_EINVAL, "NULL out");
    DevBuf dout;
    RR_CUDA(dout.reserve(count * 8));
    k_draw<<<grid_1d(count, 256), 256>>>(key, first, count, dout.as<uint64_t>());
    RR_LAUNCHED();
    RR_CUDA(cudaMemcpy(out, dout.p, count * 8, cudaMemcpyDeviceToHost));
    return RR_OK;
}

}  // namespace rr
