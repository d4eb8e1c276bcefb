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
// sm_103a has no carry-less multiply instruction. A 32x32 -> 64 carry-less
// product is formed from ordinary integer products of operands with holes:
// split each operand into the four bit classes i mod 4 (masks 0x1111..,
// 0x2222.., ...). In the integer product of a class-i part and a class-j part
// every non-zero partial sum sits at a position = i+j (mod 4) and counts at
// most 8 bit pairs, so it fits in the 4-bit slot up to the next such position
// and its lowest bit is the XOR of the pairs. XOR-ing the four products that
// land in class c and masking class c gives the carry-less product's class-c
// bits (the bit-masked multiply technique described by T. Pornin for
// constant-time GHASH). 16 mul.wide.u32 per 32x32 product.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t clmul32(uint32_t a, uint32_t b)
{
    const uint32_t m0 = 0x11111111u, m1 = 0x22222222u, m2 = 0x44444444u, m3 = 0x88888888u;
    const uint64_t a0 = a & m0, a1 = a & m1, a2 = a & m2, a3 = a & m3;
    const uint64_t b0 = b & m0, b1 = b & m1, b2 = b & m2, b3 = b & m3;
    const uint64_t z0 = (a0 * b0) ^ (a1 * b3) ^ (a2 * b2) ^ (a3 * b1);
    const uint64_t z1 = (a0 * b1) ^ (a1 * b0) ^ (a2 * b3) ^ (a3 * b2);
    const uint64_t z2 = (a0 * b2) ^ (a1 * b1) ^ (a2 * b0) ^ (a3 * b3);
    const uint64_t z3 = (a0 * b3) ^ (a1 * b2) ^ (a2 * b1) ^ (a3 * b0);
    return (z0 & 0x1111111111111111ULL) | (z1 & 0x2222222222222222ULL) |
           (z2 & 0x4444444444444444ULL) | (z3 & 0x8888888888888888ULL);
}

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

// 64x64 carry-less product by one level of Karatsuba over 32-bit halves
// (three clmul32), then reduction.
__host__ __device__ __forceinline__ uint64_t gf64_mul(uint64_t a, uint64_t b)
{
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t L = clmul32(a0, b0);
    const uint64_t H = clmul32(a1, b1);
    const uint64_t M = clmul32(a0 ^ a1, b0 ^ b1) ^ L ^ H;
    const uint64_t lo = L ^ (M << 32);
    const uint64_t hi = H ^ (M >> 32);
    return gf64_reduce(hi, lo);
}

}  // namespace rr
