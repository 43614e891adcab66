// ea_device.cuh -- device helpers shared by the library's kernels.
#pragma once

#include <cstdint>

namespace ea {
namespace dev {

// c ? x : y, bitwise
__device__ __forceinline__ uint32_t sel(uint32_t c, uint32_t x, uint32_t y)
{
    return (c & x) | (~c & y);
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c)
{
    return (a & b) | (a & c) | (b & c);
}

// Lane realignment of a word read across the periodic wrap of the word lattice:
// a rotation of the block index inside each group of lanes of one axis.
__device__ __forceinline__ uint32_t realign(uint32_t w, int sA, uint32_t mA, int sB, uint32_t mB)
{
    return ((w >> sA) & mA) | ((w << sB) & mB);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies by 0xD2511F53 and 0xCD9E8D57; the key is bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same with the ten round keys precomputed (rk[2r], rk[2r+1] = key of round r).
// Each 32 x 32 -> 64-bit product is one wide multiply: the same multiplier
// time as separate low and high halves, but one issue slot instead of two.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

constexpr uint32_t kStreamCouplings = 0u << 30;
constexpr uint32_t kStreamSpins = 1u << 30;
constexpr uint32_t kStreamHeat = 2u << 30;         // heat-bath coin words and gaps
constexpr uint32_t kStreamMetropolis = 3u << 30;   // Metropolis geometric gaps

}  // namespace dev
}  // namespace ea
