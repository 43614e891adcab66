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

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the TMA engine's cp.async.bulk) into shared memory,
// completed on an mbarrier that counts the bytes still in flight.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make the initialised barriers visible to the async proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of copies to complete this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// Has the phase of the given parity completed?  (Does not block.)
__device__ __forceinline__ bool mbar_test_parity(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity, at most `limit` polls (with a short
// sleep between them); false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0;; ++it) {
        if (mbar_test_parity(bar, parity))
            return true;
        if (it >= limit)
            return false;
        __nanosleep(32);
    }
}

// Order this thread's earlier shared-memory accesses before later async-proxy
// writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to shared memory; the barrier's transaction count drops by `bytes` on arrival.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Four independent Philox4x32-10 calls advanced round by round together: each
// round key serves four calls, and the four multiply chains overlap.
__device__ __forceinline__ void philox10_rk_x4(uint4 (&c)[4], const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c[k].x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[k].z;
            c[k] = make_uint4((uint32_t)(p1 >> 32) ^ c[k].y ^ rk[2 * r], (uint32_t)p1,
                              (uint32_t)(p0 >> 32) ^ c[k].w ^ rk[2 * r + 1], (uint32_t)p0);
        }
    }
}

constexpr uint32_t kStreamCouplings = 0u << 30;
constexpr uint32_t kStreamSpins = 1u << 30;
constexpr uint32_t kStreamHeat = 2u << 30;         // heat-bath coin words and gaps
constexpr uint32_t kStreamMetropolis = 3u << 30;   // Metropolis geometric gaps

}  // namespace dev
}  // namespace ea
