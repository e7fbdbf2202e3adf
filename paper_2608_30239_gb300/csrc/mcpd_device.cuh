// Device helpers shared by the sampling kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcpd {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32 S-box with the Weyl
// key schedule.
static __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same with the round keys (k0 + i W0, k1 + i W1), i = 0..9, given as rk[2 i], rk[2 i + 1].
static __device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * round], lo1, hi0 ^ c.w ^ rk[2 * round + 1], lo0);
    }
    return c;
}

// Word 0 of a block, out of line (the rare draw of a uniform's low half).
static __device__ __noinline__ uint32_t philox_low_word(uint4 c, uint32_t k0, uint32_t k1) {
    return philox10(c, k0, k1).x;
}

// Fire-and-forget global reductions (no value returned, no wait).
static __device__ __forceinline__ void red_add(long long *a, long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}
static __device__ __forceinline__ void red_max(unsigned long long *a, unsigned long long v) {
    asm volatile("red.global.max.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}
static __device__ __forceinline__ void red_or(uint32_t *a, uint32_t v) {
    asm volatile("red.global.or.b32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Add G and G^2 (128-bit, carried into the high word) of one slot to bucket N*_p - 1.
static __device__ __forceinline__ void bucket_add(unsigned long long *S1, unsigned long long *S2lo,
                                           unsigned long long *S2hi, int na, int bkt, int j, long long g) {
    const size_t idx = static_cast<size_t>(bkt) * na + j;
    atomicAdd(&S1[idx], static_cast<unsigned long long>(g));
    const unsigned long long a = static_cast<unsigned long long>(g < 0 ? -g : g);
    const unsigned long long lo = a * a, hi = __umul64hi(a, a);
    const unsigned long long old = atomicAdd(&S2lo[idx], lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&S2hi[idx], hi + carry);
}

}  // namespace mcpd
