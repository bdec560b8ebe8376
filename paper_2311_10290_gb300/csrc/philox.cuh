// Philox4x32-10 on the device (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11).
//
// Every random number of the samplers is the low 64 bits of one Philox block:
//   Wilson draw at node u, its k-th draw, sample i : counter (u, k, i, 0)
//   uniform-start walk, sample i, step t           : counter (t, 0, i, 1)
//   pi-start walk, sample i, step t                : counter (t, 0, i, 2)
// with key (seed_lo, seed_hi).  Keying Wilson draws by (node, draw index)
// makes each draw an entry of Wilson's per-node stack (Section 3.4, stack
// representation), so results do not depend on execution order.
#pragma once

#include <cstdint>

namespace lap {

__device__ __forceinline__ uint64_t philox_r64(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a0 = 0xD2511F53u * c0;
        const uint32_t b0 = __umulhi(0xD2511F53u, c0);
        const uint32_t a2 = 0xCD9E8D57u * c2;
        const uint32_t b2 = __umulhi(0xCD9E8D57u, c2);
        c0 = b2 ^ c1 ^ k0;
        c1 = a2;
        c2 = b0 ^ c3 ^ k1;
        c3 = a0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return (uint64_t)c0 | ((uint64_t)c1 << 32);
}

// Uniform integer in [0, r): the high 64 bits of x * r.
__device__ __forceinline__ uint64_t below(uint64_t x, uint64_t r) { return __umul64hi(x, r); }

}  // namespace lap
