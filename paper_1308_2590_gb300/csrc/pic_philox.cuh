// Philox-4x64 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011): the counter-based generator of the
// ionisation and collision passes.  x is the 4-word counter, replaced by the
// 4 output words; (k0, k1) is the key.
#pragma once
#include <stdint.h>

namespace pic {

__device__ inline void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
        const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
        const uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0;
        x[1] = lo1;
        x[2] = y2;
        x[3] = lo0;
    }
}

// Output word o of a block as a uniform number in [0, 1): (o >> 11) 2^-53.
__device__ inline double philox_uniform(uint64_t o) { return (double)(o >> 11) * 0x1.0p-53; }

}  // namespace pic
