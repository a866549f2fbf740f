// philox.cuh -- the counter-based generator behind every random initial state
// (x(0), y(0), the tangents' dx(0), the twins' offsets): one definition for
// all the kernels that draw, so that they draw the same numbers.
#pragma once
#include <stdint.h>

namespace gsb {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box, key
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * ctr.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

// Uniform value in [-range, range): k = top 24 bits - 2^23, times range 2^-23,
// one FP32 rounding. Counter (i, r, stream, 0), key = seed.
__device__ __forceinline__ float uniform_draw(int i, int r, uint32_t stream, uint2 key,
                                              float scale) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)r, stream, 0u), key);
    const int k = (int)(w.x >> 8) - 8388608;
    return __fmul_rn((float)k, scale);
}

}  // namespace gsb
