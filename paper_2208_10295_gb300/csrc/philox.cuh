// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), device side.
//
// Round: (hi0, lo0) = M0 * x0, (hi1, lo1) = M1 * x2 (128-bit products);
//        x = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0).
// Key schedule: k += (W0, W1) before every round but the first.
#pragma once
#include <stdint.h>

namespace lidar {

struct U64x4 {
    uint64_t x0, x1, x2, x3;
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c.x0), lo0 = M0 * c.x0;
        const uint64_t hi1 = __umul64hi(M1, c.x2), lo1 = M1 * c.x2;
        U64x4 n;
        n.x0 = hi1 ^ c.x1 ^ k0;
        n.x1 = lo1;
        n.x2 = hi0 ^ c.x3 ^ k1;
        n.x3 = lo0;
        c = n;
    }
    return c;
}

// Standard normal for (beam, frame, sensor, sub-ray): counter
// (beam, frame | sensor << 32, sub, 0), key (seed, 0); uniforms
// u = ((x >> 11) + 1/2) 2^-53 in (0, 1); Box-Muller z = sqrt(-2 ln u0) cos(2 pi u1)
// evaluated in FP32 with CUDA's logf, sqrtf and cospif.
__device__ __forceinline__ float range_noise_normal(uint64_t seed, uint32_t beam, uint32_t frame, uint32_t sensor,
                                                    uint32_t sub)
{
    U64x4 c;
    c.x0 = beam;
    c.x1 = (uint64_t)frame | ((uint64_t)sensor << 32);
    c.x2 = sub;
    c.x3 = 0;
    U64x4 r = philox4x64_10(c, seed, 0);
    const float u0 = (float)(((double)(r.x0 >> 11) + 0.5) * 0x1p-53);
    const float u1 = (float)(((double)(r.x1 >> 11) + 0.5) * 0x1p-53);
    return sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
}

}  // namespace lidar
