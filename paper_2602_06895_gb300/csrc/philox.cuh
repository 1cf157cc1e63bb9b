// philox.cuh -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the device code of the
// phase-space library: ten rounds of two 32x32->64 multiplies with the Weyl key schedule.
#pragma once
#include <cstdint>

namespace ps {
namespace rng {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

}  // namespace rng
}  // namespace ps
