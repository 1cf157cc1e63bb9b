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

// (k + 1/2) 2^-52 for the top 52 bits k of (hi:lo), exactly: the double 1 + k 2^-52 is
// assembled from bits and (1 - 2^-53) subtracted, which is exact by Sterbenz's lemma.
__device__ __forceinline__ double unit_from_bits(uint32_t hi, uint32_t lo) {
    unsigned long long k = ((static_cast<unsigned long long>(hi) << 32) | lo) >> 12;
    double one_plus = __longlong_as_double(0x3FF0000000000000ULL | k);
    return one_plus - 0x1.fffffffffffffp-1;
}

// The float form of a point coordinate, for the mixed-precision programs: (k + 1/2) 2^-23 for the
// top 23 bits k of hi, exactly: the float 1 + k 2^-23 assembled from bits minus (1 - 2^-24),
// exact by Sterbenz's lemma.  It lies in the same 2^-23 cell as the double form, so every VEGAS
// bin and grid cell agrees with it.
__device__ __forceinline__ float unit_from_bits_f(uint32_t hi) {
    const float one_plus = __int_as_float(0x3F800000u | (hi >> 9));
    return one_plus - 0x1.fffffep-1f;
}

}  // namespace rng
}  // namespace ps
