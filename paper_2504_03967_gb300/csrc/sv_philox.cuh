// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the device, and the
// library's shot-uniform convention: shot s draws word s mod 4 of block
// Philox(counter = (s div 4, 0, 0, 0), key = (seed, 0)), u = (w >> 11) 2^-53.
#pragma once

#include <stdint.h>

namespace sv {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t s) {
    uint64_t c[4] = {s >> 2, 0, 0, 0};
    philox4x64_10(c, seed, 0);
    const uint64_t w = (s & 3) == 0 ? c[0] : (s & 3) == 1 ? c[1] : (s & 3) == 2 ? c[2] : c[3];
    return (double)(w >> 11) * 0x1.0p-53;
}

}  // namespace sv
