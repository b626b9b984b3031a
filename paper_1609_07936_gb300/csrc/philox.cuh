// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), written for the device.  Ten rounds; each
// round multiplies counter words 0 and 2 by the two round multipliers, keeps the
// 64-bit products' high and low halves, and mixes the high halves with words 1 and 3
// and the round key; the key advances by the two Weyl increments between rounds.
#pragma once
#include <cstdint>

namespace sail {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint2 philox_key(uint64_t seed) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// A word to a uniform on (0, 1): (w + 1/2) 2^-32, exact in FP64.
__device__ __forceinline__ double unit64(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

// The top 24 bits of a word to a uniform on (0, 1): exact in FP32.
__device__ __forceinline__ float unit32(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }

// Bin choice of a move (zero-length index walk, Sec. 2.3): p uniform on [0, n),
// s uniform on the other n - 1 bins.
__device__ __forceinline__ void move_bins(uint32_t w0, uint32_t w1, int n, int &p, int &s) {
    p = (int)(((uint64_t)w0 * (uint64_t)n) >> 32);
    s = (int)(((uint64_t)w1 * (uint64_t)(n - 1)) >> 32);
    s += (s >= p);
}

}  // namespace sail
