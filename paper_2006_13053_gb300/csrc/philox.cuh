// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128-bit multiplications with the
// published multipliers and Weyl key increments.  One implementation for host and device code,
// so that draws made on either side are identical.
#pragma once
#include <stdint.h>

namespace sfft {

__host__ __device__ __forceinline__ void philox_mulhilo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
#ifdef __CUDA_ARCH__
    *hi = __umul64hi(a, b);
    *lo = a * b;
#else
    const unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
#endif
}

// word 0 of the output block for counter (c0, c1, c2, c3) and key (key0, 0)
__host__ __device__ __forceinline__ uint64_t philox4x64_w0(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2,
                                                            uint64_t c3) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, k0 = key0, k1 = 0;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        philox_mulhilo(M0, x0, &hi0, &lo0);
        philox_mulhilo(M1, x2, &hi1, &lo1);
        const uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    return x0;
}

// (u64 >> 11) * 2^-53: a double uniform in [0, 1)
__host__ __device__ __forceinline__ double philox4x64_u01(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2,
                                                           uint64_t c3) {
    return (double)(philox4x64_w0(key0, c0, c1, c2, c3) >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace sfft
