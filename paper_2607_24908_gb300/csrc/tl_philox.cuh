// Philox-2x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), the counter-based generator the paper
// takes from Random123 for its random fields (Sec. 2).  Per round the first
// counter word is multiplied by the published 64-bit multiplier; the new first
// word is hi(product) xor key xor second word, the new second word
// lo(product); the key advances by the published Weyl increment.
//
// On the device the 64 x 64 -> 128-bit product is __umul64hi and a 64-bit
// multiply (forming it instead from four 32 x 32 -> 64-bit partial products
// made the Langevin step, which this generator bounds, 18% slower); on the
// host it is a 128-bit integer product, so that the same header compiles for
// the host, where a test checks it against the generator's published known
// answers.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define TL_PHILOX_FN __host__ __device__ __forceinline__
#else
#define TL_PHILOX_FN inline
#endif

namespace tl {

// (hi, lo) = a * b for a, b < 2^64.
TL_PHILOX_FN void mul_64x64_128(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo)
{
#if defined(__CUDA_ARCH__)
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    const unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

TL_PHILOX_FN void philox2x64_10(uint64_t c0, uint64_t c1, uint64_t key, uint64_t &o0, uint64_t &o1)
{
    const uint64_t M = 0xD2B74407B1CE6E93ULL;
    const uint64_t Wk = 0x9E3779B97F4A7C15ULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi, lo;
        mul_64x64_128(M, c0, hi, lo);
        c0 = hi ^ key ^ c1;
        c1 = lo;
        key += Wk;
    }
    o0 = c0;
    o1 = c1;
}

}  // namespace tl
