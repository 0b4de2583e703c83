// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), restated for the
// library: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by the
// Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.  Usable from host
// code (tree draws) and device code (the sweeps).
//
// Streams: key = (seed_lo, seed_hi ^ domain).  The domain words and the
// counter layout of every stream are part of the library's definition of the
// Markov chain; they are restated, not shared, by the CPU checker.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SQA_HD __host__ __device__ __forceinline__
#else
#define SQA_HD inline
#endif

namespace sqa {

constexpr uint32_t kDomInit = 0x6A09E667u;
constexpr uint32_t kDomSweepHi = 0xBB67AE85u;
constexpr uint32_t kDomSweepLo = 0x3C6EF372u;
constexpr uint32_t kDomSwap = 0xA54FF53Au;
constexpr uint32_t kDomTree = 0x510E527Fu;
constexpr uint32_t kDomWStart = 0x9B05688Cu;  // cluster start slice
constexpr uint32_t kDomWBond = 0x1F83D9ABu;   // cluster bond bit-planes
constexpr uint32_t kDomWAcc = 0x5BE0CD19u;    // cluster acceptance

struct U4 {
    uint32_t x, y, z, w;
};

// The 32x32 -> 64 product of a round, high and low words.  On the device one
// wide multiply gives both (measured 8 % faster per block than separate
// high and low products).
SQA_HD void mul_wide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#if defined(__CUDA_ARCH__)
    asm("{\n\t.reg .b64 t;\n\tmul.wide.u32 t, %2, %3;\n\tmov.b64 {%0, %1}, t;\n\t}"
        : "=r"(lo), "=r"(hi)
        : "r"(a), "r"(b));
#else
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

// One Philox4x32-10 block.  The key schedule k + r*W is formed per round.
SQA_HD U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; r++) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c0, hi0, lo0);
        mul_wide(0xCD9E8D57u, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// The same block with its ten round keys given (ka[r] = k0 + r * 0x9E3779B9,
// kb[r] = k1 + r * 0xBB67AE85), e.g. precomputed once per launch.
SQA_HD U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t (&ka)[10],
                    const uint32_t (&kb)[10])
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; r++) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c0, hi0, lo0);
        mul_wide(0xCD9E8D57u, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ ka[r], n2 = hi0 ^ c3 ^ kb[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// The same block with each product formed by one 32x32->64 multiply.
SQA_HD U4 philox_wide(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

SQA_HD uint32_t word_of(const U4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

}  // namespace sqa
