// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of
//   (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
// with the key (k0, k1) advanced by the Weyl constants (W0, W1) after each
// round.  The sweep kernels use a form with the rounds that do not depend on
// the varying counter word hoisted out of the per-field loop.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define ISING_HD __host__ __device__ __forceinline__
#else
#define ISING_HD inline
#endif

namespace ising {

// Philox4x32-10 constants (Salmon, Moraes, Dror, Shaw, SC'11): round
// multipliers and the Weyl increments of the key schedule.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// hi, lo of the 64-bit product a * b.  On the device as two 32-bit
// multiplies (high and low half): measured 0.7-5.6% faster on GB300 than one
// 32x32->64 multiply, whose register-pair result constrains the allocation.
ISING_HD void mul_hilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo)
{
#if defined(__CUDA_ARCH__)
    hi = __umulhi(a, b);
    lo = a * b;
#else
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

// Generic Philox4x32 round with round key (k0, k1).
ISING_HD void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                             uint32_t& x3, uint32_t k0, uint32_t k1)
{
    uint32_t h0, l0, h1, l1;
    mul_hilo(kPhiloxM0, x0, h0, l0);
    mul_hilo(kPhiloxM1, x2, h1, l1);
    x0 = h1 ^ x1 ^ k0;
    x1 = l1;
    x2 = h0 ^ x3 ^ k1;
    x3 = l0;
}

// Full Philox4x32-10 of one counter (used by the init kernel and test hook).
ISING_HD void philox10(uint32_t x[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r)
        philox_round(x[0], x[1], x[2], x[3], k0 + (uint32_t)r * kPhiloxW0,
                     k1 + (uint32_t)r * kPhiloxW1);
}

// Round keys (k0 + r W0, k1 + r W1), r = 0..9, built once on the host so that
// the rounds read them as launch constants.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

ISING_HD PhiloxKeys philox_keys(uint32_t k0, uint32_t k1)
{
    PhiloxKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0 + (uint32_t)r * kPhiloxW0;
        rk.k1[r] = k1 + (uint32_t)r * kPhiloxW1;
    }
    return rk;
}

// Philox4x32-10 for counters (g, m, tl, th) where g, tl, th are fixed for the
// thread and m varies.  Every product and XOR of the first three rounds that
// does not depend on m is computed once here, leaving 16 multiplies per call.
struct PhiloxRowKey {
    uint32_t a;      // round 0: y0 = a ^ m
    uint32_t y3k;    // round 1: z2 = hi(M0 y0) ^ y3k
    uint32_t z1k;    // round 2: v0 = hi(M1 z2) ^ z1k
    uint32_t hiC;    // round 2: v2 = hiC ^ lo(M0 y0)
    uint32_t v3;     // round 2: v3 (independent of m)
};

ISING_HD PhiloxRowKey philox_row_key(uint32_t g, uint32_t tl, uint32_t th, const PhiloxKeys& rk)
{
    PhiloxRowKey p;
    uint32_t h0, l0, h1, l1;
    // round 0 on (g, m, tl, th)
    mul_hilo(kPhiloxM0, g, h0, l0);
    mul_hilo(kPhiloxM1, tl, h1, l1);
    p.a = h1 ^ rk.k0[0];                    // y0 = h1 ^ m ^ k0
    const uint32_t y1 = l1;
    const uint32_t y2 = h0 ^ th ^ rk.k1[0];
    const uint32_t y3 = l0;
    // round 1: the x2 product is fixed
    uint32_t h1b, l1b;
    mul_hilo(kPhiloxM1, y2, h1b, l1b);
    const uint32_t z0 = h1b ^ y1 ^ rk.k0[1];
    const uint32_t z1 = l1b;
    p.y3k = y3 ^ rk.k1[1];                  // z2 = hi(M0 y0) ^ y3 ^ k1
    // round 2: the x0 product is fixed
    uint32_t h0c, l0c;
    mul_hilo(kPhiloxM0, z0, h0c, l0c);
    p.z1k = z1 ^ rk.k0[2];                  // v0 = hi(M1 z2) ^ z1 ^ k0
    p.hiC = h0c ^ rk.k1[2];                 // v2 = h0c ^ z3 ^ k1
    p.v3 = l0c;
    return p;
}

// ROUNDS = 10 is Philox4x32-10; ROUNDS = 7 the opt-in cheaper member of the
// same family (the same iteration stopped after 7 rounds).
template <int ROUNDS = 10>
ISING_HD void philox_row(const PhiloxRowKey& p, const PhiloxKeys& rk, uint32_t m, uint32_t out[4])
{
    static_assert(ROUNDS >= 3 && ROUNDS <= 10, "3..10 rounds");
    uint32_t h, l;
    const uint32_t y0 = p.a ^ m;
    mul_hilo(kPhiloxM0, y0, h, l);
    const uint32_t z2 = h ^ p.y3k;
    const uint32_t z3 = l;
    mul_hilo(kPhiloxM1, z2, h, l);
    uint32_t x0 = h ^ p.z1k;
    uint32_t x1 = l;
    uint32_t x2 = p.hiC ^ z3;
    uint32_t x3 = p.v3;
#pragma unroll
    for (int r = 3; r < ROUNDS; ++r)
        philox_round(x0, x1, x2, x3, rk.k0[r], rk.k1[r]);
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

}  // namespace ising
