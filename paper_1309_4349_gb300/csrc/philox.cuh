// philox.cuh -- the library's one implementation of Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
// four 32-bit counter words and two key words; each of ten rounds takes the two
// 32x32->64 products of words 0 and 2 with fixed multipliers, mixes their high
// halves with words 1 and 3 and the round key, and bumps the key by two Weyl
// constants.  Every random number of the library -- phase parameters, draws,
// initial placement, fraction-of-first-neighbour and image samples -- comes from
// here.  Include at file scope (outside any namespace).
#pragma once

#include <stdint.h>

namespace klmc {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // multiplier of word 0
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;  // multiplier of word 2
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // key bump of key word 0
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;  // key bump of key word 1

struct Philox4 {
    uint32_t v[4];
};

// One round on (c0, c1, c2, c3) with round key (k0, k1).
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                             uint32_t k1)
{
    const unsigned long long p0 = (unsigned long long)c0 * kPhiloxM0;
    const unsigned long long p1 = (unsigned long long)c2 * kPhiloxM1;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
}

// All four output words of counter {c0, c1, c2, c3} under key {k0, k1}.
__device__ __forceinline__ Philox4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                           uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    Philox4 out;
    out.v[0] = c0; out.v[1] = c1; out.v[2] = c2; out.v[3] = c3;
    return out;
}

// The draws of one phase use counters {site, f, s_lo, s_hi} that differ only in
// word 0.  In the first two rounds the products that do not depend on word 0 --
// s_lo * M1 in round 0 and, from it, the round-1 product of the new word 0 -- are
// the same for every draw of the phase; DrawKey holds them (with the round keys
// folded in) so that a draw pays two fewer multiplications.  The result is the
// same word 0 as philox4's.
struct DrawKey {
    uint32_t sk;  // s_hi ^ k1                       (round 0, word 2)
    uint32_t bk;  // lo(s_lo * M1) ^ (k0 + W0)       (round 1, word 0)
    uint32_t hk;  // hi(A * M0) ^ (k1 + W1), A = hi(s_lo * M1) ^ f ^ k0   (round 1, word 2)
    uint32_t la;  // lo(A * M0)                      (round 1, word 3)
    uint32_t k0, k1;
};

__device__ __forceinline__ DrawKey draw_key(uint32_t f, uint32_t s_lo, uint32_t s_hi, uint32_t k0, uint32_t k1)
{
    const unsigned long long p1 = (unsigned long long)s_lo * kPhiloxM1;
    const uint32_t A = (uint32_t)(p1 >> 32) ^ f ^ k0;
    const unsigned long long pa = (unsigned long long)A * kPhiloxM0;
    DrawKey d;
    d.sk = s_hi ^ k1;
    d.bk = (uint32_t)p1 ^ (k0 + kPhiloxW0);
    d.hk = (uint32_t)(pa >> 32) ^ (k1 + kPhiloxW1);
    d.la = (uint32_t)pa;
    d.k0 = k0;
    d.k1 = k1;
    return d;
}

// Word 0 of Philox4x32-10 at counters {a0, f, s_lo, s_hi} and {b0, f, s_lo, s_hi}
// (the phase's DrawKey), the two chains in lockstep.
__device__ __forceinline__ void philox2_w0_key(uint32_t a0, uint32_t b0, const DrawKey &d, uint32_t &ra,
                                               uint32_t &rb)
{
    // rounds 0 and 1 with the phase constants
    const unsigned long long qa = (unsigned long long)a0 * kPhiloxM0;
    const unsigned long long qb = (unsigned long long)b0 * kPhiloxM0;
    const uint32_t a2r = (uint32_t)(qa >> 32) ^ d.sk, b2r = (uint32_t)(qb >> 32) ^ d.sk;
    const unsigned long long ta = (unsigned long long)a2r * kPhiloxM1;
    const unsigned long long tb = (unsigned long long)b2r * kPhiloxM1;
    uint32_t xa0 = (uint32_t)(ta >> 32) ^ d.bk, xa1 = (uint32_t)ta, xa2 = d.hk ^ (uint32_t)qa, xa3 = d.la;
    uint32_t xb0 = (uint32_t)(tb >> 32) ^ d.bk, xb1 = (uint32_t)tb, xb2 = d.hk ^ (uint32_t)qb, xb3 = d.la;
    uint32_t k0 = d.k0 + 2u * kPhiloxW0, k1 = d.k1 + 2u * kPhiloxW1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {  // the rounds of philox_round, the products of both chains first
        const unsigned long long pa0 = (unsigned long long)xa0 * kPhiloxM0;
        const unsigned long long pa1 = (unsigned long long)xa2 * kPhiloxM1;
        const unsigned long long pb0 = (unsigned long long)xb0 * kPhiloxM0;
        const unsigned long long pb1 = (unsigned long long)xb2 * kPhiloxM1;
        const uint32_t na0 = (uint32_t)(pa1 >> 32) ^ xa1 ^ k0;
        const uint32_t na2 = (uint32_t)(pa0 >> 32) ^ xa3 ^ k1;
        const uint32_t nb0 = (uint32_t)(pb1 >> 32) ^ xb1 ^ k0;
        const uint32_t nb2 = (uint32_t)(pb0 >> 32) ^ xb3 ^ k1;
        xa1 = (uint32_t)pa1; xa3 = (uint32_t)pa0; xa0 = na0; xa2 = na2;
        xb1 = (uint32_t)pb1; xb3 = (uint32_t)pb0; xb0 = nb0; xb2 = nb2;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    ra = xa0;
    rb = xb0;
}

// philox2_w0_key with the keys of rounds 2..9 read from rk (rk[0][r-2] = k0 + r W0,
// rk[1][r-2] = k1 + r W1), for callers that keep them in the kernel's parameter
// space, where an operand costs no instruction.
__device__ __forceinline__ void philox2_w0_rk(uint32_t a0, uint32_t b0, const DrawKey &d, const uint32_t (&rk)[2][8],
                                              uint32_t &ra, uint32_t &rb)
{
    const unsigned long long qa = (unsigned long long)a0 * kPhiloxM0;
    const unsigned long long qb = (unsigned long long)b0 * kPhiloxM0;
    const uint32_t a2r = (uint32_t)(qa >> 32) ^ d.sk, b2r = (uint32_t)(qb >> 32) ^ d.sk;
    const unsigned long long ta = (unsigned long long)a2r * kPhiloxM1;
    const unsigned long long tb = (unsigned long long)b2r * kPhiloxM1;
    uint32_t xa0 = (uint32_t)(ta >> 32) ^ d.bk, xa1 = (uint32_t)ta, xa2 = d.hk ^ (uint32_t)qa, xa3 = d.la;
    uint32_t xb0 = (uint32_t)(tb >> 32) ^ d.bk, xb1 = (uint32_t)tb, xb2 = d.hk ^ (uint32_t)qb, xb3 = d.la;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const unsigned long long pa0 = (unsigned long long)xa0 * kPhiloxM0;
        const unsigned long long pa1 = (unsigned long long)xa2 * kPhiloxM1;
        const unsigned long long pb0 = (unsigned long long)xb0 * kPhiloxM0;
        const unsigned long long pb1 = (unsigned long long)xb2 * kPhiloxM1;
        const uint32_t na0 = (uint32_t)(pa1 >> 32) ^ xa1 ^ rk[0][r];
        const uint32_t na2 = (uint32_t)(pa0 >> 32) ^ xa3 ^ rk[1][r];
        const uint32_t nb0 = (uint32_t)(pb1 >> 32) ^ xb1 ^ rk[0][r];
        const uint32_t nb2 = (uint32_t)(pb0 >> 32) ^ xb3 ^ rk[1][r];
        xa1 = (uint32_t)pa1; xa3 = (uint32_t)pa0; xa0 = na0; xa2 = na2;
        xb1 = (uint32_t)pb1; xb3 = (uint32_t)pb0; xb0 = nb0; xb2 = nb2;
    }
    ra = xa0;
    rb = xb0;
}

__device__ __forceinline__ uint32_t philox_w0_rk(uint32_t a0, const DrawKey &d, const uint32_t (&rk)[2][8])
{
    const unsigned long long qa = (unsigned long long)a0 * kPhiloxM0;
    const uint32_t a2r = (uint32_t)(qa >> 32) ^ d.sk;
    const unsigned long long ta = (unsigned long long)a2r * kPhiloxM1;
    uint32_t x0 = (uint32_t)(ta >> 32) ^ d.bk, x1 = (uint32_t)ta, x2 = d.hk ^ (uint32_t)qa, x3 = d.la;
#pragma unroll
    for (int r = 0; r < 8; ++r) philox_round(x0, x1, x2, x3, rk[0][r], rk[1][r]);
    return x0;
}

// Word 0 of one counter {a0, f, s_lo, s_hi} with the phase's DrawKey.
__device__ __forceinline__ uint32_t philox_w0_key(uint32_t a0, const DrawKey &d)
{
    const unsigned long long qa = (unsigned long long)a0 * kPhiloxM0;
    const uint32_t a2r = (uint32_t)(qa >> 32) ^ d.sk;
    const unsigned long long ta = (unsigned long long)a2r * kPhiloxM1;
    uint32_t x0 = (uint32_t)(ta >> 32) ^ d.bk, x1 = (uint32_t)ta, x2 = d.hk ^ (uint32_t)qa, x3 = d.la;
    uint32_t k0 = d.k0 + 2u * kPhiloxW0, k1 = d.k1 + 2u * kPhiloxW1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        philox_round(x0, x1, x2, x3, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return x0;
}

}  // namespace klmc
