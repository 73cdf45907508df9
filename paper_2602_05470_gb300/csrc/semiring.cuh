// Counting max-plus semiring on the device.
//
// Paper Eq. (2) is the min-sum tropical contraction; the counting paragraph after
// it pairs every value with the number of configurations attaining it, and the
// MWIS paragraph encodes hard constraints as (infinity, 0). The library contracts
// the max-plus network of the negated energies, so
//   (a, c) (+) (b, d) = (max(a, b), c + d if a == b else the count of the larger)
//   (a, c) (x) (b, d) = (a + b, c * d)
// Counts are residues in 64-bit words, one word per count plane, in one of two forms:
//  - wide: one residue modulo a prime p = 2^61 - c with c < 2^10;
//  - pair: two residues, the low 32 bits modulo q0 = 2^30 - d0 and the high 32 bits
//    modulo q1 = 2^30 - d1 (d0, d1 < 2^10). A product of two pair residues is two
//    32 x 32 -> 64-bit multiplies, and sixteen of them sum without overflow, where a
//    wide product needs a 64 x 64 -> 128-bit multiply.
// A plane's form and constants travel in one 32-bit word `c`: c < 2^10 is the wide
// prime's c; c = kPairFlag | d0 | d1 << 10 is a pair.
#pragma once
#include <stdint.h>

namespace bbtn {

constexpr int32_t kNeg = -(1 << 29);        // -infinity sentinel, count 0
constexpr int32_t kFiniteMin = -(1 << 28);  // below: infeasible
constexpr uint64_t kM61 = (1ull << 61) - 1;
constexpr int kMaxPlanes = 9;               // up to 8 CRT primes + 1 check prime

typedef unsigned __int128 u128;

// a * b mod p for p = 2^61 - c, a, b < p, c < 2^10.
// x = q 2^61 + r == r + c q (mod p) because 2^61 == c; folding twice leaves a
// value below 2^61 + 2^21 < 2p, fixed by one conditional subtraction.
__host__ __device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b, uint32_t c) {
    const uint64_t p = (1ull << 61) - c;
    u128 x = (u128)a * b;
    uint64_t r = (uint64_t)x & kM61;
    uint64_t q = (uint64_t)(x >> 61);
    u128 y = (u128)q * (uint64_t)c + r;
    uint64_t yr = (uint64_t)y & kM61;
    uint64_t yq = (uint64_t)(y >> 61);
    uint64_t z = yr + yq * (uint64_t)c;
    return z >= p ? z - p : z;
}

// x mod p for p = 2^61 - c, any x < 2^128 (same folding as mulmod61, one more round).
__host__ __device__ __forceinline__ uint64_t reduce128_61(u128 x, uint32_t c) {
    const uint64_t p = (1ull << 61) - c;
    // x = q 2^61 + r, q < 2^67: fold q * c (< 2^77) + r, then as in mulmod61
    u128 y = (u128)(uint64_t)(x >> 61) * (uint64_t)c + ((uint64_t)x & kM61) + ((u128)(uint64_t)(x >> 125) << 64) * c;
    uint64_t r = (uint64_t)y & kM61;
    u128 z = (u128)(uint64_t)(y >> 61) * (uint64_t)c + r;      // y >> 61 < 2^17
    uint64_t zr = (uint64_t)z & kM61;
    uint64_t zq = (uint64_t)(z >> 61);
    uint64_t w = zr + zq * (uint64_t)c;
    return w >= p ? w - p : w;
}

__host__ __device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b, uint32_t c) {
    const uint64_t p = (1ull << 61) - c;
    uint64_t s = a + b;                // < 2^62, no wrap
    return s >= p ? s - p : s;
}

constexpr uint32_t kPairFlag = 1u << 31;
constexpr uint64_t kM30 = (1ull << 30) - 1;

__host__ __device__ __forceinline__ bool is_pair(uint32_t c) { return (c & kPairFlag) != 0; }
__host__ __device__ __forceinline__ uint32_t pair_d0(uint32_t c) { return c & 1023u; }
__host__ __device__ __forceinline__ uint32_t pair_d1(uint32_t c) { return (c >> 10) & 1023u; }

// x mod q for q = 2^30 - d, d < 2^10, any x < 2^64: 2^30 == d (mod q), so
// x = h 2^30 + l == h d + l; h < 2^34 gives y < 2^44 + 2^30, and folding y once more
// gives z < 2^30 + 2^25 < 2q, fixed by one conditional subtraction.
__host__ __device__ __forceinline__ uint32_t fold64_30(uint64_t x, uint32_t d) {
    const uint64_t y = (x >> 30) * d + (x & kM30);
    return (uint32_t)(y >> 30) * d + (uint32_t)(y & kM30);
}

__host__ __device__ __forceinline__ uint32_t reduce64_30(uint64_t x, uint32_t d) {
    const uint32_t z = fold64_30(x, d);   // z < 2q, congruent to x
    const uint32_t q = (1u << 30) - d;
    return z >= q ? z - q : z;
}

__host__ __device__ __forceinline__ uint64_t mulmod_pair(uint64_t a, uint64_t b, uint32_t c) {
    const uint32_t lo = reduce64_30((uint64_t)(uint32_t)a * (uint32_t)b, pair_d0(c));
    const uint32_t hi = reduce64_30((a >> 32) * (b >> 32), pair_d1(c));
    return (uint64_t)hi << 32 | lo;
}

// both halves below 2^30, so their sums do not carry into each other
__host__ __device__ __forceinline__ uint64_t addmod_pair(uint64_t a, uint64_t b, uint32_t c) {
    uint64_t s = a + b;
    const uint32_t q0 = (1u << 30) - pair_d0(c), q1 = (1u << 30) - pair_d1(c);
    if ((uint32_t)s >= q0) s -= q0;
    if ((uint32_t)(s >> 32) >= q1) s -= (uint64_t)q1 << 32;
    return s;
}

// the count 1 of a plane, and the semiring product / sum of two residue words
__host__ __device__ __forceinline__ uint64_t count_one(uint32_t c) { return is_pair(c) ? 0x100000001ull : 1ull; }

// the same with the form fixed at compile time (kernels templated on it keep one code path)
template <bool PR>
__host__ __device__ __forceinline__ uint64_t rmul(uint64_t a, uint64_t b, uint32_t c) {
    if constexpr (PR) return mulmod_pair(a, b, c);
    else return mulmod61(a, b, c);
}
template <bool PR>
__host__ __device__ __forceinline__ uint64_t radd(uint64_t a, uint64_t b, uint32_t c) {
    if constexpr (PR) return addmod_pair(a, b, c);
    else return addmod61(a, b, c);
}
template <bool PR>
__host__ __device__ constexpr uint64_t rone() { return PR ? 0x100000001ull : 1ull; }

__host__ __device__ __forceinline__ uint64_t cmul(uint64_t a, uint64_t b, uint32_t c) {
    return is_pair(c) ? mulmod_pair(a, b, c) : mulmod61(a, b, c);
}

__host__ __device__ __forceinline__ uint64_t cadd(uint64_t a, uint64_t b, uint32_t c) {
    return is_pair(c) ? addmod_pair(a, b, c) : addmod61(a, b, c);
}

}  // namespace bbtn
