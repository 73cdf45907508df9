// Counting max-plus semiring on the device.
//
// Paper Eq. (2) is the min-sum tropical contraction; the counting paragraph after
// it pairs every value with the number of configurations attaining it, and the
// MWIS paragraph encodes hard constraints as (infinity, 0). The library contracts
// the max-plus network of the negated energies, so
//   (a, c) (+) (b, d) = (max(a, b), c + d if a == b else the count of the larger)
//   (a, c) (x) (b, d) = (a + b, c * d)
// Counts are residues modulo primes p = 2^61 - c with c < 2^10.
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

}  // namespace bbtn
