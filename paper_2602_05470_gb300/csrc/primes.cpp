// Count residues: prime selection (deterministic Miller-Rabin) and Chinese-remainder
// recombination (Garner's mixed-radix algorithm) into an exact big integer.
#include <mutex>

#include "common.h"
#include "semiring.cuh"

namespace bbtn {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string &msg) { g_err = msg; }
const char *get_error() { return g_err.c_str(); }

typedef unsigned __int128 u128;

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

uint64_t powmod_host(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod_host(r, a, p);
        a = mulmod_host(a, a, p);
        e >>= 1;
    }
    return r;
}

// Deterministic for all 64-bit n with the first twelve prime bases.
bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t q : small) {
        if (n % q == 0) return n == q;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (uint64_t a : small) {
        uint64_t x = powmod_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; i++) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

const std::vector<uint64_t> &prime_table() {
    static std::vector<uint64_t> tab;
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint64_t c = 1; tab.size() < (size_t)BBTN_MAX_PRIMES + 1 && c < 1024; c++) {
            uint64_t p = (1ull << 61) - c;
            if (is_prime_u64(p)) tab.push_back(p);
        }
    });
    return tab;
}

const std::vector<uint64_t> &pair_prime_table() {
    static std::vector<uint64_t> tab;
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint64_t d = 1; tab.size() < 2 * ((size_t)BBTN_MAX_PRIMES + 1) && d < 1024; d++) {
            uint64_t q = (1ull << 30) - d;
            if (is_prime_u64(q)) tab.push_back(q);
        }
    });
    return tab;
}

// A plane's modulus word: a prime 2^61 - c (one residue per word), or a pair
// q1 << 32 | q0 of distinct primes 2^30 - d (two residues per word); every plane of
// one call takes the same form.
void plane_moduli(int np, const uint64_t *primes, uint32_t *c) {
    if (np < 0 || np > kMaxPlanes) fail(BBTN_EINVAL, "np out of range");
    if (np > 0 && !primes) fail(BBTN_EINVAL, "primes missing");
    auto small = [](uint64_t q) { return q < (1ull << 30) && (1ull << 30) - q < 1024 && is_prime_u64(q); };
    for (int t = 0; t < np; t++) {
        const uint64_t m = primes[t];
        if (m >= (1ull << 61)) {
            const uint64_t q0 = m & 0xffffffffull, q1 = m >> 32;
            if (!small(q0) || !small(q1) || q0 == q1)
                fail(BBTN_EINVAL, "a pair modulus must be q1 << 32 | q0, distinct primes 2^30 - d with d < 1024");
            c[t] = kPairFlag | (uint32_t)((1ull << 30) - q0) | (uint32_t)((1ull << 30) - q1) << 10;
        } else {
            uint64_t cc = (1ull << 61) - m;
            if (cc >= 1024 || !is_prime_u64(m)) fail(BBTN_EINVAL, "primes must be primes 2^61 - c with c < 1024");
            c[t] = (uint32_t)cc;
        }
        if (is_pair(c[t]) != is_pair(c[0])) fail(BBTN_EINVAL, "all count planes of a call take the same modulus form");
    }
}

namespace {
// little-endian base-2^32 big integer
struct Big {
    std::vector<uint32_t> d;
    void mul_add(uint64_t m, uint64_t a) {   // *this = *this * m + a
        u128 carry = a;
        for (auto &x : d) {
            u128 t = (u128)x * m + carry;
            x = (uint32_t)t;
            carry = t >> 32;
        }
        while (carry) {
            d.push_back((uint32_t)carry);
            carry >>= 32;
        }
    }
    bool zero() const {
        for (auto x : d) if (x) return false;
        return true;
    }
    uint32_t divmod(uint32_t q) {          // *this /= q, return remainder
        uint64_t rem = 0;
        for (size_t i = d.size(); i-- > 0;) {
            uint64_t cur = (rem << 32) | d[i];
            d[i] = (uint32_t)(cur / q);
            rem = cur % q;
        }
        return (uint32_t)rem;
    }
};

std::vector<uint64_t> garner_digits(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p) {
    const size_t k = r.size();
    std::vector<uint64_t> x(k);
    for (size_t i = 0; i < k; i++) {
        uint64_t xi = r[i] % p[i];
        for (size_t j = 0; j < i; j++) {
            uint64_t inv = powmod_host(p[j] % p[i], p[i] - 2, p[i]);   // p[i] prime
            uint64_t diff = (xi + p[i] - x[j] % p[i]) % p[i];
            xi = mulmod_host(diff, inv, p[i]);
        }
        x[i] = xi;
    }
    return x;
}
}  // namespace

std::string crt_decimal(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p) {
    if (r.empty()) return "0";
    std::vector<uint64_t> x = garner_digits(r, p);
    // value = x0 + p0 (x1 + p1 (x2 + ...)): Horner from the top digit
    Big b;
    b.d.assign(1, 0);
    for (size_t i = x.size(); i-- > 0;) b.mul_add(p[i], x[i]);   // first step multiplies 0
    if (b.zero()) return "0";
    std::string s;
    while (!b.zero()) {
        uint32_t rem = b.divmod(1000000000u);
        char buf[16];
        snprintf(buf, sizeof buf, "%09u", rem);
        s = std::string(buf) + s;
    }
    size_t nz = s.find_first_not_of('0');
    return nz == std::string::npos ? "0" : s.substr(nz);
}

uint64_t crt_mod(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p, uint64_t q) {
    std::vector<uint64_t> x = garner_digits(r, p);
    uint64_t acc = 0;
    for (size_t i = x.size(); i-- > 0;) {
        acc = mulmod_host(acc, p[i] % q, q);
        acc = (acc + x[i] % q) % q;
    }
    return acc;
}

}  // namespace bbtn
